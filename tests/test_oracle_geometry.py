"""Pins of the oracle's geometry and Fried operator (Sect. 3, Sect. 2.3)."""

import json
import os

import numpy as np
import pytest

from oracle import fried, geometry
from synth.wfs import FineGridSensor

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "paper_counts.json")))["cases"])
def test_valid_counts_match_paper(case):
    g = geometry.make_geometry(case["n_sub"], case["obstruction"])
    assert g.n_act == case["n_act"]
    if "n_subv" in case:
        assert g.n_subv == case["n_subv"]
        assert g.n == case["n"]
        assert g.p == case["p"]


def test_mask_symmetry_and_annulus():
    # the pupil is centred: the masks are invariant under the dihedral symmetries of the grid
    for n, obs in [(16, 0.0), (40, 0.14), (80, 0.28)]:
        s = geometry.subaperture_mask(n, obs)
        assert np.array_equal(s, s[::-1, :]) and np.array_equal(s, s[:, ::-1]) and np.array_equal(s, s.T)
        if obs > 0:
            assert not s[n // 2, n // 2]      # the obstruction removes the centre


def test_brute_force_area_rule():
    # brute force on a tiny grid: exact area fraction by dense sampling agrees away from ties
    n = 8
    s = geometry.subaperture_mask(n, 0.0)
    fine = 400
    t = (np.arange(fine) + 0.5) / fine
    for r in range(n):
        for c in range(n):
            x = c + t[None, :] - n / 2
            y = r + t[:, None] - n / 2
            frac = np.mean(x * x + y * y <= (n / 2) ** 2)
            if abs(frac - 0.5) > 0.02:
                assert s[r, c] == (frac >= 0.5)


def test_domains_partition_actuators():
    for n, obs, b, h in [(8, 0.0, 4, 1), (40, 0.14, 4, 2), (80, 0.28, 4, 2), (16, 0.0, 4, 2)]:
        g = geometry.make_geometry(n, obs)
        doms = geometry.make_domains(g, b, h)
        owned = np.concatenate([d.owned_act for d in doms])
        assert np.array_equal(np.sort(owned), np.arange(g.n_act))  # each actuator owned once
        for d in doms:
            assert d.owned_act.size > 0
            # every observed subaperture lies in the block grown by the halo
            rc = g.sub_rc[d.obs_sub]
            assert np.all(rc[:, 0] >= b * d.I - h) and np.all(rc[:, 0] < b * (d.I + 1) + h)
            assert np.all(rc[:, 1] >= b * d.J - h) and np.all(rc[:, 1] < b * (d.J + 1) + h)


def test_tiny_domain_sizes():
    g = geometry.make_geometry(8, 0.0)
    doms = geometry.make_domains(g, 4, 1)
    assert len(doms) == 4
    assert all(d.obs_sub.size == 22 for d in doms)   # 44 slopes per domain


def test_fried_closed_forms():
    g = geometry.make_geometry(16, 0.0)
    D = fried.fried_matrix(g)
    r, c = g.act_rc[:, 0].astype(float), g.act_rc[:, 1].astype(float)
    ns = g.n_subv
    alpha, beta = 0.37, -1.25
    s = D @ (alpha * c + beta * r)                    # tilt: slopes equal the tilt in every subaperture
    assert np.allclose(s[:ns], alpha, atol=1e-12) and np.allclose(s[ns:], beta, atol=1e-12)
    assert np.allclose(D @ np.ones(g.n_act), 0.0, atol=1e-12)          # piston is invisible
    waffle = (-1.0) ** (g.act_rc[:, 0] + g.act_rc[:, 1])
    assert np.allclose(D @ waffle, 0.0, atol=1e-12)                    # waffle is invisible
    # a single poked actuator in the interior moves exactly four subapertures by +-1/2 in each direction
    k = g.act_index[8, 8]
    e = np.zeros(g.n_act)
    e[k] = 1.0
    sx, sy = (D @ e)[:ns], (D @ e)[ns:]
    assert np.count_nonzero(sx) == 4 and np.allclose(np.sort(sx[sx != 0]), [-0.5, -0.5, 0.5, 0.5])
    assert np.count_nonzero(sy) == 4 and np.allclose(np.sort(sy[sy != 0]), [-0.5, -0.5, 0.5, 0.5])


def test_fried_matches_fine_sensor_at_one_sample_per_pitch():
    # the generator's sensor is an independent code path; with q = 1 it is the corner difference
    rng = np.random.default_rng(7)
    n = 12
    g = geometry.make_geometry(n, 0.1)
    phi = rng.standard_normal((n + 1, n + 1))
    sx, sy, pa = FineGridSensor(n, 1).measure(phi)
    D = fried.fried_matrix(g)
    s = D @ phi[g.act_valid]
    assert np.allclose(s[: g.n_subv], sx[g.sub_valid], atol=1e-12)
    assert np.allclose(s[g.n_subv:], sy[g.sub_valid], atol=1e-12)
    assert np.array_equal(pa, phi)


def test_actuator_mask_brute_force():
    # an actuator (grid corner) is valid iff at least one of the (up to four) subapertures it
    # touches is valid
    rng = np.random.default_rng(7)
    for n in (1, 3, 6):
        sub = rng.random((n, n)) < 0.5
        act = geometry.actuator_mask(sub)
        for i in range(n + 1):
            for j in range(n + 1):
                near = [sub[r, c] for r in (i - 1, i) for c in (j - 1, j) if 0 <= r < n and 0 <= c < n]
                assert act[i, j] == any(near), (n, i, j)


# Domain statistics of the workloads' systems under the reading above (half-illumination rule,
# 4 x 4 blocks, last actuator row/column folded), counted independently of this module when the
# hot-path scope was fixed: (N, obstruction, halo) -> (valid subapertures, valid actuators,
# domains, n_loc min/median/max, p_loc min/median/max, sum p_loc); n_loc counts both state
# instants, p_loc both slope directions.
DOMAIN_STATS = [
    ((8, 0.0, 1), (52, 69, 4, (26, 34, 44), (44, 44, 44), 176)),
    ((40, 0.14, 2), (1240, 1332, 92, (2, 32, 40), (16, 124, 128), 9472)),
    ((80, 0.28, 2), (4632, 4836, 332, (2, 32, 40), (16, 128, 128), 36328)),
    ((16, 0.0, 2), (208, 241, 16, (12, 32, 40), (48, 88, 128), 1408)),
    ((32, 0.10, 2), (808, 876, 60, (6, 32, 40), (38, 120, 128), 6088)),
    ((64, 0.20, 2), (3104, 3256, 222, (2, 32, 40), (14, 128, 128), 24188)),
    ((100, 0.28, 2), (7244, 7500, 505, (2, 32, 40), (20, 128, 128), 57028)),
]


@pytest.mark.parametrize("key,want", DOMAIN_STATS)
def test_domain_statistics_of_the_workload_systems(key, want):
    n, obs, h = key
    g = geometry.make_geometry(n, obs)
    doms = geometry.make_domains(g, 4, h)
    nl = [2 * d.owned_act.size for d in doms]
    pl = [2 * d.obs_sub.size for d in doms]
    got = (g.n_subv, g.n_act, len(doms), (min(nl), int(np.median(nl)), max(nl)),
           (min(pl), int(np.median(pl)), max(pl)), sum(pl))
    assert got == want


@pytest.mark.parametrize("n,obs,b,h,off", [(8, 0.0, 4, 1, 0), (8, 0.0, 4, 0, 0), (13, 0.2, 4, 2, 0),
                                           (40, 0.14, 4, 2, 0), (80, 0.28, 4, 2, 0), (10, 0.0, 3, 1, 0),
                                           (9, 0.3, 5, 3, 0), (8, 0.0, 4, 1, 2), (40, 0.14, 4, 2, 2),
                                           (13, 0.2, 4, 2, 3), (10, 0.0, 3, 1, 1)])
def test_domains_equal_brute_force_membership(n, obs, b, h, off):
    """Every domain's owned actuators and observed subapertures equal a brute-force membership test
    written per element (distance of the element's grid cell to the block, clipped to the grid),
    so a dropped or extra halo row or column, at the grid edge or inside, fails.  Also for block
    grids shifted by `off` subapertures (the second partition of Sect. 5)."""
    g = geometry.make_geometry(n, obs)
    doms = geometry.make_domains(g, b, h, offset=off)
    by_block = {(d.I, d.J): d for d in doms}
    # owned actuators: an actuator (r, c) belongs to the block whose span of subaperture rows and
    # columns, [b I - off, b (I + 1) - off), contains it; the corner row/column n lies past the
    # last subaperture row and belongs to that row's block
    def block_of(r):
        return (min(r, n - 1) + off) // b
    want_owned = {}
    for k, (r, c) in enumerate(g.act_rc):
        want_owned.setdefault((block_of(r), block_of(c)), set()).add(k)
    assert set(by_block) == set(want_owned)          # no block without valid actuators is kept
    for IJ, d in by_block.items():
        assert set(d.owned_act.tolist()) == want_owned[IJ]
        assert np.all(np.diff(d.owned_act) > 0)
        # observed subapertures: valid, and the Chebyshev gap between the subaperture's cell and
        # the block's cells is at most the halo in each direction
        I, J = IJ
        want = set()
        for k, (r, c) in enumerate(g.sub_rc):
            gap_r = max(b * I - off - r, r - (b * (I + 1) - off - 1), 0)
            gap_c = max(b * J - off - c, c - (b * (J + 1) - off - 1), 0)
            if gap_r <= h and gap_c <= h:
                want.add(k)
        assert set(d.obs_sub.tolist()) == want, (IJ, sorted(want ^ set(d.obs_sub.tolist())))
        assert np.all(np.diff(d.obs_sub) > 0)
