"""Pins of the oracle's differential-piston removal (oracle.piston; Sect. 3.1, Sect. 5): planted
per-domain pistons are recovered exactly from noise-free slopes, the fit satisfies its normal
equations and adds no piston, a KKT solve of the constrained least-squares problem agrees, a single
domain needs no correction, and on the tiny workload the correction lowers the residual (the
paper's observation for Fig. 3)."""

import numpy as np
import pytest

from oracle import etkf, geometry, piston
from oracle.fried import fried_matrix

CASES = [(8, 0.0, 4, 1), (16, 0.0, 4, 2), (24, 0.2, 4, 2), (20, 0.1, 5, 1)]


def _setup(n_sub, obstruction, b, h):
    g = geometry.make_geometry(n_sub, obstruction)
    return g, geometry.make_domains(g, b, h)


@pytest.mark.parametrize("case", CASES)
def test_planted_pistons_recovered(case):
    g, doms = _setup(*case)
    rng = np.random.default_rng(7)
    phi = rng.standard_normal(g.n_act)
    y = fried_matrix(g) @ phi
    c = rng.standard_normal(len(doms)) * 3.0
    P = piston.ownership(g, doms)
    x = phi + P @ c
    xc = piston.remove_differential_pistons(x, y, g, doms)
    # the pistons are identified up to one constant, fixed by adding no piston to x
    kappa = (P @ c).sum() / g.n_act
    np.testing.assert_allclose(xc - phi, kappa, atol=1e-10)


@pytest.mark.parametrize("case", CASES)
def test_normal_equations_gauge_idempotent(case):
    g, doms = _setup(*case)
    rng = np.random.default_rng(11)
    x = rng.standard_normal(g.n_act)
    y = rng.standard_normal(2 * g.n_subv)
    D = fried_matrix(g)
    P = piston.ownership(g, doms)
    xc = piston.remove_differential_pistons(x, y, g, doms)
    assert np.abs((D @ P).T @ (y - D @ xc)).max() < 1e-9
    assert abs((xc - x).sum()) < 1e-9
    assert np.abs(piston.differential_pistons(xc, y, g, doms)).max() < 1e-9
    assert len(np.unique(piston.domain_groups(g, doms))) == 1


def test_kkt_and_brute_force_minimum():
    g, doms = _setup(8, 0.0, 4, 1)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(g.n_act)
    y = rng.standard_normal(2 * g.n_subv)
    D = fried_matrix(g)
    P = piston.ownership(g, doms)
    A = D @ P
    r = y - D @ x
    n_own = P.sum(axis=0)
    nd = len(doms)
    # minimise ||r - A delta||^2 subject to n_own . delta = 0 via its KKT system
    K = np.zeros((nd + 1, nd + 1))
    K[:nd, :nd] = A.T @ A
    K[:nd, nd] = n_own
    K[nd, :nd] = n_own
    rhs = np.concatenate([A.T @ r, [0.0]])
    d_kkt = np.linalg.solve(K, rhs)[:nd]
    d = piston.differential_pistons(x, y, g, doms)
    np.testing.assert_allclose(d, d_kkt, atol=1e-10)
    cost = np.sum((r - A @ d) ** 2)
    for _ in range(200):
        e = rng.standard_normal(nd) * 0.1
        e -= np.dot(n_own, e) / n_own.sum()
        assert np.sum((r - A @ (d + e)) ** 2) >= cost - 1e-12


def test_single_domain_needs_no_correction():
    g = geometry.make_geometry(8, 0.0)
    doms = geometry.make_domains(g, 8, 0)
    assert len(doms) == 1
    rng = np.random.default_rng(5)
    x = rng.standard_normal(g.n_act)
    y = rng.standard_normal(2 * g.n_subv)
    assert np.abs(piston.differential_pistons(x, y, g, doms)).max() == 0.0


def test_filter_modes_and_residual():
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from _gpu_common import model, slopes
    w, g, doms, L, Ls = model("tiny-8x8")
    n_fr, burn = 300, 100
    y, phi = slopes("tiny-8x8", n_fr)
    rms = {}
    for mode in ("off", "output", "in_loop"):
        o = etkf.OracleFilter(g, doms, w.m, w.ar1_a, w.sigma, seed=w.seed, L=L, L_stat=Ls, piston=mode)
        pred = np.array([o.step(y[k]) for k in range(n_fr)])
        e = phi[1:n_fr + 1] - pred
        e -= e.mean(axis=1, keepdims=True)
        rms[mode] = float(np.sqrt(np.mean(e[burn:] ** 2)))
        if mode == "output":
            # output mode leaves the ensemble as the filter without correction would
            o2 = etkf.OracleFilter(g, doms, w.m, w.ar1_a, w.sigma, seed=w.seed, L=L, L_stat=Ls)
            for k in range(n_fr):
                o2.step(y[k])
            np.testing.assert_array_equal(o.X, o2.X)
    assert rms["output"] < rms["off"] and rms["in_loop"] < rms["off"]
    with pytest.raises(ValueError):
        etkf.OracleFilter(g, None, w.m, w.ar1_a, w.sigma, seed=w.seed, L=L, piston="output")
