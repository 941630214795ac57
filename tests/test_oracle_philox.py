"""Pins of the oracle's counter-based generator (Philox4x32-10 + Box-Muller)."""

import os

import numpy as np
from scipy import stats

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_known_answer_vectors():
    for ctr, key, out in _kat():
        got = philox.philox4x32_10(np.array(ctr, dtype=np.uint32), np.array(key, dtype=np.uint32))
        assert [int(x) for x in got] == out


def test_vectorised_equals_scalar_calls():
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(17, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(17, 2), dtype=np.uint64).astype(np.uint32)
    batch = philox.philox4x32_10(ctr, key)
    for i in range(17):
        assert np.array_equal(batch[i], philox.philox4x32_10(ctr[i], key[i]))


def test_normals_layout_and_distribution():
    z = philox.normals(seed=1310595400, stream=1, frame=5, m=64, count=1001)
    assert z.shape == (1001, 64)
    # a member's column is a prefix of the same stream drawn with a larger count
    z2 = philox.normals(seed=1310595400, stream=1, frame=5, m=64, count=1024)
    assert np.array_equal(z, z2[:1001])
    # distinct streams / frames / members differ
    assert not np.allclose(z2, philox.normals(1310595400, 0, 5, 64, 1024))
    assert not np.allclose(z2, philox.normals(1310595400, 1, 6, 64, 1024))
    flat = z2.ravel()
    assert abs(flat.mean()) < 5.0 / np.sqrt(flat.size)
    assert abs(flat.var() - 1.0) < 5.0 * np.sqrt(2.0 / flat.size)
    assert stats.kstest(flat, "norm").pvalue > 1e-4


def test_box_muller_invariants():
    # radius and angle of each output pair recover the two uniforms: r^2 = -2 ln u_a, angle = 2 pi u_b
    rng = np.random.default_rng(5)
    wa = rng.integers(0, 2 ** 32, size=1000, dtype=np.uint64).astype(np.uint32)
    wb = rng.integers(0, 2 ** 32, size=1000, dtype=np.uint64).astype(np.uint32)
    z0, z1 = philox.box_muller(wa, wb)
    ua = (wa.astype(np.float64) + 0.5) / 2 ** 32
    ub = (wb.astype(np.float64) + 0.5) / 2 ** 32
    assert np.allclose(z0 ** 2 + z1 ** 2, -2 * np.log(ua), rtol=1e-12)
    ang = np.mod(np.arctan2(z1, z0), 2 * np.pi)
    assert np.allclose(ang, 2 * np.pi * ub, atol=1e-9)
