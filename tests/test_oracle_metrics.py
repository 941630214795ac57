"""The performance measure (Sect. 3: residual phase, coherent energy) in the oracle, pinned by
hand-computed values and the Marechal limit, and the benchmark's own residual RMS checked against it."""

import importlib.util
import math
import os

import numpy as np

from oracle import metrics


def test_residual_removes_the_piston():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 7))
    # a prediction off by a constant per frame has no residual (piston is invisible to the sensor)
    assert np.allclose(metrics.residual(x + np.array([[1.0], [-2.0], [0.5]]), x), 0.0, atol=1e-15)
    # a zero-mean error is left as it is
    e = rng.standard_normal((3, 7))
    e -= e.mean(axis=1, keepdims=True)
    np.testing.assert_allclose(metrics.residual(x + e, x), e, atol=1e-15)


def test_residual_variance_by_hand():
    eps = np.array([[1.0, -1.0, 0.0, 0.0], [2.0, 0.0, -2.0, 0.0]])
    # frame 0: (1 + 1) / 4 = 0.5; frame 1: (4 + 4) / 4 = 2; mean over frames 1.25
    assert metrics.residual_variance(eps) == 1.25


def test_coherent_energy_is_marechal():
    assert metrics.coherent_energy(0.0) == 1.0
    assert math.isclose(metrics.coherent_energy(1.0), 1.0 / math.e, rel_tol=1e-15)
    v = 1e-4      # small variance: 1 - v to second order
    assert abs(metrics.coherent_energy(v) - (1.0 - v)) < v * v


def test_benchmark_residual_rms_is_the_oracle_metric():
    spec = importlib.util.spec_from_file_location(
        "bench_mod", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    rng = np.random.default_rng(1)
    n_frames, n_act, burn = 40, 25, 10
    phi = rng.standard_normal((n_frames + 1, n_act))
    pred = phi[1:] + 0.1 * rng.standard_normal((n_frames, n_act)) + 3.0
    ref = metrics.residual_variance(metrics.residual(phi[1:], pred)[burn:])
    assert math.isclose(bench.residual_rms(pred, phi, burn) ** 2, ref, rel_tol=1e-12)
