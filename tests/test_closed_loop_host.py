"""Closed-loop evaluation pieces on the host (Sect. 3): the deformable mirror with coupling 0.3,
the coherent energy, and the multi-layer frozen-flow truth of the paper's 8 m case."""

import math

import numpy as np
import pytest

from paper_1310_5954_gb300.closed_loop import DeformableMirror, coherent_energy
from synth import workload, TruthStream
from oracle import geometry


def _mirror(n_sub=8, obstruction=0.0, q=4):
    g = geometry.make_geometry(n_sub, obstruction)
    return g, DeformableMirror(g.sub_valid, g.act_valid, q)


def test_influence_at_the_actuator_points():
    g, dm = _mirror()
    F = dm.F
    assert np.allclose(np.diag(F), 1.0)
    rc = np.argwhere(g.act_valid)
    d2 = ((rc[:, None, :] - rc[None, :, :]) ** 2).sum(-1)
    assert np.allclose(F[d2 == 1], 0.3)          # nearest neighbours: the coupling factor
    assert np.allclose(F[d2 == 2], 0.09)         # diagonal neighbours
    assert np.all(F[d2 > 9] == 0.0)              # cut beyond three pitches
    assert np.all(np.linalg.eigvalsh(F) > 0)


def test_mirror_passes_through_the_commanded_phase_at_the_actuators():
    g, dm = _mirror(q=4)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(g.n_act)
    surf = np.full(dm.pupil.shape, np.nan)
    surf[dm.pupil] = dm.correction(x)
    ar, ac = np.nonzero(g.act_valid)
    np.testing.assert_allclose(surf[ar * dm.q, ac * dm.q], x, atol=1e-10)


def test_a_mirror_shape_is_corrected_exactly_and_piston_is_ignored():
    g, dm = _mirror(n_sub=8, obstruction=0.2, q=5)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(g.n_act)
    phi = np.zeros(dm.pupil.shape)
    phi[dm.pupil] = dm.correction(x) + 3.7      # the mirror's own shape plus a piston
    assert dm.residual_variance(phi, x) < 1e-20
    # a known residual: the variance of a zero-mean pattern, whatever the piston
    pat = rng.standard_normal(dm.n_pix)
    phi[dm.pupil] = dm.correction(x) + pat + 1.0
    assert math.isclose(dm.residual_variance(phi, x), float(np.var(pat)), rel_tol=1e-12)


def test_pupil_pixels_of_an_unobstructed_grid():
    # every subaperture of an 8x8 grid with q = 4 valid after removing the corners' mask: the pixels
    # touching a valid subaperture are the union of their closed squares
    sub = np.ones((8, 8), dtype=bool)
    sub[0, 0] = False
    act = np.zeros((9, 9), dtype=bool)
    for r, c in np.argwhere(sub):
        act[r:r + 2, c:c + 2] = True
    dm = DeformableMirror(sub, act, 4)
    brute = np.zeros((33, 33), dtype=bool)
    for r, c in np.argwhere(sub):
        brute[4 * r:4 * r + 5, 4 * c:4 * c + 5] = True
    assert np.array_equal(dm.pupil, brute)


def test_coherent_energy_is_the_marechal_average():
    assert coherent_energy([0.0, 0.0]) == 1.0
    assert math.isclose(coherent_energy([0.2, 0.4]), 0.5 * (math.exp(-0.2) + math.exp(-0.4)), rel_tol=1e-15)


def test_layers_add_up_to_the_total_r0():
    # Sect. 3: three layers with relative Cn2 0.5, 0.17, 0.33; r0_l = r0 f^(-3/5), so that
    # sum f_l equals 1 and sum r0_l^(-5/3) = r0^(-5/3)
    w = workload("scao-8m")
    assert math.isclose(sum(f for f, _, _ in w.layers), 1.0, rel_tol=1e-12)
    assert [v for _, v, _ in w.layers] == [7.5, 12.5, 15.0]
    ts = TruthStream(w, n_pix=256)
    assert len(ts.screens) == 3
    assert math.isclose(sum(s.r0 ** (-5.0 / 3.0) for s in ts.screens), w.r0 ** (-5.0 / 3.0), rel_tol=1e-12)
    g = geometry.make_geometry(w.n_sub, w.obstruction)
    assert g.n_act == 241                                    # the paper's count for the 8 m case
    # the zero-lag covariance of the layered turbulence is that of r0 itself
    np.testing.assert_allclose(w._lagged_cov(g.act_rc[:20], 0), w._lag_gather(g.act_rc[:20]), rtol=1e-12)
    # each layer moves at its own speed and direction: the phase a frame later is the sum of the
    # layers' screens, each shifted by its own path
    phi0, phi1 = ts.phase_fine(0), ts.phase_fine(1)
    x, y = ts._xg, ts._yg
    ref = sum(s.sample(x + v / w.frame_rate * math.cos(a), y + v / w.frame_rate * math.sin(a))
              for s, (_, v, a) in zip(ts.screens, w.layers))
    np.testing.assert_allclose(phi1, ref, rtol=1e-12, atol=1e-12)
    assert not np.allclose(phi0, phi1)


def test_pseudo_open_loop_slopes_equal_the_open_loop_ones():
    # Sect. 3 closed loop: the sensor sees the residual phi - (mirror surface); adding back the
    # sensor's response to the known mirror shape (its interaction with the commands) restores the
    # open-loop slopes exactly, because the sensor is linear: the filter's input does not change
    from synth import FineGridSensor
    g, dm = _mirror(n_sub=8, obstruction=0.0, q=4)
    sensor = FineGridSensor(8, 4)
    rng = np.random.default_rng(5)
    phi = rng.standard_normal(dm.pupil.shape)
    x = rng.standard_normal(g.n_act)
    surface = np.zeros(dm.pupil.shape)
    surface[dm.pupil] = dm.correction(x)
    ol = sensor.measure(phi)[:2]
    cl = sensor.measure(phi - surface)[:2]
    response = sensor.measure(surface)[:2]           # the interaction of the commands
    for a, b, c in zip(ol, cl, response):
        np.testing.assert_allclose((b + c)[g.sub_valid], a[g.sub_valid], rtol=0, atol=1e-12)
