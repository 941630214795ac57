"""Checks of the seeded input generators (turbulence statistics, sensor, workloads)."""

import math

import numpy as np
from scipy import integrate, special

from synth import TruthStream, VKScreen, vk_phase_covariance, vk_structure_function_kolmogorov, workload
from synth.turbulence import vk_psd


def test_vk_covariance_is_hankel_transform_of_psd():
    r0, L0 = 0.5, 25.0
    var = integrate.quad(lambda f: 2 * math.pi * f * vk_psd(f * f, r0, L0), 0, np.inf, limit=500)[0]
    # 0.023 is the rounded PSD constant, so agreement is at the 1 % level
    assert abs(vk_phase_covariance(np.array([0.0]), r0, L0)[0] / var - 1) < 0.01
    c1 = integrate.quad(lambda f: 2 * math.pi * f * vk_psd(f * f, r0, L0) * special.j0(2 * math.pi * f),
                        0, 50, limit=2000)[0]
    assert abs(vk_phase_covariance(np.array([1.0]), r0, L0)[0] / c1 - 1) < 0.01


def test_structure_function_kolmogorov_limit():
    # r << L0: D(r) = 6.88 (r/r0)^(5/3) [1 - 1.485 (r/L0)^(1/3) + ...] (first outer-scale term)
    for r0, L0 in [(0.3, 1e5), (0.5, 25.0)]:
        r = np.array([0.01, 0.05, 0.2]) if L0 > 1e3 else np.array([0.001, 0.003, 0.01])
        C0 = vk_phase_covariance(np.array([0.0]), r0, L0)[0]
        Dr = 2 * (C0 - vk_phase_covariance(r, r0, L0))
        ref = vk_structure_function_kolmogorov(r, r0) * (1 - 1.485 * (r / L0) ** (1 / 3))
        assert np.allclose(Dr / ref, 1.0, rtol=2e-3)


def test_fft_screen_structure_function():
    r0, L0, dx = 0.5, 25.0, 0.125
    scr = VKScreen(1024, dx, r0, L0, seed=4)
    C0 = vk_phase_covariance(np.array([0.0]), r0, L0)[0]
    for lag in (2, 4, 8, 32):   # lag 1 misses the power above the grid Nyquist frequency
        emp = np.mean((scr.phase[:, lag:] - scr.phase[:, :-lag]) ** 2)
        ref = 2 * (C0 - vk_phase_covariance(np.array([lag * dx]), r0, L0)[0])
        assert abs(emp / ref - 1) < 0.1


def test_process_noise_is_frozen_flow_innovation_covariance():
    w = workload("tiny-8x8")
    rc = np.array([(r, c) for r in range(3) for c in range(3)])
    L = w.process_noise_sqrt(rc, jitter=0.0)
    P = rc[:, ::-1] * w.pitch
    s = np.array([w.wind / w.frame_rate, 0.0])
    a = w.ar1_a
    # brute force: Cov(phi_{k+1}(i) - a phi_k(i), phi_{k+1}(j) - a phi_k(j)), phi_{k+1}(x) = phi_k(x - s)
    Q = np.zeros((9, 9))
    for i in range(9):
        for j in range(9):
            c = lambda u, v: vk_phase_covariance(np.array([np.linalg.norm(u - v)]), w.r0, w.L0)[0]
            Q[i, j] = (c(P[i] - s, P[j] - s) - a * c(P[i] - s, P[j]) - a * c(P[i], P[j] - s)
                       + a * a * c(P[i], P[j]))
    assert np.allclose(L @ L.T, Q, rtol=1e-8, atol=1e-12)


def test_truth_stream_shapes_and_determinism():
    w = workload("tiny-8x8")
    a = TruthStream(w).frames(0, 3)
    b = TruthStream(w).frames(0, 3)
    assert a["slopes"].shape == (3, 2, 8, 8) and a["phi_act"].shape == (3, 9, 9)
    assert np.array_equal(a["slopes"], b["slopes"]) and np.array_equal(a["phi_act"], b["phi_act"])
    # frozen flow: consecutive frames differ by a small shift of the same screen
    d = np.std(a["phi_act"][1] - a["phi_act"][0])
    assert 0 < d < 0.5 * np.std(a["phi_act"][0])


def test_ar2_process_noise_is_the_ar2_innovation_covariance():
    import dataclasses
    w = dataclasses.replace(workload("tiny-8x8"), ar1_a=1.6, ar2_a=-0.65)
    rc = np.array([(r, c) for r in range(3) for c in range(3)])
    L = w.process_noise_sqrt(rc, jitter=0.0)
    P = rc[:, ::-1] * w.pitch
    s = np.array([w.wind / w.frame_rate, 0.0])
    a, a2 = w.ar1_a, w.ar2_a
    # brute force: e = phi_{k+1} - a phi_k - a2 phi_{k-1} with phi_{k+j}(x) = phi_k(x - j s)
    cov = lambda u, v: vk_phase_covariance(np.array([np.linalg.norm(u - v)]), w.r0, w.L0)[0]
    coef = [1.0, -a, -a2]           # weights of phi_{k+1}, phi_k, phi_{k-1}
    Q = np.zeros((9, 9))
    for i in range(9):
        for j in range(9):
            Q[i, j] = sum(coef[p] * coef[q] * cov(P[i] - (1 - p) * s, P[j] - (1 - q) * s)
                          for p in range(3) for q in range(3))
    assert np.allclose(L @ L.T, Q, rtol=1e-8, atol=1e-12)


def test_yule_walker_recovers_a_known_ar2_process():
    from synth import yule_walker_ar2
    a1, a2 = 1.5, -0.6
    # autocovariances of x_k = a1 x_{k-1} + a2 x_{k-2} + e_k (unit e): closed form
    g0 = (1 - a2) / ((1 + a2) * ((1 - a2) ** 2 - a1 ** 2))
    g1 = a1 * g0 / (1 - a2)
    g2 = a1 * g1 + a2 * g0
    b1, b2 = yule_walker_ar2(g0, g1, g2)
    assert abs(b1 - a1) < 1e-12 and abs(b2 - a2) < 1e-12
    # the fit of the frozen-flow workload is a stable AR(2)
    from oracle import geometry
    w = workload("vlt-40x40")
    g = geometry.make_geometry(w.n_sub, w.obstruction)
    f1, f2 = w.ar2_fit(g.act_rc)
    assert abs(f2) < 1 and f1 + f2 < 1 and f2 - f1 < 1


def test_lag_table_entries_are_the_covariance_at_the_shifted_lag():
    from synth import actuator_covariance_lag_table, vk_phase_covariance
    n, pitch, r0, L0, shift = 5, 0.5, 0.3, 25.0, (0.07, -0.02)
    T = actuator_covariance_lag_table(n, pitch, r0, L0, shift)
    assert T.shape == (2 * n - 1, 2 * n - 1)
    for dr in range(-(n - 1), n):
        for dc in range(-(n - 1), n):
            r = np.hypot(pitch * dc + shift[0], pitch * dr + shift[1])
            assert math.isclose(T[dr + n - 1, dc + n - 1], float(vk_phase_covariance(np.array(r), r0, L0)), rel_tol=1e-12)


def test_nonstationary_schedule():
    # the non-stationary ELT run: r0 halves at frame 3000 (phase std x 2^(5/6)), the wind goes
    # linearly from 10 m/s along x to 25 m/s along y over frames 6000-7000, the slope noise steps
    # from 0.1 to 0.3 rad at frame 8000; stationary workloads ignore the schedule
    w = workload("elt-80x80-nonstationary")
    assert w.screen_scale(2999) == 1.0 and math.isclose(w.screen_scale(3000), 2.0 ** (5.0 / 6.0))
    assert w.wind_at(5999) == (10.0, 0.0) and w.wind_at(7000) == (25.0, math.pi / 2)
    v, ang = w.wind_at(6500)
    assert math.isclose(v, 17.5) and math.isclose(ang, math.pi / 4)
    assert w.sigma_at(7999) == 0.1 and w.sigma_at(8000) == 0.3
    s = workload("elt-80x80")
    assert s.screen_scale(5000) == 1.0 and s.wind_at(6500) == (s.wind, s.wind_angle) and s.sigma_at(9000) == s.sigma
    assert s.layer_list() == ((1.0, s.wind, s.wind_angle),)
