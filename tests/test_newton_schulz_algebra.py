"""The coupled Newton-Schulz iteration of the fused and global paths (inverse square root of
A_s = (I + G/c)/s for the transform of Sect. 2.2), checked in FP64 on the host:

  P = Z Y, T = (3I - P)/2, Y <- Y T, Z <- T Z from Y_0 = A_s, Z_0 = I; Z -> A_s^(-1/2).

On an eigenvalue p of P the step is p <- p (3 - p)^2 / 4, so 1 - p_next = 0.75 e^2 + 0.25 e^3 for
e = 1 - p (the predicted last update), and (0, 3) maps into (0, 1]; the scale
s = (1 + ||G||_F / c) / 2.5 keeps every eigenvalue of A_s in (0, 2.5] since ||G||_F bounds the
largest eigenvalue of G.
"""

import numpy as np

from oracle import etkf


def test_error_map_of_one_step():
    e = np.linspace(-1.999, 0.999, 4001)                # p = 1 - e in (0, 3)
    p = 1.0 - e
    p_next = p * (3.0 - p) ** 2 / 4.0
    np.testing.assert_allclose(1.0 - p_next, 0.75 * e ** 2 + 0.25 * e ** 3, rtol=0, atol=1e-14)
    assert np.all(p_next > 0.0) and np.all(p_next <= 1.0 + 1e-15)


def test_scaled_start_lies_in_the_convergence_interval_and_converges_to_the_transform():
    rng = np.random.default_rng(12)
    for p_loc, m, scale in [(128, 100, 1.0), (24, 100, 5.0), (128, 50, 20.0)]:
        Yp = scale * rng.standard_normal((p_loc, m))
        Yp -= Yp.mean(axis=1, keepdims=True)
        sigma, c = 0.2, m - 1.0
        G = Yp.T @ Yp / sigma ** 2
        s_ns = (1.0 + np.linalg.norm(G) / c) / 2.5
        A = (np.eye(m) + G / c) / s_ns
        lam = np.linalg.eigvalsh(A)
        assert lam.min() > 0.0 and lam.max() <= 2.5 * (1 + 1e-12)
        Y, Z = A.copy(), np.eye(m)
        for _ in range(60):
            P = Z @ Y
            if np.linalg.norm(np.eye(m) - P) < 1e-13:
                break
            T = 1.5 * np.eye(m) - 0.5 * P
            Y, Z = Y @ T, T @ Z
        _, T_ref = etkf.ensemble_transform(Yp, np.zeros(p_loc), sigma)
        # T = (I + G/c)^(-1/2) = Z / sqrt(s_ns)
        assert np.abs(Z / np.sqrt(s_ns) - T_ref).max() < 1e-9
