"""The observation-space (dual) form of the ETKF analysis that the fused kernel uses when the
ensemble is wider than a tensor-core tile, and that its FP32 SIMT analysis uses when a domain has
fewer slopes than members (Sect. 2.2 restated in p-space), checked in FP64 against the oracle's
m x m symmetric square root:

  w_bar = [(m-1)I + S^T S]^-1 S^T d = S^T (cI + K)^-1 d,               K = S S^T, c = m - 1
  T = (I + S^T S / c)^(-1/2) = I - W^T (I + Z)^-1 W,  Z = (I + K/c)^(-1/2),  W = Z S / sqrt(c)
  (I + Z)^-1 by Newton's iteration X <- X (2I - (I + Z) X) from 2/3 I: four steps to 1e-8 (the
  kernel takes the first step elementwise and predicts the last from the residual's square).
"""

import numpy as np
import pytest

from oracle import etkf


def _inv_sqrt(A):
    lam, U = np.linalg.eigh(A)
    return (U / np.sqrt(lam)) @ U.T


@pytest.mark.parametrize("p,m,scale", [(16, 100, 1.0), (52, 100, 15.0), (40, 150, 3.0), (128, 256, 1.0)])
def test_dual_form_reproduces_the_symmetric_square_root(p, m, scale):
    rng = np.random.default_rng(p * 1000 + m)
    sigma = 0.2
    Yp = scale * rng.standard_normal((p, m))
    Yp -= Yp.mean(axis=1, keepdims=True)
    d = rng.standard_normal(p)
    w_ref, T_ref = etkf.ensemble_transform(Yp, d, sigma)
    S, dt, c = Yp / sigma, d / sigma, m - 1.0
    K = S @ S.T
    Z = _inv_sqrt(np.eye(p) + K / c)
    u = Z @ (Z @ dt) / c                                   # (cI + K)^-1 d
    # FP64 rounding times the conditioning of (m-1)I + G (up to ~1e5 in the scaled case)
    assert np.linalg.norm(S.T @ u - w_ref) <= 1e-9 * np.linalg.norm(w_ref)
    W = Z @ S / np.sqrt(c)
    M = np.eye(p) + Z
    X = (2.0 / 3.0) * np.eye(p)
    for _ in range(4):
        X = X @ (2.0 * np.eye(p) - M @ X)
    assert np.abs(X @ M - np.eye(p)).max() < 1e-7       # (1/3)^16
    T = np.eye(m) - W.T @ X @ W
    assert np.abs(T - T_ref).max() < 1e-7
    # the transform of the own rows as the kernel forms it: X'_E - ((X'_E S^T) Z / c) X Z S
    E = rng.standard_normal((20, m))
    E -= E.mean(axis=1, keepdims=True)
    out = E - (((E @ S.T) @ Z) @ X @ Z / c) @ S
    np.testing.assert_allclose(out, E @ T_ref, rtol=0, atol=1e-7 * np.abs(E @ T_ref).max() + 1e-12)


def test_newton_inverse_start_contracts_for_every_z_in_the_unit_interval():
    # the eigenvalues of Z = (I + K/c)^(-1/2) lie in (0, 1], so those of (I + Z) X_0 = (2/3)(I + Z)
    # lie in (2/3, 4/3]: |1 - mu| <= 1/3, squared by every step
    z = np.linspace(1e-9, 1.0, 10001)
    mu = (2.0 / 3.0) * (1.0 + z)
    assert np.abs(1.0 - mu).max() <= 1.0 / 3.0 + 1e-15
    e = np.abs(1.0 - mu)
    for _ in range(4):
        e = e * e
    assert e.max() < 3e-8


@pytest.mark.parametrize("p,seed", [(16, 1), (64, 2), (128, 3)])
def test_newton_inverse_elementwise_start_and_predicted_last_update(p, seed):
    # The kernel's schedule for (I + Z)^-1: X_1 = X_0 (2I - M X_0) with X_0 = 2/3 I is the
    # elementwise 4/3 I - 4/9 M (with X_0 = alpha I, 2 alpha I - alpha^2 M); R_k = I - M X_k squares at every update (X_k is a polynomial in M),
    # so ||R_{k+1}||_F <= ||R_k||_F^2 and an update taken when ||R_k||_F^2 is under the bound is the
    # last; at least one update runs.
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((p, p)))
    z = rng.uniform(0.02, 1.0, p)                    # eigenvalues of Z in (0, 1]
    Z = (Q * z) @ Q.T
    M = np.eye(p) + Z
    X0 = (2.0 / 3.0) * np.eye(p)
    X = (4.0 / 3.0) * np.eye(p) - (4.0 / 9.0) * M
    np.testing.assert_allclose(X, X0 @ (2.0 * np.eye(p) - M @ X0), rtol=0, atol=1e-15)
    # the kernel's start alpha I, alpha = 2 / (3 + s^(-1/2)), s = 1 + ||K||_F / c, contracts at least
    # as fast as 2/3 I: here K = c (Z^-2 - I), so s^(-1/2) is a lower bound on Z's spectrum
    c = 99.0
    K = c * (np.linalg.inv(Z @ Z) - np.eye(p))
    s_scale = 1.0 + np.linalg.norm(K) / c
    assert z.min() >= s_scale ** -0.5 * (1 - 1e-12)
    alpha = 2.0 / (3.0 + s_scale ** -0.5)
    rho = np.abs(1.0 - alpha * (1.0 + z)).max()
    assert rho <= (1.0 - s_scale ** -0.5) / (3.0 + s_scale ** -0.5) + 1e-12 <= 1.0 / 3.0 + 1e-12
    X = 2.0 * alpha * np.eye(p) - alpha * alpha * M
    np.testing.assert_allclose(X, alpha * (2.0 * np.eye(p) - alpha * M), rtol=0, atol=1e-15)
    tol = 1e-6 * p
    updates = 0
    for k in range(6):
        R = np.eye(p) - M @ X
        r2 = float(np.sum(R * R))
        if k > 0 and np.sqrt(r2) < tol:
            break
        last = r2 < tol
        Xn = X @ (2.0 * np.eye(p) - M @ X)
        Rn = np.eye(p) - M @ Xn
        np.testing.assert_allclose(Rn, R @ R, rtol=0, atol=1e-12)
        assert np.linalg.norm(Rn) <= r2 * (1 + 1e-12) + 1e-14
        X = Xn
        updates += 1
        if last:
            break
    assert 1 <= updates <= 4
    assert np.linalg.norm(np.eye(p) - M @ X) < tol
    np.testing.assert_allclose(X, np.linalg.inv(M), rtol=0, atol=1e-6)
