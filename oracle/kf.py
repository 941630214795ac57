"""Classical Kalman filter with the asymptotic (Riccati) gain, and the sample-covariance gain.

Sect. 2.1: the optimal prediction estimate is Eq. 1,
    x_hat(k+1|k) = A1 x_hat(k|k-1) + A1 H (y_k - C x_hat(k|k-1)),
with H the Kalman gain.  For a stationary model the gain comes off line from the
asymptotic solution of the Riccati equation; the prediction-error covariance P
solves the discrete algebraic Riccati equation (DARE)
    P = A P A^T - A P C^T (C P C^T + R)^-1 C P A^T + Q,
and H = P C^T (C P C^T + R)^-1.

The DARE is solved here by the structure-preserving doubling algorithm (a
published method: Chu, Fan, Lin, Wang, 2004), started from A_0 = A^T,
G_0 = C^T R^-1 C, H_0 = Q; its H_k converges quadratically to P.

The ETKF substitutes empirical covariances for the true ones (Sect. 2.2): with
P_f = X' X'^T / (m-1) the explicit gain is K = P_f C^T (C P_f C^T + R)^-1.
"""

from __future__ import annotations

import numpy as np


def dare(A: np.ndarray, C: np.ndarray, Q: np.ndarray, R: np.ndarray,
         tol: float = 1e-13, maxit: int = 200) -> np.ndarray:
    """Stationary prediction-error covariance P of the filter DARE, by doubling."""
    n = A.shape[0]
    Ak = A.T.copy()
    Gk = C.T @ np.linalg.solve(R, C)
    Hk = Q.copy()
    I = np.eye(n)
    for _ in range(maxit):
        W = np.linalg.inv(I + Gk @ Hk)
        A_next = Ak @ W @ Ak
        G_next = Gk + Ak @ W @ Gk @ Ak.T
        H_next = Hk + Ak.T @ Hk @ W @ Ak
        H_next = 0.5 * (H_next + H_next.T)
        G_next = 0.5 * (G_next + G_next.T)
        done = np.linalg.norm(H_next - Hk) <= tol * max(1.0, np.linalg.norm(H_next))
        Ak, Gk, Hk = A_next, G_next, H_next
        if done:
            break
    return Hk


def kalman_gain(P: np.ndarray, C: np.ndarray, R: np.ndarray) -> np.ndarray:
    """H = P C^T (C P C^T + R)^-1."""
    S = C @ P @ C.T + R
    return np.linalg.solve(S.T, (P @ C.T).T).T


def kf_predict(x_pred: np.ndarray, y: np.ndarray, A: np.ndarray, C: np.ndarray,
               H: np.ndarray) -> np.ndarray:
    """Eq. 1: x_hat(k+1|k) = A x_hat(k|k-1) + A H (y_k - C x_hat(k|k-1))."""
    return A @ (x_pred + H @ (y - C @ x_pred))


def sample_gain(Xf: np.ndarray, C: np.ndarray, R: np.ndarray) -> np.ndarray:
    """K = P_f C^T (C P_f C^T + R)^-1 with the empirical P_f = X'X'^T/(m-1)."""
    m = Xf.shape[1]
    Xp = Xf - Xf.mean(axis=1, keepdims=True)
    Pf = Xp @ Xp.T / (m - 1)
    return kalman_gain(Pf, C, R)


def ar1_companion(n_act: int, a: float) -> np.ndarray:
    """A1 = [[a I, 0], [I, 0]] for the two-instant state (Sect. 2.1)."""
    A = np.zeros((2 * n_act, 2 * n_act))
    A[:n_act, :n_act] = a * np.eye(n_act)
    A[n_act:, :n_act] = np.eye(n_act)
    return A


def process_covariance(L: np.ndarray) -> np.ndarray:
    """Q of the two-instant state: L L^T on the first block, zero elsewhere."""
    n_act = L.shape[0]
    Q = np.zeros((2 * n_act, 2 * n_act))
    Q[:n_act, :n_act] = L @ L.T
    return Q
