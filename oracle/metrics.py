"""Performance measure of the control law (Sect. 3): residual phase and coherent energy.

The paper compares control laws by coherent energy.  Reading used: the residual
at frame k is eps_k = phi_true(k+1) - x_hat(k+1|k) on the valid actuators, with
its piston (mean over valid actuators) removed; the residual variance is the
mean over frames after burn-in of ||eps_k||^2 / n_act, and the coherent energy
is its Marechal approximation exp(-variance).
"""

from __future__ import annotations

import numpy as np


def residual(phi_true_next: np.ndarray, x_pred: np.ndarray) -> np.ndarray:
    e = np.asarray(phi_true_next, dtype=np.float64) - np.asarray(x_pred, dtype=np.float64)
    return e - e.mean(axis=-1, keepdims=True)


def residual_variance(eps: np.ndarray) -> float:
    """eps: (frames, n_act) residuals -> mean over frames of ||eps||^2 / n_act."""
    eps = np.atleast_2d(eps)
    return float(np.mean(np.sum(eps ** 2, axis=1) / eps.shape[1]))


def coherent_energy(variance: float) -> float:
    return float(np.exp(-variance))
