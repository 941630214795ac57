"""Global ETKF and local ETKF in FP64 (Sect. 2.2, 2.3; Eq. 1 ordering).

The paper does not print the ETKF equations; it cites the transform form of
Bishop et al., Sakov & Oke and Hunt et al. (refs. [8-10], [14]).  The form used
is the symmetric-square-root transform of Hunt et al. with unscaled anomalies,
no inflation and hard domains (no observation tapering):

    x_bar = X_f 1/m,  X' = X_f - x_bar 1^T           (ensemble mean and anomalies)
    Y = C X_f,  y_bar = Y 1/m,  Y' = Y - y_bar 1^T,  d = y - y_bar
    G = Y'^T R^-1 Y'                                 (m x m)
    (m-1) I + G = U diag(m-1+lambda) U^T             (symmetric eigendecomposition)
    w_bar = U diag(1/(m-1+lambda)) U^T Y'^T R^-1 d
    T     = U diag(sqrt((m-1)/(m-1+lambda))) U^T  =  sqrt(m-1) [(m-1)I + G]^(-1/2)
    X_a   = x_bar 1^T + X' (w_bar 1^T + T)

The local ETKF (Sect. 2.3) applies the same transform independently per domain,
with Y', d and R restricted to the domain's observation region and the update
restricted to the domain's own actuators (both phase instants).  Every actuator
is owned by exactly one domain, so the scattered domain estimates are the
whole-pupil estimate (Sect. 3.2).  A domain with no observation keeps its
forecast (G = 0 gives w_bar = 0, T = I).

Forecast (Sect. 2.1, AR(1) on a two-instant state): A1 = [[a I, 0], [I, 0]],
x_f(k+1) = A1 x_a(k) + [v_k; 0] per member, v_k = L xi_k with Q = L L^T.
One filter step takes y_k, runs the analysis, then the forecast, and returns
x_hat(k+1|k) (Eq. 1 is the prediction form).  With differential-piston removal (module
`piston`), the step then fits one piston per domain to the slope residual of x_hat(k+1|k)
against y_k and adds it to the returned prediction ("output") or to the prediction and every
member of both instants of the forecast ensemble ("in_loop").
"""

from __future__ import annotations

from typing import List, Optional

import numpy as np
import scipy.sparse as sp

from . import philox
from . import piston as _piston
from .fried import fried_matrix
from .geometry import Domain, Geometry


def ensemble_transform(Yp: np.ndarray, d: np.ndarray, sigma: float):
    """(w_bar, T) of the symmetric ETKF for anomalies Yp (p x m), innovation d, R = sigma^2 I."""
    m = Yp.shape[1]
    c = m - 1.0
    G = (Yp.T @ Yp) / sigma ** 2
    b = (Yp.T @ d) / sigma ** 2
    lam, U = np.linalg.eigh(c * np.eye(m) + G)       # eigenvalues of (m-1)I + G
    wbar = U @ ((U.T @ b) / lam)
    T = (U * np.sqrt(c / lam)) @ U.T
    return wbar, T


def etkf_analysis(Xf: np.ndarray, y: np.ndarray, C, sigma: float) -> np.ndarray:
    """Global ETKF analysis (Sect. 2.2): every state row against every observation."""
    xbar = Xf.mean(axis=1)
    Xp = Xf - xbar[:, None]
    Y = C @ Xf
    ybar = Y.mean(axis=1)
    wbar, T = ensemble_transform(Y - ybar[:, None], y - ybar, sigma)
    return xbar[:, None] + Xp @ (wbar[:, None] + T)


def letkf_analysis(Xf: np.ndarray, y: np.ndarray, C, sigma: float, domains: List[Domain],
                   n_act: int, n_subv: int) -> np.ndarray:
    """Local ETKF analysis (Sect. 2.3): one independent transform per domain."""
    xbar = Xf.mean(axis=1)
    Xp = Xf - xbar[:, None]
    Y = C @ Xf
    ybar = Y.mean(axis=1)
    Yp = Y - ybar[:, None]
    Xa = Xf.copy()
    for dom in domains:
        rows = dom.rows(n_act)
        orows = dom.obs_rows(n_subv)
        if orows.size == 0:
            continue
        wbar, T = ensemble_transform(Yp[orows], y[orows] - ybar[orows], sigma)
        Xa[rows] = xbar[rows, None] + Xp[rows] @ (wbar[:, None] + T)
    return Xa


def forecast(Xa: np.ndarray, a: float, V: np.ndarray, a2: float = 0.0) -> np.ndarray:
    """Forecast of every member with the two-instant companion matrix of the AR model (Sect. 2.1,
    "AR 1 or AR 2"): A1 = [[a I, a2 I], [I, 0]], i.e. phi_{k+1} = a phi_k + a2 phi_{k-1} + v_k;
    a2 = 0 is the AR(1) model."""
    n_act = Xa.shape[0] // 2
    Xf = np.empty_like(Xa)
    Xf[:n_act] = a * Xa[:n_act] + V
    if a2 != 0.0:
        Xf[:n_act] += a2 * Xa[n_act:]
    Xf[n_act:] = Xa[:n_act]
    return Xf


def sparse_observation(geom: Geometry, obs_block: int = 1):
    """C = [0 D] (obs_block 1) or [D 0] as a sparse matrix."""
    D = sp.csr_matrix(fried_matrix(geom))
    Z = sp.csr_matrix(D.shape)
    return sp.hstack([Z, D] if obs_block == 1 else [D, Z]).tocsr()


class OracleFilter:
    """A running FP64 filter: initial ensemble, analysis, forecast, step (Sect. 2.2-2.3)."""

    def __init__(self, geom: Geometry, domains: Optional[List[Domain]], m: int, a: float,
                 sigma: float, seed: int, L: Optional[np.ndarray] = None, q_white: float = 0.0,
                 obs_block: int = 1, X0: Optional[np.ndarray] = None,
                 L_stat: Optional[np.ndarray] = None, a2: float = 0.0, piston: str = "off"):
        if piston not in ("off", "output", "in_loop"):
            raise ValueError("piston must be 'off', 'output' or 'in_loop'")
        if piston != "off" and domains is None:
            raise ValueError("differential pistons exist only between domains")
        self.geom, self.domains, self.m, self.a = geom, domains, m, float(a)
        self.piston = piston
        self.a2 = float(a2)
        self.sigma, self.seed, self.L, self.q_white = float(sigma), int(seed), L, float(q_white)
        self.L_stat = L_stat
        self.C = sparse_observation(geom, obs_block)
        self.frame = 0
        self.X = self.initial_ensemble() if X0 is None else np.array(X0, dtype=np.float64)

    def _noise(self, xi: np.ndarray) -> np.ndarray:
        return self.L @ xi if self.L is not None else self.q_white * xi

    def initial_ensemble(self) -> np.ndarray:
        """Initial ensemble (Sect. 2.2), one AR(1) pair per member: the second block is drawn
        from the stationary phase covariance, block2 = L_stat xi0 (L_stat defaults to
        L / sqrt(1 - a^2), or q_white / sqrt(1 - a^2) for white noise), and the first block
        follows the model, block1 = a block2 + L xi1 (for AR(2) the stationary variance of the
        AR(2) model replaces 1 / (1 - a^2))."""
        na = self.geom.n_act
        xi2 = philox.normals(self.seed, 0, 0, self.m, na)
        xi1 = philox.normals(self.seed, 0, 1, self.m, na)
        if self.L_stat is not None:
            b2 = self.L_stat @ xi2
        else:
            # stationary variance of the AR model with unit innovations: for AR(2)
            # (1 - a2) / ((1 + a2) ((1 - a2)^2 - a^2)), i.e. 1 / (1 - a^2) when a2 = 0
            a, a2 = self.a, self.a2
            b2 = self._noise(xi2) * np.sqrt((1.0 - a2) / ((1.0 + a2) * ((1.0 - a2) ** 2 - a * a)))
        b1 = self.a * b2 + self._noise(xi1)
        return np.vstack([b1, b2])

    def perturbation(self, frame: int) -> np.ndarray:
        return self._noise(philox.normals(self.seed, 1, frame, self.m, self.geom.n_act))

    def analyze(self, y: np.ndarray, sigma: Optional[float] = None) -> None:
        if sigma is not None and sigma > 0:
            self.sigma = float(sigma)
        if self.domains is None:
            self.X = etkf_analysis(self.X, y, self.C, self.sigma)
        else:
            self.X = letkf_analysis(self.X, y, self.C, self.sigma, self.domains,
                                    self.geom.n_act, self.geom.n_subv)

    def forecast(self, V: Optional[np.ndarray] = None) -> None:
        if V is None:
            V = self.perturbation(self.frame)
        self.X = forecast(self.X, self.a, V, self.a2)
        self.frame += 1

    def step(self, y: np.ndarray, sigma: Optional[float] = None,
             V: Optional[np.ndarray] = None) -> np.ndarray:
        """Analysis with y_k, then forecast; returns x_hat(k+1|k) on the first block (corrected
        for differential pistons when that mode is on)."""
        self.analyze(y, sigma)
        self.forecast(V)
        na = self.geom.n_act
        xhat = self.X[:na].mean(axis=1)
        if self.piston == "off":
            return xhat
        shift = _piston.ownership(self.geom, self.domains) @ _piston.differential_pistons(
            xhat, y, self.geom, self.domains)
        if self.piston == "in_loop":
            self.X[:na] += shift[:, None]
            self.X[na:] += shift[:, None]
        return xhat + shift
