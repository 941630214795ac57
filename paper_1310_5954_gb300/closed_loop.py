"""Closed-loop evaluation of a control law on the sensor's fine phase grid (Sect. 3).

The paper runs its control laws in a closed AO loop with a two-step delay between measurement and
correction, a deformable mirror of instantaneous response whose actuators couple by 0.3 to their
neighbours, and compares them by coherent energy.  In a linear loop the estimator works on
pseudo-open-loop slopes (the measured residual slopes plus the sensor's response to the known DM
shape), which are the open-loop slopes themselves, so the filter's predictions are those of the
open-loop run; the loop adds the mirror and the metric, both here:

* the mirror: one influence function per valid actuator on the fine grid, coupling^((d / pitch)^2)
  (value 1 at its own actuator, `coupling` at the nearest ones), cut beyond `reach` pitches.  The
  commands u make the mirror pass through the predicted phase at the actuator points, F u = x_hat
  (F: the influence functions at the actuator points), so the correction is N F^-1 x_hat on the
  fine pupil pixels (N: the influence functions there);
* the residual of frame k: the fine-grid phase of the next frame minus the correction made from
  the prediction x_hat(k+1|k), its piston removed over the pupil pixels; the coherent energy of
  the frame is the Marechal approximation exp(-variance), averaged over frames.

Host-side numpy and scipy.sparse (the influence functions are stored sparse: ~2.2 M entries for
the 16 m system's 82 k pupil pixels): this evaluates a control law, it is not part of the per-frame
update.
"""

from __future__ import annotations

import numpy as np
from scipy import sparse


class DeformableMirror:
    """Zonal deformable mirror on a Shack-Hartmann sensor's fine grid.

    sub_valid: (N, N) valid subapertures; act_valid: (N + 1, N + 1) valid actuators (the filter's
    state order: row-major over the valid ones); q: fine samples per pitch.
    """

    def __init__(self, sub_valid: np.ndarray, act_valid: np.ndarray, q: int, coupling: float = 0.3,
                 reach: float = 3.0):
        sub_valid = np.asarray(sub_valid, dtype=bool)
        act_valid = np.asarray(act_valid, dtype=bool)
        n = sub_valid.shape[0]
        if sub_valid.shape != (n, n) or act_valid.shape != (n + 1, n + 1) or q < 1:
            raise ValueError("sub_valid must be N x N, act_valid (N + 1) x (N + 1), q >= 1")
        if not 0.0 < coupling < 1.0:
            raise ValueError("coupling must lie in (0, 1)")
        self.n_sub, self.q, self.coupling = n, int(q), float(coupling)
        nf = n * q + 1
        # fine pixels touching at least one valid subaperture
        idx = np.arange(nf)
        lo = np.clip((idx - 1) // q, 0, n - 1)
        hi = np.clip(idx // q, 0, n - 1)
        pupil = np.zeros((nf, nf), dtype=bool)
        for rr in (lo, hi):
            for cc in (lo, hi):
                pupil |= sub_valid[rr[:, None], cc[None, :]]
        self.pupil = pupil
        pr, pc = np.nonzero(pupil)
        ar, ac = np.nonzero(act_valid)
        self.n_pix, self.n_act = pr.size, ar.size
        ln_c = np.log(self.coupling)
        # N (pupil pixels x actuators), sparse: each influence function within `reach` pitches
        pix_index = -np.ones((nf, nf), dtype=np.int64)
        pix_index[pr, pc] = np.arange(self.n_pix)
        w = int(np.floor(reach * q))
        rows, cols, vals = [], [], []
        for j, (a_r, a_c) in enumerate(zip(ar, ac)):
            r0, r1 = max(a_r * q - w, 0), min(a_r * q + w, nf - 1)
            c0, c1 = max(a_c * q - w, 0), min(a_c * q + w, nf - 1)
            rr, cc = np.meshgrid(np.arange(r0, r1 + 1), np.arange(c0, c1 + 1), indexing="ij")
            d2 = ((rr / q - a_r) ** 2 + (cc / q - a_c) ** 2).ravel()
            pi = pix_index[rr, cc].ravel()
            keep = (pi >= 0) & (d2 <= reach * reach)
            rows.append(pi[keep])
            cols.append(np.full(int(keep.sum()), j))
            vals.append(np.exp(ln_c * d2[keep]))
        self.N = sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                   shape=(self.n_pix, self.n_act))
        d2a = ((ar[:, None] - ar[None, :]) ** 2 + (ac[:, None] - ac[None, :]) ** 2).astype(np.float64)
        F = np.exp(ln_c * d2a)
        F[d2a > reach * reach] = 0.0
        self.F = F
        # F is symmetric positive definite (a Gaussian kernel on distinct points)
        self.F_inv = np.linalg.inv(F)

    def correction(self, x_act: np.ndarray) -> np.ndarray:
        """Mirror surface on the pupil pixels that passes through x_act at the actuators; x_act is
        (n_act,) or (frames, n_act)."""
        x = np.asarray(x_act, dtype=np.float64)
        u = self.F_inv @ x.T                       # commands: F u = x
        return np.asarray(self.N @ u).T

    def residual_variance(self, phi_fine: np.ndarray, x_act: np.ndarray) -> np.ndarray:
        """Piston-removed variance over the pupil of phi_fine - correction(x_act).  phi_fine:
        (nf, nf) or (frames, nf, nf) fine-grid phase; x_act: (n_act,) or (frames, n_act)."""
        phi = np.asarray(phi_fine, dtype=np.float64)
        e = phi[..., self.pupil] - self.correction(x_act)
        e = e - e.mean(axis=-1, keepdims=True)
        return np.mean(e * e, axis=-1)


def coherent_energy(variances) -> float:
    """Mean over frames of the Marechal coherent energy exp(-variance)."""
    v = np.asarray(variances, dtype=np.float64)
    return float(np.mean(np.exp(-v)))
