"""Von Karman turbulence for the synthetic AO workloads (Sect. 3 set-up).

The paper simulates von Karman turbulence moved across the pupil by Taylor's
frozen-flow hypothesis.  This module draws periodic FFT phase screens from the
von Karman power spectrum and samples them along a wind trajectory.  It also
gives the closed-form von Karman phase covariance, from which callers build the
process-noise covariance of the filter's AR(1) model.

Units: lengths in metres, phase in radians at the sensing wavelength.
"""

from __future__ import annotations

import math

import numpy as np
from scipy import special

# 0.023 is the numerical constant of the Kolmogorov / von Karman phase power
# spectrum, Phi(f) = 0.023 r0^(-5/3) (f^2 + 1/L0^2)^(-11/6).
_PSD_CONST = 0.023


def vk_psd(f2: np.ndarray, r0: float, L0: float) -> np.ndarray:
    """Von Karman phase power spectral density at squared spatial frequency f2 (m^-2)."""
    return _PSD_CONST * r0 ** (-5.0 / 3.0) * (f2 + 1.0 / L0 ** 2) ** (-11.0 / 6.0)


def _vk_cov_prefactor(r0: float, L0: float) -> float:
    # (L0/r0)^(5/3) Gamma(11/6) / (2^(5/6) pi^(8/3)) (24/5 Gamma(6/5))^(5/6)
    return ((L0 / r0) ** (5.0 / 3.0) * special.gamma(11.0 / 6.0)
            / (2.0 ** (5.0 / 6.0) * math.pi ** (8.0 / 3.0))
            * (24.0 / 5.0 * special.gamma(6.0 / 5.0)) ** (5.0 / 6.0))


def vk_phase_covariance(r: np.ndarray, r0: float, L0: float) -> np.ndarray:
    """Von Karman phase covariance C(r) between two points a distance r apart.

    C(r) = P (2 pi r / L0)^(5/6) K_{5/6}(2 pi r / L0), with P from
    _vk_cov_prefactor; at r = 0 the limit x^(5/6) K_{5/6}(x) -> 2^(-1/6) Gamma(5/6)
    gives the phase variance.  C is the Hankel transform of vk_psd.
    """
    r = np.asarray(r, dtype=np.float64)
    pref = _vk_cov_prefactor(r0, L0)
    x = 2.0 * math.pi * r / L0
    out = np.empty_like(x)
    small = x < 1e-12
    xs = x[~small]
    out[~small] = pref * xs ** (5.0 / 6.0) * special.kv(5.0 / 6.0, xs)
    out[small] = pref * 2.0 ** (-1.0 / 6.0) * special.gamma(5.0 / 6.0)
    return out


def vk_structure_function_kolmogorov(r: np.ndarray, r0: float) -> np.ndarray:
    """Kolmogorov phase structure function 6.88 (r/r0)^(5/3), the r << L0 limit."""
    return 6.88 * (np.asarray(r, dtype=np.float64) / r0) ** (5.0 / 3.0)


def actuator_covariance_lag_table(n_side: int, pitch: float, r0: float, L0: float,
                                  shift=(0.0, 0.0)) -> np.ndarray:
    """Covariance between grid points for every integer lag, optionally plus a metric shift.

    Returns T of shape (2*n_side-1, 2*n_side-1) with
    T[dr + n_side - 1, dc + n_side - 1] = C(|pitch * (dc, dr) + shift|), where shift =
    (sx, sy) in metres.  With shift = 0 this is the covariance between grid points
    (dr, dc) apart; with shift = the wind displacement of one frame it is the
    covariance between a point now and another point one frame later under frozen
    flow.  Covariance matrices between grid points are then gathers from the table,
    which avoids evaluating the Bessel function n^2 times for large grids.
    """
    d = np.arange(-(n_side - 1), n_side, dtype=np.float64)
    dx = pitch * d[None, :] + shift[0]
    dy = pitch * d[:, None] + shift[1]
    return vk_phase_covariance(np.sqrt(dx * dx + dy * dy), r0, L0)


class VKScreen:
    """A periodic von Karman phase screen sampled on an n_pix x n_pix grid of spacing dx.

    The screen is the real part of the inverse FFT of complex white noise shaped by
    sqrt(PSD) (the FFT method).  It is periodic, so frozen flow may wrap around.
    The screen must be several outer scales across for the low spatial frequencies
    to be represented; callers pick n_pix * dx >= 4 L0.
    """

    def __init__(self, n_pix: int, dx: float, r0: float, L0: float, seed: int):
        self.n_pix, self.dx, self.r0, self.L0 = int(n_pix), float(dx), float(r0), float(L0)
        rng = np.random.default_rng(seed)
        df = 1.0 / (self.n_pix * self.dx)
        f = np.fft.fftfreq(self.n_pix, self.dx)
        f2 = f[:, None] ** 2 + f[None, :] ** 2
        amp = np.sqrt(vk_psd(f2, self.r0, self.L0)) * df
        amp[0, 0] = 0.0
        noise = rng.standard_normal((self.n_pix, self.n_pix)) + 1j * rng.standard_normal((self.n_pix, self.n_pix))
        scr = np.fft.ifft2(noise * amp) * (self.n_pix * self.n_pix)
        self.phase = np.ascontiguousarray(scr.real)

    def sample(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        """Bilinear, periodic sample of the screen at metric coordinates (x, y)."""
        u = np.asarray(x, dtype=np.float64) / self.dx
        v = np.asarray(y, dtype=np.float64) / self.dx
        u0 = np.floor(u)
        v0 = np.floor(v)
        fu = u - u0
        fv = v - v0
        n = self.n_pix
        i0 = np.mod(v0.astype(np.int64), n)
        j0 = np.mod(u0.astype(np.int64), n)
        i1 = (i0 + 1) % n
        j1 = (j0 + 1) % n
        p = self.phase
        return ((1 - fv) * ((1 - fu) * p[i0, j0] + fu * p[i0, j1])
                + fv * ((1 - fu) * p[i1, j0] + fu * p[i1, j1]))
