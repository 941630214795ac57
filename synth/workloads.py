"""Synthetic AO workloads: parameters, seeds and the per-frame truth stream.

The paper's workloads are Matlab simulations of single-conjugate AO systems
(Sect. 3): von Karman turbulence (r0, L0), Taylor frozen flow at a given wind
speed, a Shack-Hartmann sensor in Fried geometry with white slope noise, and an
AR(1) turbulence model inside the filter.  No public dataset is involved; these
seeded generators stand in for those simulations at the sizes listed below.

Seeds: workload i uses base seed 1310595400 + i.  Within a workload the phase
screen uses sub-seed 3 and the slope noise sub-seed 2 (numpy PCG64 streams).
The filter's own random draws (initial ensemble, process noise) are not made
here: both implementations of the filter draw them from a counter-based
Philox4x32-10 generator keyed by the workload seed.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

from .turbulence import VKScreen, actuator_covariance_lag_table
from .wfs import FineGridSensor

BASE_SEED = 1310595400


@dataclasses.dataclass
class Workload:
    name: str
    n_sub: int               # subapertures across the pupil (Fried: n_sub+1 actuators across)
    obstruction: float       # central obstruction ratio
    m: int                   # ensemble size
    dom_sub: int             # estimation-domain side, in subapertures
    halo: int                # observation halo, in subapertures
    ar1_a: float             # AR coefficient of phi_k in the turbulence model
    sigma: float             # slope-noise std (rad per slope)
    tel_diam: float          # telescope diameter (m)
    d_over_r0: float
    L0: float                # outer scale (m)
    wind: float              # wind speed (m/s)
    frame_rate: float        # Hz
    n_frames: int
    seed: int
    wind_angle: float = 0.0  # radians
    obs_block: int = 1       # slopes observe the state's second block (one-frame sensor delay)
    q: int = 4               # fine samples per pitch in the truth sensor
    nonstationary: bool = False
    ar2_a: float = 0.0       # AR coefficient of phi_{k-1} (0: AR(1) model)
    # frozen-flow layers ((Cn2 fraction, speed m/s, direction rad), ...), fractions summing to 1;
    # empty: one layer moving at (wind, wind_angle), or the non-stationary schedule
    layers: tuple = ()

    def layer_list(self):
        return self.layers if self.layers else ((1.0, self.wind, self.wind_angle),)

    @property
    def pitch(self) -> float:
        return self.tel_diam / self.n_sub

    @property
    def r0(self) -> float:
        return self.tel_diam / self.d_over_r0

    # --- non-stationary schedule (r0 halves at 3000; wind 10 -> 25 m/s and +90 deg over
    # frames 6000-7000; noise 0.1 -> 0.3 rad at 8000).  Stationary workloads ignore it.
    def screen_scale(self, k: int) -> float:
        if self.nonstationary and k >= 3000:
            return 2.0 ** (5.0 / 6.0)   # phase std scales as r0^(-5/6)
        return 1.0

    def wind_at(self, k: int):
        if not self.nonstationary:
            return self.wind, self.wind_angle
        if k < 6000:
            return 10.0, 0.0
        if k >= 7000:
            return 25.0, math.pi / 2
        s = (k - 6000) / 1000.0
        return 10.0 + 15.0 * s, s * math.pi / 2

    def sigma_at(self, k: int) -> float:
        if not self.nonstationary:
            return self.sigma
        return 0.1 if k < 8000 else 0.3

    def _lag_gather(self, act_rc: np.ndarray, shift=(0.0, 0.0)) -> np.ndarray:
        act_rc = np.asarray(act_rc, dtype=np.int64)
        n_side = self.n_sub + 1
        lag = actuator_covariance_lag_table(n_side, self.pitch, self.r0, self.L0, shift)
        dr = act_rc[:, 0][:, None] - act_rc[:, 0][None, :] + n_side - 1
        dc = act_rc[:, 1][:, None] - act_rc[:, 1][None, :] + n_side - 1
        return lag[dr, dc]

    @staticmethod
    def _chol(S: np.ndarray, jitter: float) -> np.ndarray:
        S = S.copy()
        S[np.diag_indices_from(S)] += jitter * np.trace(S) / S.shape[0]
        return np.linalg.cholesky(S)

    def stationary_sqrt(self, act_rc: np.ndarray, jitter: float = 1e-8) -> np.ndarray:
        """Lower-triangular L0 with L0 L0^T = Sigma_phi + eps I: von Karman phase covariance
        of one phase instant at the given actuators ((n_act, 2) row, column positions)."""
        return self._chol(self._lag_gather(act_rc), jitter)

    def _shift(self, frames: int = 1, layer: int = 0):
        if self.layers:
            _, v, ang = self.layers[layer]
        else:
            v, ang = self.wind_at(0)
        return (frames * v / self.frame_rate * math.cos(ang), frames * v / self.frame_rate * math.sin(ang))

    def _lagged_cov(self, act_rc: np.ndarray, frames: int) -> np.ndarray:
        """Covariance between the phase at the actuators now and `frames` frames later: the sum over
        independent layers of fraction x (von Karman covariance at r0, shifted by that layer's path);
        a layer of fraction f has r0_l = r0 f^(-3/5), and the covariance scales as r0^(-5/3)."""
        return sum(f * self._lag_gather(act_rc, self._shift(frames, l)) for l, (f, _, _) in enumerate(self.layer_list()))

    def process_noise_sqrt(self, act_rc: np.ndarray, jitter: float = 1e-8) -> np.ndarray:
        """Lower-triangular L with L L^T = Q + eps I, Q the covariance of the AR innovation
        e = phi_{k+1} - a phi_k - a2 phi_{k-1} when the true phase is von Karman turbulence under
        frozen flow at the workload's wind:
            Q = (1 + a^2 + a2^2) S(0) - (a - a a2) (S(s) + S(s)^T) - a2 (S(2s) + S(2s)^T),
        S(js)_ij the covariance between actuator i now and actuator j j frames (shift js) later
        (a2 = 0: the AR(1) innovation (1 + a^2) S(0) - a (S(s) + S(s)^T))."""
        a, a2 = self.ar1_a, self.ar2_a
        S0 = self._lag_gather(act_rc)
        S1 = self._lagged_cov(act_rc, 1)
        Q = (1.0 + a * a + a2 * a2) * S0 - (a - a * a2) * (S1 + S1.T)
        if a2 != 0.0:
            S2 = self._lagged_cov(act_rc, 2)
            Q = Q - a2 * (S2 + S2.T)
        return self._chol(Q, jitter)

    def ar2_fit(self, act_rc: np.ndarray):
        """(a, a2) of the AR(2) model fitted to the frozen-flow turbulence: the Yule-Walker
        equations on the phase autocovariance summed over the actuators, t_j = tr S(js)."""
        t = [float(np.trace(self._lagged_cov(act_rc, j))) for j in range(3)]
        return yule_walker_ar2(*t)


def yule_walker_ar2(t0: float, t1: float, t2: float):
    """AR(2) coefficients from the autocovariances at lags 0, 1, 2: [[t0, t1], [t1, t0]] a = [t1, t2]."""
    det = t0 * t0 - t1 * t1
    return (t1 * t0 - t1 * t2) / det, (t0 * t2 - t1 * t1) / det


def _wl(i, **kw) -> Workload:
    return Workload(seed=BASE_SEED + i, **kw)


WORKLOADS = {
    # 8x8 Fried system, 4 domains of 4x4 subapertures with a 1-subaperture halo; FP64.
    "tiny-8x8": _wl(0, name="tiny-8x8", n_sub=8, obstruction=0.0, m=20, dom_sub=4, halo=1,
                    ar1_a=0.99, sigma=0.1, tel_diam=4.0, d_over_r0=10.0, L0=25.0, wind=10.0,
                    frame_rate=1000.0, n_frames=200),
    # VLT-class 40x40, 14% obstruction, m = 50, 4x4 domains, halo 2.
    "vlt-40x40": _wl(1, name="vlt-40x40", n_sub=40, obstruction=0.14, m=50, dom_sub=4, halo=2,
                     ar1_a=0.995, sigma=0.15, tel_diam=8.0, d_over_r0=20.0, L0=25.0, wind=10.0,
                     frame_rate=1000.0, n_frames=2000),
    # ELT-class 80x80, 28% obstruction, m = 100, 4x4 domains, halo 2.
    "elt-80x80": _wl(2, name="elt-80x80", n_sub=80, obstruction=0.28, m=100, dom_sub=4, halo=2,
                     ar1_a=0.995, sigma=0.2, tel_diam=40.0, d_over_r0=40.0, L0=25.0, wind=15.0,
                     frame_rate=1000.0, n_frames=5000),
    # Global ETKF (one domain), the paper's 16 m case: 32x32 unobstructed, n = 1754, 197 members.
    "etkf-16m": _wl(5, name="etkf-16m", n_sub=32, obstruction=0.0, m=197, dom_sub=32, halo=0,
                    ar1_a=0.99, sigma=0.1, tel_diam=16.0, d_over_r0=20.0, L0=25.0, wind=10.0,
                    frame_rate=1000.0, n_frames=2000),
    # Global ETKF at ELT scale with a large ensemble: the 80x80 system above, 1024 members.
    "etkf-elt-m1024": _wl(6, name="etkf-elt-m1024", n_sub=80, obstruction=0.28, m=1024, dom_sub=80, halo=0,
                          ar1_a=0.995, sigma=0.2, tel_diam=40.0, d_over_r0=40.0, L0=25.0, wind=15.0,
                          frame_rate=1000.0, n_frames=5000),
    # The paper's 8 m SCAO case (Sect. 3, Sect. 3.1): 16x16 Fried system (241 actuators), r0 =
    # 0.525 m, L0 = 25 m, three frozen-flow layers (7.5, 12.5, 15 m/s; Cn2 0.5, 0.17, 0.33), 500 Hz,
    # ten fine samples per subaperture; the layer directions are not given (0, 60, 120 degrees here).
    "scao-8m": _wl(7, name="scao-8m", n_sub=16, obstruction=0.0, m=100, dom_sub=4, halo=2,
                   ar1_a=0.99, sigma=0.1, tel_diam=8.0, d_over_r0=8.0 / 0.525, L0=25.0, wind=7.5,
                   frame_rate=500.0, n_frames=2000, q=10,
                   layers=((0.5, 7.5, 0.0), (0.17, 12.5, math.pi / 3), (0.33, 15.0, 2 * math.pi / 3))),
    # The paper's 16 m case (Sect. 3.2, Fig. 3): 32x32 unobstructed (877 actuators), the same
    # turbulence and loop rate.
    "scao-16m": _wl(8, name="scao-16m", n_sub=32, obstruction=0.0, m=197, dom_sub=4, halo=2,
                    ar1_a=0.99, sigma=0.1, tel_diam=16.0, d_over_r0=16.0 / 0.525, L0=25.0, wind=7.5,
                    frame_rate=500.0, n_frames=2000, q=10,
                    layers=((0.5, 7.5, 0.0), (0.17, 12.5, math.pi / 3), (0.33, 15.0, 2 * math.pi / 3))),
    # The ELT system above with 200 members (the same seed, so the same frames): every domain takes
    # the observation-space (dual) form of the analysis, as the serving mix's m = 200 systems do.
    "elt-80x80-m200": _wl(2, name="elt-80x80-m200", n_sub=80, obstruction=0.28, m=200, dom_sub=4, halo=2,
                          ar1_a=0.995, sigma=0.2, tel_diam=40.0, d_over_r0=40.0, L0=25.0, wind=15.0,
                          frame_rate=1000.0, n_frames=5000),
    # The same ELT system under a non-stationary schedule (see Workload methods).
    "elt-80x80-nonstationary": _wl(3, name="elt-80x80-nonstationary", n_sub=80, obstruction=0.28,
                                   m=100, dom_sub=4, halo=2, ar1_a=0.995, sigma=0.1, tel_diam=40.0,
                                   d_over_r0=40.0, L0=25.0, wind=10.0, frame_rate=1000.0,
                                   n_frames=10000, nonstationary=True),
}


def workload(name: str) -> Workload:
    return dataclasses.replace(WORKLOADS[name])


def serving_mix(n_systems: int = 16, seed: int = BASE_SEED + 4) -> List[dict]:
    """The 16-system serving mix: sizes cycle over {16,32,40,64,80,100} subapertures and
    ensemble sizes over {20,50,100,200}; obstruction, D/r0, wind, noise and Poisson
    arrival rate are seeded uniform draws.  Returns [{'workload': Workload, 'rate_hz': float}]."""
    rng = np.random.default_rng(seed)
    sizes = [16, 32, 40, 64, 80, 100]
    ms = [20, 50, 100, 200]
    out = []
    for s in range(n_systems):
        n = sizes[s % len(sizes)]
        w = Workload(name=f"serve-{s:02d}-{n}x{n}-m{ms[s % len(ms)]}", n_sub=n,
                     obstruction=float(rng.uniform(0.0, 0.28)), m=ms[s % len(ms)], dom_sub=4, halo=2,
                     ar1_a=0.995, sigma=float(rng.uniform(0.1, 0.3)), tel_diam=0.5 * n,
                     d_over_r0=float(rng.uniform(10.0, 50.0)), L0=25.0,
                     wind=float(rng.uniform(5.0, 25.0)), frame_rate=1000.0, n_frames=20000,
                     seed=seed * 100 + s, wind_angle=float(rng.uniform(0, 2 * math.pi)))
        out.append({"workload": w, "rate_hz": float(rng.uniform(500.0, 2000.0))})
    return out


class TruthStream:
    """Per-frame truth of a workload: sensor slopes (with noise) and actuator-point phase.

    frame k: the true phase phi_k is the screen shifted by the wind path integrated up to
    frame k.  The sensor reading delivered at frame k measures phi_{k - obs_block} (a
    one-frame sensor delay when obs_block = 1) plus white noise of std sigma_at(k).
    """

    def __init__(self, w: Workload, n_pix: Optional[int] = None):
        self.w = w
        self.sensor = FineGridSensor(w.n_sub, w.q)
        dx = w.pitch / w.q
        if n_pix is None:
            vmax = max(v for _, v, _ in w.layer_list())
            need = max(4.0 * w.L0, 2.0 * w.tel_diam + vmax * w.n_frames / w.frame_rate)
            n_pix = 1 << int(math.ceil(math.log2(max(256.0, need / dx))))
            n_pix = min(n_pix, 4096)
        # one screen per layer (r0_l = r0 f^(-3/5)); the first keeps the single-layer seed
        self.screens = [VKScreen(n_pix, dx, w.r0 * f ** (-0.6), w.L0, seed=w.seed * 16 + 3 + 100 * l)
                        for l, (f, _, _) in enumerate(w.layer_list())]
        self.screen = self.screens[0]
        self.noise_seed = w.seed * 16 + 2
        self._xg, self._yg = self.sensor.fine_coords(w.pitch)
        self._shift = [(0.0, 0.0)]

    def _shift_at(self, k: int):
        while len(self._shift) <= k:
            j = len(self._shift) - 1
            v, ang = self.w.wind_at(j)
            sx, sy = self._shift[-1]
            dt = 1.0 / self.w.frame_rate
            self._shift.append((sx + v * math.cos(ang) * dt, sy + v * math.sin(ang) * dt))
        return self._shift[k]

    def phase_fine(self, k: int) -> np.ndarray:
        if k < 0:
            k = 0
        if self.w.layers:
            out = np.zeros_like(self._xg)
            for l, scr in enumerate(self.screens):
                sx, sy = self.w._shift(k, l)
                out += scr.sample(self._xg + sx, self._yg + sy)
            return out
        sx, sy = self._shift_at(k)
        return self.w.screen_scale(k) * self.screen.sample(self._xg + sx, self._yg + sy)

    def frames(self, k0: int, k1: int):
        """Frames k0..k1-1: returns dict of
        slopes (nf, 2, N, N) float64 [x then y, every subaperture, noise included],
        phi_act (nf, N+1, N+1) float64 true phase at the actuator points at frame k,
        sigma (nf,) noise std used at each frame."""
        n = self.w.n_sub
        nf = k1 - k0
        slopes = np.empty((nf, 2, n, n))
        phi = np.empty((nf, n + 1, n + 1))
        sig = np.empty(nf)
        for i, k in enumerate(range(k0, k1)):
            sxs, sys_, _ = self.sensor.measure(self.phase_fine(k - self.w.obs_block))
            _, _, pa = self.sensor.measure(self.phase_fine(k))
            rng = np.random.default_rng([self.noise_seed, k])
            s = self.w.sigma_at(k)
            slopes[i, 0] = sxs + s * rng.standard_normal((n, n))
            slopes[i, 1] = sys_ + s * rng.standard_normal((n, n))
            phi[i] = pa
            sig[i] = s
        return {"slopes": slopes, "phi_act": phi, "sigma": sig}


def _compressed_chunk(args):
    w, k0, k1, sub_valid, act_valid = args
    fr = TruthStream(w).frames(k0, k1)
    s = fr["slopes"]
    y = np.concatenate([s[:, 0][:, sub_valid], s[:, 1][:, sub_valid]], axis=1).astype(np.float32)
    return y, fr["phi_act"][:, act_valid].astype(np.float32), fr["sigma"]


def compressed_frames(w: Workload, k0: int, k1: int, sub_valid: np.ndarray, act_valid: np.ndarray,
                      workers: int = 1):
    """Frames k0..k1-1 of TruthStream(w) on the given valid subapertures / actuators: slopes
    (nf, p) FP32 (all x then all y), true actuator phase (nf, n_act) FP32 and the noise std
    (nf,).  With workers > 1 the frames are made in chunks by spawned processes (each frame
    depends only on its index, so the result is the same)."""
    sub_valid = np.asarray(sub_valid, dtype=bool)
    act_valid = np.asarray(act_valid, dtype=bool)
    n = k1 - k0
    if workers <= 1 or n < 64:
        return _compressed_chunk((w, k0, k1, sub_valid, act_valid))
    import concurrent.futures
    import multiprocessing
    edges = np.linspace(k0, k1, workers + 1).astype(int)
    jobs = [(w, int(a), int(b), sub_valid, act_valid) for a, b in zip(edges[:-1], edges[1:]) if b > a]
    with concurrent.futures.ProcessPoolExecutor(max_workers=workers,
                                                mp_context=multiprocessing.get_context("spawn")) as ex:
        parts = list(ex.map(_compressed_chunk, jobs))
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
            np.concatenate([p[2] for p in parts]))
