"""A context object over the C ABI that takes torch device tensors.

All arithmetic happens in libletkf's kernels; this class only allocates output
tensors with torch, checks shapes and dtypes, and passes raw pointers and the
current torch stream.
"""

from __future__ import annotations

import ctypes
import json
import os
from typing import Optional

import numpy as np

from . import _lib

_PREC = {"fp64": _lib.LETKF_PREC_FP64, "fp32": _lib.LETKF_PREC_FP32, "mixed": _lib.LETKF_PREC_MIXED}
_PATH = {"plain": _lib.LETKF_PATH_PLAIN, "fused": _lib.LETKF_PATH_FUSED, "global": _lib.LETKF_PATH_GLOBAL}
_PISTON = {"off": _lib.LETKF_PISTON_OFF, "output": _lib.LETKF_PISTON_OUTPUT, "in_loop": _lib.LETKF_PISTON_IN_LOOP}


def make_params(n_sub: int, m: int, ar1_a: float, sigma: float, dom_sub: int = 4, halo: int = 2,
                obstruction: float = 0.0, sub_valid: Optional[np.ndarray] = None,
                q_sqrt: Optional[np.ndarray] = None, q_white: float = 0.0, p0_sqrt: Optional[np.ndarray] = None,
                precision: str = "fp32", path: str = "plain", seed: int = 0, obs_block: int = 1,
                ar2_a: float = 0.0, piston: str = "off", simt_q_max: int = 0, dom_offset: int = 0):
    """letkf_params for the C ABI, and the host arrays it points to (keep them alive while it is used).

    piston: "off", "output" or "in_loop" (differential-piston removal between domains);
    simt_q_max: fused path, domains with min(p_loc, m) <= this take the FP32 analysis on the CUDA
    cores (0: the library default, negative: every domain on the tensor cores);
    dom_offset: shift of the domains' block grid in subapertures (0 <= dom_offset < dom_sub).
    """
    p = _lib.letkf_params()
    keep = []
    p.n_sub = int(n_sub)
    if sub_valid is not None:
        sv = np.ascontiguousarray(sub_valid, dtype=np.uint8)
        keep.append(sv)
        p.sub_valid = sv.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    p.obstruction = float(obstruction)
    p.ar1_a = float(ar1_a)
    p.obs_block = int(obs_block)
    if q_sqrt is not None:
        qs = np.ascontiguousarray(q_sqrt, dtype=np.float64)
        keep.append(qs)
        p.q_sqrt = qs.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.q_white = float(q_white)
    if p0_sqrt is not None:
        ps = np.ascontiguousarray(p0_sqrt, dtype=np.float64)
        keep.append(ps)
        p.p0_sqrt = ps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.sigma = float(sigma)
    p.m = int(m)
    p.dom_sub = int(dom_sub)
    p.halo = int(halo)
    p.precision = _PREC[precision]
    p.path = _PATH[path]
    p.seed = int(seed)
    p.ar2_a = float(ar2_a)
    if piston not in _PISTON:
        raise ValueError(f"piston must be one of {sorted(_PISTON)}")
    p.piston = _PISTON[piston]
    p.simt_q_max = int(simt_q_max)
    p.dom_offset = int(dom_offset)
    return p, keep


def footprint(**kw) -> int:
    """Device bytes a context with these parameters (as for LETKF) holds once created."""
    p, keep = make_params(**kw)
    return _lib.letkf_footprint(p)


class LETKF:
    """One adaptive-optics system's local ETKF, resident on one GPU."""

    def __init__(self, n_sub: int, m: int, ar1_a: float, sigma: float, dom_sub: int = 4, halo: int = 2,
                 obstruction: float = 0.0, sub_valid: Optional[np.ndarray] = None,
                 q_sqrt: Optional[np.ndarray] = None, q_white: float = 0.0,
                 p0_sqrt: Optional[np.ndarray] = None, precision: str = "fp32", path: str = "plain",
                 seed: int = 0, obs_block: int = 1, device: Optional[int] = None, stream=None,
                 ar2_a: float = 0.0, piston: str = "off", simt_q_max: int = 0, dom_offset: int = 0):
        import torch
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("LETKF needs a CUDA device")
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = torch.device("cuda", dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p, keep = make_params(n_sub=n_sub, m=m, ar1_a=ar1_a, sigma=sigma, dom_sub=dom_sub, halo=halo,
                              obstruction=obstruction, sub_valid=sub_valid, q_sqrt=q_sqrt, q_white=q_white,
                              p0_sqrt=p0_sqrt, precision=precision, path=path, seed=seed, obs_block=obs_block,
                              ar2_a=ar2_a, piston=piston, simt_q_max=simt_q_max, dom_offset=dom_offset)
        self._keep = keep
        p.device = dev
        p.stream = self.stream.cuda_stream
        with torch.cuda.device(self.device):
            self.ctx = _lib.letkf_create(p)
        self._keep = []
        self.info = _lib.letkf_get_info(self.ctx)
        self.noise_kind = "dense" if q_sqrt is not None else ("white" if q_white > 0 else "none")
        self.dtype = torch.float64 if self.info.state_bytes == 8 else torch.float32
        self.precision, self.path = precision, path
        self.piston = piston

    # --- geometry -------------------------------------------------------------------
    def geometry(self):
        n = self.info.n_sub
        sv = np.zeros((n, n), dtype=np.uint8)
        av = np.zeros((n + 1, n + 1), dtype=np.uint8)
        _lib.letkf_get_geometry(self.ctx, sv.ctypes.data, av.ctypes.data)
        return sv.astype(bool), av.astype(bool)

    # --- filter ---------------------------------------------------------------------
    def _dev(self, t, n, name):
        if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name}: expected a contiguous {self.dtype} tensor of {n} elements on {self.device}, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device} (contiguous: {t.is_contiguous()})")
        return t.data_ptr()

    def analyze(self, y, sigma: float = 0.0) -> None:
        _lib.letkf_analyze(self.ctx, self._dev(y, self.info.p, "y"), sigma)

    def forecast(self, v=None) -> None:
        ptr = 0 if v is None else self._dev(v, self.info.n_act * self.info.m, "v")
        _lib.letkf_forecast(self.ctx, ptr)

    def step(self, y, sigma: float = 0.0, out=None):
        """One frame (Eq. 1 order): analysis with y, forecast; returns x_hat(k+1|k) (n_act)."""
        if out is None:
            out = self._torch.empty(self.info.n_act, dtype=self.dtype, device=self.device)
        _lib.letkf_step(self.ctx, self._dev(y, self.info.p, "y"), sigma, self._dev(out, self.info.n_act, "out"))
        return out

    def get_state(self, out=None):
        if out is None:
            out = self._torch.empty((self.info.n, self.info.m), dtype=self.dtype, device=self.device)
        frame = _lib.letkf_get_state(self.ctx, self._dev(out, self.info.n * self.info.m, "x"))
        return out, frame

    def set_state(self, x, frame: int) -> None:
        _lib.letkf_set_state(self.ctx, self._dev(x, self.info.n * self.info.m, "x"), frame)

    def profile(self, enable: bool):
        """Start (True) or stop (False) stage timing; stopping returns {stage: (ms, launches)}."""
        return _lib.letkf_profile(self.ctx, 1 if enable else 0)

    def set_domain_mask(self, active=None) -> None:
        """Skip the domains whose entry of `active` (n_domains booleans) is False from the next
        analysis on (their actuators keep the forecast); None restores every domain."""
        if active is None:
            _lib.letkf_set_domain_mask(self.ctx, 0)
            return
        a = np.ascontiguousarray(active, dtype=np.uint8)
        if a.size != self.info.n_domains:
            raise ValueError(f"active: expected {self.info.n_domains} entries, got {a.size}")
        _lib.letkf_set_domain_mask(self.ctx, a.ctypes.data)

    def global_stats(self):
        """Global path: (Newton-Schulz steps, spectral bound s) of the last analysis."""
        return _lib.letkf_global_stats(self.ctx)

    def capture_transform(self, domain: Optional[int]):
        """Fused path, test instrument: from the next analysis on, domain `domain` (numbering of
        letkf_domain_tables) writes its mean weights and transform into a device buffer, which
        `captured()` reads; None stops it."""
        import torch
        if domain is None:
            _lib.letkf_set_capture(self.ctx, -1, 0, 0)
            self._cap = None
            return
        i = self.info
        n = 8 + i.m + max(i.m * i.m, 2 * max(i.p_loc_max, 1) * i.m)
        self._cap = torch.zeros(n, dtype=torch.float32, device=self.device)
        _lib.letkf_set_capture(self.ctx, int(domain), self._cap.data_ptr(), n)

    def captured(self) -> dict:
        """The captured domain's last analysis: form ("mm" or "dual", "tensor" or "simt"), the
        conditioning bound s, the Newton-Schulz steps, w_bar (m) and T (m x m; for the dual forms
        T = I - W^T M from the captured W and M = (I + Z)^-1 W, formed here in float64)."""
        self.sync()
        c = self._cap.cpu().numpy().astype(np.float64)
        form, q, s, it = int(c[0]), int(c[1]), c[2], int(c[3])
        m = self.info.m
        wbar = c[8:8 + m].copy()
        if form in (0, 2):
            T = c[8 + m:8 + m + m * m].reshape(m, m).copy()
            W = M = None
        else:
            W = c[8 + m:8 + m + q * m].reshape(q, m).copy()
            M = c[8 + m + q * m:8 + m + 2 * q * m].reshape(q, m).copy()
            T = np.eye(m) - W.T @ M
        return {"form": ("mm" if form in (0, 2) else "dual") + ("/tensor" if form in (0, 1) else "/simt"),
                "q": q, "s": s, "ns_steps": it, "wbar": wbar, "T": T, "W": W, "M": M}

    def set_graph(self, enable: bool) -> None:
        """Fused path: run each step as one CUDA graph launch, or as separate launches (default)."""
        _lib.letkf_set_graph(self.ctx, 1 if enable else 0)

    def tuning(self) -> dict:
        return _lib.letkf_get_tuning(self.ctx)

    def set_tuning(self, fused_grid: int = 0, graph: int = 0) -> None:
        _lib.letkf_set_tuning(self.ctx, fused_grid, graph)

    def tuning_key(self) -> str:
        """What the launch tuning depends on: geometry, domains, ensemble, path and the GPU."""
        import torch
        i = self.info
        props = torch.cuda.get_device_properties(self.device)
        return (f"n_sub={i.n_sub} n_act={i.n_act} n_subv={i.n_subv} domains={i.n_domains} m={i.m} "
                f"precision={self.precision} path={self.path} noise={self.noise_kind} "
                f"gpu={props.name} sms={props.multi_processor_count}")

    def autotune(self, y, frames: int = 20, cache: Optional[str] = None) -> dict:
        """Pick the fastest launch tuning for this system (letkf_autotune) and apply it.  With a
        cache path (JSON), a stored result for the same tuning_key() is applied without trials
        and new results are added to the file."""
        key = self.tuning_key()
        data = {}
        if cache and os.path.exists(cache):
            with open(cache) as fh:
                data = json.load(fh)
            if key in data:
                self.set_tuning(**data[key]["tuning"])
                return data[key]
        tuning, ms = _lib.letkf_autotune(self.ctx, self._dev(y, self.info.p, "y"), frames)
        rec = {"tuning": tuning, "ms_per_frame": ms, "frames": int(frames)}
        if cache:
            data[key] = rec
            tmp = cache + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(data, fh, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return rec

    def graph(self) -> bool:
        """Whether steps currently run as CUDA graph launches."""
        return bool(_lib.letkf_get_graph(self.ctx))

    def sync(self) -> int:
        return _lib.letkf_sync(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            _lib.letkf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LETKFPair:
    """Two local ETKFs run together on the same slopes with two domain partitions (Sect. 5): the
    second filter's block grid is shifted by `offset` subapertures (default dom_sub // 2) and its
    noise streams by its seed (default seed + 1); each step returns the mean of the two filters'
    predictions (letkf_step_pair).  Keyword arguments as for LETKF (fused path)."""

    def __init__(self, offset: Optional[int] = None, seed_b: Optional[int] = None, **kw):
        kw = dict(kw)
        kw["path"] = "fused"
        dom_sub = kw.get("dom_sub", 4)
        off = dom_sub // 2 if offset is None else int(offset)
        seed = int(kw.get("seed", 0))
        self.a = LETKF(**dict(kw, dom_offset=0))
        self.b = LETKF(**dict(kw, dom_offset=off, seed=seed + 1 if seed_b is None else int(seed_b),
                              stream=self.a.stream))
        self.info, self.dtype, self.device, self.stream = self.a.info, self.a.dtype, self.a.device, self.a.stream

    def step(self, y, sigma: float = 0.0, out=None):
        """One frame of both filters; returns the mean of their x_hat(k+1|k) (n_act)."""
        if out is None:
            out = self.a._torch.empty(self.info.n_act, dtype=self.dtype, device=self.device)
        _lib.letkf_step_pair(self.a.ctx, self.b.ctx, self.a._dev(y, self.info.p, "y"), sigma,
                             self.a._dev(out, self.info.n_act, "out"))
        return out

    def sync(self) -> int:
        ra, rb = self.a.sync(), self.b.sync()
        return ra or rb

    def close(self) -> None:
        self.a.close()
        self.b.close()
