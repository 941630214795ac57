"""Serving loop over the C ABI of include/letkf_serve.h: many AO systems on one GPU.

The scheduling, batching, copies and timing all run in libletkf (native code); this
class marshals numpy host arrays and torch device tensors into its calls.
"""

from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _lib
from .letkf import make_params


class Server:
    """Device-resident ensembles of many systems, frames batched continuously into one kernel launch."""

    def __init__(self, device: Optional[int] = None, hbm_budget: int = 0, max_systems: int = 64, slots: int = 2,
                 max_pending: int = 64, max_batch: int = 32):
        import torch
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("Server needs a CUDA device")
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = torch.device("cuda", dev)
        p = _lib.letkf_server_params()
        p.device, p.hbm_budget, p.max_systems = dev, int(hbm_budget), int(max_systems)
        p.slots, p.max_pending, p.max_batch = int(slots), int(max_pending), int(max_batch)
        with torch.cuda.device(self.device):
            self.srv = _lib.letkf_server_create(p)
        self.systems = {}     # id -> letkf_info
        self._outputs = {}

    def admit(self, **kw) -> int:
        """Admit a system (keyword arguments as for LETKF; path is forced to 'fused').  Raises
        LETKFError with status LETKF_EBUSY when its footprint does not fit the HBM budget left."""
        kw = dict(kw)
        kw["path"] = "fused"
        kw.setdefault("precision", "mixed")
        p, keep = make_params(**kw)
        sid = _lib.letkf_server_admit(self.srv, p)
        del keep
        self.systems[sid] = _lib.letkf_get_info(_lib.letkf_server_context(self.srv, sid))
        return sid

    def release(self, sid: int) -> None:
        _lib.letkf_server_release(self.srv, sid)
        self.systems.pop(sid, None)
        self._outputs.pop(sid, None)

    def set_output(self, sid: int, n_frames: int) -> np.ndarray:
        """Keep every completed frame's prediction: row k % n_frames of the returned array."""
        out = np.zeros((int(n_frames), self.systems[sid].n_act), dtype=np.float32)
        _lib.letkf_server_set_output(self.srv, sid, out.ctypes.data, n_frames)
        self._outputs[sid] = out
        return out

    def submit(self, sid: int, y: np.ndarray, sigma: float = 0.0, t_arrival_ns: int = 0) -> int:
        """Queue one frame of slopes (host FP32, p values); returns LETKF_OK or LETKF_EBUSY."""
        y = np.ascontiguousarray(y, dtype=np.float32)
        if y.size != self.systems[sid].p:
            raise ValueError(f"system {sid} takes {self.systems[sid].p} slopes, got {y.size}")
        return _lib.letkf_server_submit(self.srv, sid, y.ctypes.data, sigma, t_arrival_ns)

    def pump(self) -> int:
        return _lib.letkf_server_pump(self.srv)

    def drain(self) -> None:
        _lib.letkf_server_drain(self.srv)

    def records(self) -> list:
        return _lib.letkf_server_records(self.srv)

    def info(self) -> dict:
        return _lib.letkf_server_get_info(self.srv)

    def state(self, sid: int):
        """(ensemble n x m as a torch device tensor, frame counter) of a system, between frames."""
        ctx = _lib.letkf_server_context(self.srv, sid)
        inf = self.systems[sid]
        out = self._torch.empty((inf.n, inf.m), dtype=self._torch.float32, device=self.device)
        frame = _lib.letkf_get_state(ctx, out.data_ptr())
        _lib.letkf_sync(ctx)
        return out, frame

    def replay(self, sys_ids, t_ns, ys, sigma=None) -> int:
        """Real-time replay of an arrival trace: ys[i] (host FP32 arrays, kept alive by the caller)
        arrives for system sys_ids[i] at t_ns[i] after the start.  Returns the refused count."""
        ptrs = []
        for s, y in zip(sys_ids, ys):
            if not (isinstance(y, np.ndarray) and y.dtype == np.float32 and y.flags.c_contiguous
                    and y.size == self.systems[int(s)].p):
                raise ValueError("replay wants contiguous float32 slope arrays of each system's size")
            ptrs.append(y.ctypes.data)
        return _lib.letkf_server_replay(self.srv, sys_ids, t_ns, ptrs, sigma)

    def close(self) -> None:
        if getattr(self, "srv", None):
            _lib.letkf_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def now_ns() -> int:
    return _lib.letkf_now_ns()
