"""ctypes binding of libletkf (include/letkf.h): argument marshalling only.

Every entry point of the C ABI has a Python function of the same name taking
plain integers for pointers.  The library is loaded from this package's lib/
directory; if it is missing, loading raises instead of falling back to any
other implementation.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libletkf.so")

LETKF_OK, LETKF_EINVAL, LETKF_ENOMEM, LETKF_ECUDA = 0, -1, -2, -3
LETKF_ETIMEOUT, LETKF_ENONFINITE, LETKF_ESTATE, LETKF_ENOCONV = -4, -5, -6, -7
LETKF_ESCRATCH = -8
LETKF_PREC_FP64, LETKF_PREC_FP32, LETKF_PREC_MIXED = 0, 1, 2
LETKF_PATH_PLAIN, LETKF_PATH_FUSED = 0, 1


class letkf_params(ctypes.Structure):
    _fields_ = [
        ("n_sub", ctypes.c_int),
        ("sub_valid", ctypes.POINTER(ctypes.c_ubyte)),
        ("obstruction", ctypes.c_double),
        ("ar1_a", ctypes.c_double),
        ("obs_block", ctypes.c_int),
        ("q_sqrt", ctypes.POINTER(ctypes.c_double)),
        ("q_white", ctypes.c_double),
        ("p0_sqrt", ctypes.POINTER(ctypes.c_double)),
        ("sigma", ctypes.c_double),
        ("m", ctypes.c_int),
        ("dom_sub", ctypes.c_int),
        ("halo", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("path", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


class letkf_info(ctypes.Structure):
    _fields_ = [
        ("n_sub", ctypes.c_int), ("n_act", ctypes.c_int), ("n_subv", ctypes.c_int), ("n", ctypes.c_int),
        ("p", ctypes.c_int), ("m", ctypes.c_int), ("n_domains", ctypes.c_int), ("n_loc_max", ctypes.c_int),
        ("p_loc_max", ctypes.c_int), ("rank_max", ctypes.c_int), ("state_bytes", ctypes.c_int),
        ("precision", ctypes.c_int), ("path", ctypes.c_int), ("frame", ctypes.c_ulonglong),
        ("device_bytes", ctypes.c_size_t), ("n_domains_observing", ctypes.c_int),
        ("sum_p_loc", ctypes.c_longlong), ("sum_n_loc", ctypes.c_longlong),
    ]


N_STAGES = 8


class letkf_stage_times(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * N_STAGES), ("launches", ctypes.c_int * N_STAGES)]


_VP = ctypes.c_void_p
_SIGS = {
    "letkf_create": (ctypes.c_int, [ctypes.POINTER(letkf_params), ctypes.POINTER(ctypes.c_void_p)]),
    "letkf_destroy": (ctypes.c_int, [_VP]),
    "letkf_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(letkf_info)]),
    "letkf_get_geometry": (ctypes.c_int, [_VP, _VP, _VP]),
    "letkf_analyze": (ctypes.c_int, [_VP, _VP, ctypes.c_double]),
    "letkf_forecast": (ctypes.c_int, [_VP, _VP]),
    "letkf_step": (ctypes.c_int, [_VP, _VP, ctypes.c_double, _VP]),
    "letkf_get_state": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_ulonglong)]),
    "letkf_set_state": (ctypes.c_int, [_VP, _VP, ctypes.c_ulonglong]),
    "letkf_sync": (ctypes.c_int, [_VP]),
    "letkf_analyze_static": (ctypes.c_int, [_VP, _VP, ctypes.c_double, _VP]),
    "letkf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "letkf_profile": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "letkf_stage_name": (ctypes.c_char_p, [ctypes.c_int]),
    "letkf_umma_selftest": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           _VP]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libletkf.so (built by paper_1310_5954_gb300.build); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libletkf.so not found at {path}: run paper_1310_5954_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LETKFError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = letkf_status_string(status)
        super().__init__(f"{where}: {msg} ({status})" if where else f"{msg} ({status})")


def _check(rc: int, where: str) -> int:
    if rc != LETKF_OK:
        raise LETKFError(rc, where)
    return rc


def letkf_status_string(status: int) -> str:
    return load().letkf_status_string(int(status)).decode()


def letkf_create(params: letkf_params) -> int:
    out = ctypes.c_void_p()
    _check(load().letkf_create(ctypes.byref(params), ctypes.byref(out)), "letkf_create")
    return out.value


def letkf_destroy(ctx: int) -> int:
    return load().letkf_destroy(ctx)


def letkf_get_info(ctx: int) -> letkf_info:
    info = letkf_info()
    _check(load().letkf_get_info(ctx, ctypes.byref(info)), "letkf_get_info")
    return info


def letkf_get_geometry(ctx: int, sub_valid_ptr: int, act_valid_ptr: int) -> int:
    return _check(load().letkf_get_geometry(ctx, sub_valid_ptr, act_valid_ptr), "letkf_get_geometry")


def letkf_analyze(ctx: int, y_ptr: int, sigma: float = 0.0) -> int:
    return _check(load().letkf_analyze(ctx, y_ptr, float(sigma)), "letkf_analyze")


def letkf_forecast(ctx: int, v_ptr: int = 0) -> int:
    return _check(load().letkf_forecast(ctx, v_ptr or None), "letkf_forecast")


def letkf_step(ctx: int, y_ptr: int, sigma: float = 0.0, xpred_ptr: int = 0) -> int:
    return _check(load().letkf_step(ctx, y_ptr, float(sigma), xpred_ptr or None), "letkf_step")


def letkf_get_state(ctx: int, x_ptr: int = 0) -> int:
    frame = ctypes.c_ulonglong()
    _check(load().letkf_get_state(ctx, x_ptr or None, ctypes.byref(frame)), "letkf_get_state")
    return frame.value


def letkf_set_state(ctx: int, x_ptr: int, frame: int) -> int:
    return _check(load().letkf_set_state(ctx, x_ptr, int(frame)), "letkf_set_state")


def letkf_analyze_static(ctx: int, y_ptr: int, sigma: float, xa_ptr: int) -> int:
    """Allocation-free analysis into the caller's buffer; returns the status code (no raise)."""
    return load().letkf_analyze_static(ctx, y_ptr, float(sigma), xa_ptr)


def letkf_sync(ctx: int) -> int:
    """Returns the latched device status (0 when clean) without raising."""
    return load().letkf_sync(ctx)


def letkf_profile(ctx: int, enable: int):
    """enable=1: start recording stage times; enable=0: stop and return {stage: (ms, launches)}."""
    if enable:
        _check(load().letkf_profile(ctx, 1, None), "letkf_profile")
        return None
    t = letkf_stage_times()
    _check(load().letkf_profile(ctx, 0, ctypes.byref(t)), "letkf_profile")
    return {letkf_stage_name(i): (t.ms[i], t.launches[i]) for i in range(N_STAGES) if t.launches[i]}


def letkf_stage_name(stage: int) -> str:
    return load().letkf_stage_name(int(stage)).decode()


def letkf_umma_selftest(a_ptr: int, b_ptr: int, d_ptr: int, n: int, k: int, terms: int, b_layout: int = 0,
                        stream: int = 0) -> int:
    return load().letkf_umma_selftest(a_ptr, b_ptr, d_ptr, n, k, terms, b_layout, stream or None)


def declared_functions(header: str) -> list:
    """Names of the functions declared in a letkf header (used to check the exports)."""
    import re
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(letkf_\w+)\s*\(", text, re.M)))
