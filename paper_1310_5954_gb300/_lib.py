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
LETKF_ESCRATCH, LETKF_EBUSY = -8, -9
LETKF_PREC_FP64, LETKF_PREC_FP32, LETKF_PREC_MIXED = 0, 1, 2
LETKF_PATH_PLAIN, LETKF_PATH_FUSED, LETKF_PATH_GLOBAL = 0, 1, 2
LETKF_PISTON_OFF, LETKF_PISTON_OUTPUT, LETKF_PISTON_IN_LOOP = 0, 1, 2


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
        ("ar2_a", ctypes.c_double),
        ("piston", ctypes.c_int),
        ("simt_q_max", ctypes.c_int),
        ("dom_offset", ctypes.c_int),
    ]


class letkf_info(ctypes.Structure):
    _fields_ = [
        ("n_sub", ctypes.c_int), ("n_act", ctypes.c_int), ("n_subv", ctypes.c_int), ("n", ctypes.c_int),
        ("p", ctypes.c_int), ("m", ctypes.c_int), ("n_domains", ctypes.c_int), ("n_loc_max", ctypes.c_int),
        ("p_loc_max", ctypes.c_int), ("state_bytes", ctypes.c_int),
        ("precision", ctypes.c_int), ("path", ctypes.c_int), ("frame", ctypes.c_ulonglong),
        ("device_bytes", ctypes.c_size_t), ("n_domains_observing", ctypes.c_int),
        ("sum_p_loc", ctypes.c_longlong), ("sum_n_loc", ctypes.c_longlong),
        ("simt_q", ctypes.c_int), ("n_domains_simt", ctypes.c_int),
    ]


class letkf_server_params(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget", ctypes.c_ulonglong), ("max_systems", ctypes.c_int),
                ("slots", ctypes.c_int), ("max_pending", ctypes.c_int), ("max_batch", ctypes.c_int)]


class letkf_frame_record(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int), ("status", ctypes.c_int), ("frame", ctypes.c_ulonglong),
                ("t_arrival_ns", ctypes.c_longlong), ("t_launch_ns", ctypes.c_longlong),
                ("t_done_ns", ctypes.c_longlong), ("batch_systems", ctypes.c_int), ("slot", ctypes.c_int),
                ("t_dev_start_ns", ctypes.c_longlong), ("t_dev_end_ns", ctypes.c_longlong)]


class letkf_server_info(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_ulonglong), ("hbm_used", ctypes.c_ulonglong), ("systems", ctypes.c_int),
                ("frames_waiting", ctypes.c_int), ("frames_in_flight", ctypes.c_int),
                ("frames_done", ctypes.c_ulonglong), ("batches", ctypes.c_ulonglong),
                ("batched_systems", ctypes.c_ulonglong)]


class letkf_domain_sizes(ctypes.Structure):
    _fields_ = [("n_sub", ctypes.c_int), ("n_act", ctypes.c_int), ("n_subv", ctypes.c_int), ("n_dom", ctypes.c_int),
                ("blocks_per_side", ctypes.c_int), ("own_total", ctypes.c_int), ("obs_total", ctypes.c_int),
                ("halo_total", ctypes.c_int)]


class letkf_tuning(ctypes.Structure):
    _fields_ = [("fused_grid", ctypes.c_int), ("graph", ctypes.c_int)]


N_STAGES = 9


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
    "letkf_footprint": (ctypes.c_int, [ctypes.POINTER(letkf_params), ctypes.POINTER(ctypes.c_ulonglong)]),
    "letkf_wait_selftest": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, _VP]),
    "letkf_gemm_selftest": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, _VP]),
    "letkf_set_graph": (ctypes.c_int, [_VP, ctypes.c_int]),
    "letkf_domain_tables": (ctypes.c_int, [ctypes.POINTER(letkf_params), ctypes.POINTER(letkf_domain_sizes),
                                           _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "letkf_get_graph": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "letkf_set_domain_mask": (ctypes.c_int, [_VP, _VP]),
    "letkf_global_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "letkf_set_capture": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_longlong]),
    "letkf_step_pair": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, _VP]),
    "letkf_fused_plan": (ctypes.c_int, [ctypes.POINTER(letkf_params), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "letkf_piston_operator": (ctypes.c_int, [ctypes.POINTER(letkf_params), _VP, ctypes.POINTER(ctypes.c_int)]),
    "letkf_get_tuning": (ctypes.c_int, [_VP, ctypes.POINTER(letkf_tuning)]),
    "letkf_set_tuning": (ctypes.c_int, [_VP, ctypes.POINTER(letkf_tuning)]),
    "letkf_autotune": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(letkf_tuning),
                                      ctypes.POINTER(ctypes.c_double)]),
    # letkf_serve.h
    "letkf_now_ns": (ctypes.c_longlong, []),
    "letkf_server_create": (ctypes.c_int, [ctypes.POINTER(letkf_server_params), ctypes.POINTER(ctypes.c_void_p)]),
    "letkf_server_destroy": (ctypes.c_int, [_VP]),
    "letkf_server_admit": (ctypes.c_int, [_VP, ctypes.POINTER(letkf_params), ctypes.POINTER(ctypes.c_int)]),
    "letkf_server_release": (ctypes.c_int, [_VP, ctypes.c_int]),
    "letkf_server_set_output": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int]),
    "letkf_server_submit": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_double, ctypes.c_longlong]),
    "letkf_server_pump": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "letkf_server_drain": (ctypes.c_int, [_VP]),
    "letkf_server_records": (ctypes.c_int, [_VP, ctypes.POINTER(letkf_frame_record), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]),
    "letkf_server_context": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "letkf_server_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(letkf_server_info)]),
    "letkf_server_replay": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.POINTER(ctypes.c_int)]),
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


def letkf_set_graph(ctx: int, enable: int) -> int:
    return _check(load().letkf_set_graph(ctx, int(enable)), "letkf_set_graph")


def letkf_get_graph(ctx: int) -> int:
    v = ctypes.c_int()
    _check(load().letkf_get_graph(ctx, ctypes.byref(v)), "letkf_get_graph")
    return v.value


def letkf_get_tuning(ctx: int) -> dict:
    t = letkf_tuning()
    _check(load().letkf_get_tuning(ctx, ctypes.byref(t)), "letkf_get_tuning")
    return {"fused_grid": t.fused_grid, "graph": t.graph}


def letkf_set_tuning(ctx: int, fused_grid: int, graph: int) -> int:
    t = letkf_tuning(int(fused_grid), int(graph))
    return _check(load().letkf_set_tuning(ctx, ctypes.byref(t)), "letkf_set_tuning")


def letkf_autotune(ctx: int, y_ptr: int, frames: int = 20):
    """Returns ({'fused_grid', 'graph'}, ms per frame of the best candidate)."""
    t = letkf_tuning()
    ms = ctypes.c_double()
    _check(load().letkf_autotune(ctx, y_ptr, int(frames), ctypes.byref(t), ctypes.byref(ms)), "letkf_autotune")
    return {"fused_grid": t.fused_grid, "graph": t.graph}, ms.value


def letkf_domain_tables(params: letkf_params) -> dict:
    """Host-side geometry and domains (numpy int32 arrays) of letkf_domain_tables."""
    import numpy as np
    sz = letkf_domain_sizes()
    _check(load().letkf_domain_tables(ctypes.byref(params), ctypes.byref(sz), None, None, None, None, None, None,
                                      None), "letkf_domain_tables")
    out = {"own_off": np.zeros(sz.n_dom + 1, np.int32), "own": np.zeros(sz.own_total, np.int32),
           "obs_off": np.zeros(sz.n_dom + 1, np.int32), "obs_sub": np.zeros(sz.obs_total, np.int32),
           "halo_off": np.zeros(sz.n_dom + 1, np.int32), "halo": np.zeros(sz.halo_total, np.int32),
           "block": np.zeros(sz.n_dom, np.int32)}
    _check(load().letkf_domain_tables(ctypes.byref(params), ctypes.byref(sz),
                                      *[out[k].ctypes.data for k in ("own_off", "own", "obs_off", "obs_sub",
                                                                      "halo_off", "halo", "block")]),
           "letkf_domain_tables")
    out.update({f: getattr(sz, f) for f, _ in letkf_domain_sizes._fields_})
    return out


def letkf_fused_plan(params: letkf_params):
    """(dynamic shared memory bytes, SIMT threshold, SIMT domains) of the fused path, host only."""
    smem, q, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().letkf_fused_plan(ctypes.byref(params), ctypes.byref(smem), ctypes.byref(q), ctypes.byref(n)),
           "letkf_fused_plan")
    return smem.value, q.value, n.value


def letkf_piston_operator(params: letkf_params):
    """The differential-piston least-squares operator K (n_dom x n_dom float64) on the host."""
    import numpy as np
    nd = ctypes.c_int()
    _check(load().letkf_piston_operator(ctypes.byref(params), None, ctypes.byref(nd)), "letkf_piston_operator")
    K = np.zeros((nd.value, nd.value), np.float64)
    _check(load().letkf_piston_operator(ctypes.byref(params), K.ctypes.data, ctypes.byref(nd)),
           "letkf_piston_operator")
    return K


def letkf_set_domain_mask(ctx: int, active_ptr: int) -> int:
    return _check(load().letkf_set_domain_mask(ctx, active_ptr), "letkf_set_domain_mask")


def letkf_global_stats(ctx: int):
    """(Newton-Schulz steps, spectral bound s) of the last global-path analysis."""
    n = ctypes.c_int()
    sb = ctypes.c_double()
    _check(load().letkf_global_stats(ctx, ctypes.byref(n), ctypes.byref(sb)), "letkf_global_stats")
    return n.value, sb.value


def letkf_step_pair(ctx_a: int, ctx_b: int, y_ptr: int, sigma: float, xpred_ptr: int) -> int:
    return _check(load().letkf_step_pair(ctx_a, ctx_b, y_ptr, sigma, xpred_ptr), "letkf_step_pair")


def letkf_set_capture(ctx: int, domain: int, cap_ptr: int, cap_floats: int) -> int:
    return _check(load().letkf_set_capture(ctx, domain, cap_ptr, cap_floats), "letkf_set_capture")


def letkf_footprint(params: letkf_params) -> int:
    out = ctypes.c_ulonglong()
    _check(load().letkf_footprint(ctypes.byref(params), ctypes.byref(out)), "letkf_footprint")
    return out.value


# ---- letkf_serve.h ---------------------------------------------------------------------------
def letkf_now_ns() -> int:
    return load().letkf_now_ns()


def letkf_server_create(params: letkf_server_params) -> int:
    out = ctypes.c_void_p()
    _check(load().letkf_server_create(ctypes.byref(params), ctypes.byref(out)), "letkf_server_create")
    return out.value


def letkf_server_destroy(server: int) -> int:
    return load().letkf_server_destroy(server)


def letkf_server_admit(server: int, params: letkf_params) -> int:
    """System id; raises LETKFError (status LETKF_EBUSY when the HBM budget is full)."""
    sid = ctypes.c_int(-1)
    _check(load().letkf_server_admit(server, ctypes.byref(params), ctypes.byref(sid)), "letkf_server_admit")
    return sid.value


def letkf_server_release(server: int, sid: int) -> int:
    return _check(load().letkf_server_release(server, int(sid)), "letkf_server_release")


def letkf_server_set_output(server: int, sid: int, host_ptr: int, n_frames: int) -> int:
    return _check(load().letkf_server_set_output(server, int(sid), host_ptr or None, int(n_frames)),
                  "letkf_server_set_output")


def letkf_server_submit(server: int, sid: int, y_ptr: int, sigma: float = 0.0, t_arrival_ns: int = 0) -> int:
    """Returns LETKF_OK or LETKF_EBUSY (queue full); raises on other errors."""
    rc = load().letkf_server_submit(server, int(sid), y_ptr, float(sigma), int(t_arrival_ns))
    if rc not in (LETKF_OK, LETKF_EBUSY):
        raise LETKFError(rc, "letkf_server_submit")
    return rc


def letkf_server_pump(server: int) -> int:
    n = ctypes.c_int()
    _check(load().letkf_server_pump(server, ctypes.byref(n)), "letkf_server_pump")
    return n.value


def letkf_server_drain(server: int) -> int:
    return _check(load().letkf_server_drain(server), "letkf_server_drain")


def letkf_server_records(server: int, max_records: int = 4096) -> list:
    buf = (letkf_frame_record * max_records)()
    out = []
    while True:
        n = ctypes.c_int()
        _check(load().letkf_server_records(server, buf, max_records, ctypes.byref(n)), "letkf_server_records")
        out.extend({f: getattr(buf[i], f) for f, _ in letkf_frame_record._fields_} for i in range(n.value))
        if n.value < max_records:
            return out


def letkf_server_context(server: int, sid: int) -> int:
    out = ctypes.c_void_p()
    _check(load().letkf_server_context(server, int(sid), ctypes.byref(out)), "letkf_server_context")
    return out.value


def letkf_server_get_info(server: int) -> dict:
    info = letkf_server_info()
    _check(load().letkf_server_get_info(server, ctypes.byref(info)), "letkf_server_get_info")
    return {f: getattr(info, f) for f, _ in letkf_server_info._fields_}


def letkf_server_replay(server: int, sys_ids, t_ns, y_ptrs, sigma=None) -> int:
    """Real-time replay of an arrival trace (arrays of equal length); returns the refused count."""
    n = len(sys_ids)
    s = (ctypes.c_int * n)(*[int(v) for v in sys_ids])
    t = (ctypes.c_longlong * n)(*[int(v) for v in t_ns])
    y = (ctypes.c_void_p * n)(*[int(v) for v in y_ptrs])
    sg = None if sigma is None else (ctypes.c_double * n)(*[float(v) for v in sigma])
    refused = ctypes.c_int()
    _check(load().letkf_server_replay(server, n, s, t, y, sg, ctypes.byref(refused)), "letkf_server_replay")
    return refused.value


def letkf_wait_selftest(limit_cycles: int, arrive: int, stream: int = 0) -> int:
    """Status of the bounded-wait self-test (no raise): LETKF_OK or LETKF_ETIMEOUT."""
    return load().letkf_wait_selftest(int(limit_cycles), int(arrive), stream or None)


def declared_functions(header: str) -> list:
    """Names of the functions declared in a letkf header (used to check the exports)."""
    import re
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:int|long long|const char\*)\s+(letkf_\w+)\s*\(", text, re.M)))
