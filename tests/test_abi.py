"""The C ABI library loads and exports every declared entry point (no GPU needed)."""

import ctypes
import os

import numpy as np

import pytest

from paper_1310_5954_gb300 import _lib
from paper_1310_5954_gb300 import build as builder

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    builder.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = []
    for h in HEADERS:
        names += _lib.declared_functions(h)
    assert "letkf_create" in names and "letkf_step" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_status_strings(lib):
    for s in range(-9, 1):
        assert _lib.letkf_status_string(s) not in ("", "unknown status")
    assert _lib.letkf_status_string(-99) == "unknown status"


def _params(**kw):
    p = _lib.letkf_params()
    p.n_sub, p.ar1_a, p.obs_block, p.sigma, p.m, p.dom_sub, p.halo = 8, 0.99, 1, 0.1, 20, 4, 1
    p.precision, p.path, p.q_white = _lib.LETKF_PREC_FP32, _lib.LETKF_PATH_PLAIN, 0.1
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [dict(m=1), dict(m=300), dict(sigma=0.0), dict(ar1_a=1.0), dict(obs_block=2),
                                 dict(n_sub=0), dict(dom_sub=0), dict(halo=-1), dict(precision=7),
                                 dict(path=3), dict(obstruction=1.5), dict(q_white=-1.0),
                                 dict(precision=_lib.LETKF_PREC_FP64, path=_lib.LETKF_PATH_FUSED),
                                 dict(precision=_lib.LETKF_PREC_MIXED, path=_lib.LETKF_PATH_PLAIN),
                                 dict(precision=_lib.LETKF_PREC_FP64, m=200), dict(dom_sub=12, halo=2),
                                 dict(piston=3), dict(piston=-1), dict(simt_q_max=129)])
def test_create_rejects_invalid_parameters_before_touching_the_device(lib, bad):
    p = _params(**bad)
    out = ctypes.c_void_p(1234)
    rc = lib.letkf_create(ctypes.byref(p), ctypes.byref(out))
    assert rc == _lib.LETKF_EINVAL
    assert out.value is None


def test_null_arguments(lib):
    assert lib.letkf_destroy(None) == _lib.LETKF_OK
    assert lib.letkf_sync(None) == _lib.LETKF_EINVAL
    assert lib.letkf_step(None, None, 0.0, None) == _lib.LETKF_EINVAL
    assert lib.letkf_create(None, None) == _lib.LETKF_EINVAL
    assert lib.letkf_set_domain_mask(None, None) == _lib.LETKF_EINVAL
    n, sb = ctypes.c_int(), ctypes.c_double()
    assert lib.letkf_global_stats(None, ctypes.byref(n), ctypes.byref(sb)) == _lib.LETKF_EINVAL
    nd = ctypes.c_int()
    assert lib.letkf_piston_operator(None, None, ctypes.byref(nd)) == _lib.LETKF_EINVAL
    assert lib.letkf_set_capture(None, 0, None, 0) == _lib.LETKF_EINVAL
    assert lib.letkf_step_pair(None, None, None, 0.0, None) == _lib.LETKF_EINVAL


def test_gemm_selftest_rejects_bad_shapes(lib):
    # checked before any device call
    assert lib.letkf_gemm_selftest(None, None, None, 1, 1, 1, 1, 64, 0, None) == _lib.LETKF_EINVAL
    one = ctypes.c_float()
    p = ctypes.byref(one)
    assert lib.letkf_gemm_selftest(p, p, p, 1, 1, 1, 2, 64, 0, None) == _lib.LETKF_EINVAL     # split
    assert lib.letkf_gemm_selftest(p, p, p, 1, 1, 1, 1, 96, 0, None) == _lib.LETKF_EINVAL     # tile width
    assert lib.letkf_gemm_selftest(p, p, p, 1, 1, 1, 1, 128, 1, None) == _lib.LETKF_EINVAL    # MN-major wide
    assert lib.letkf_gemm_selftest(p, p, p, 0, 1, 1, 1, 64, 0, None) == _lib.LETKF_EINVAL     # empty


def test_footprint_on_the_host(lib):
    from paper_1310_5954_gb300 import footprint
    base = dict(n_sub=8, m=20, ar1_a=0.99, sigma=0.1, dom_sub=4, halo=1, precision="mixed", path="fused")
    f0 = footprint(**base, q_white=0.1)
    n_act = 69                                  # 8x8 circular pupil (oracle geometry pins)
    f1 = footprint(**base, q_sqrt=np.eye(n_act))
    # a dense noise factor adds its BF16 tiles (one 128-row block x two 64-column tiles), one work
    # item (16 B), the block's table (4 ints) and the normals' tiles (2 x 64 rows x 32 columns, BF16)
    assert f1 - f0 == 2 * 128 * 64 * 2 + 16 + 16 + 2 * 64 * 32 * 2
    # only the tiles touching the lower triangle are kept for a lower-triangular factor: 16x16 has
    # 241 actuators, two row blocks of four column tiles, and 2 + 4 tiles of the eight
    b16 = dict(base, n_sub=16)
    rng = np.random.default_rng(0)
    full = rng.standard_normal((241, 241))
    assert footprint(**b16, q_sqrt=full) - footprint(**b16, q_sqrt=np.tril(full)) == 2 * 128 * 64 * 2
    # per member: the two ensemble buffers (2 x 2 n_act rows), the perturbation buffer and the
    # fused path's two noise buffers (3 x n_act), FP32; the BF16 normals tile widens from 32 to 48
    f2 = footprint(**dict(base, m=40), q_white=0.1)
    assert f2 - f0 == (4 + 1 + 2) * n_act * 20 * 4 + 128 * (48 - 32) * 2
    with pytest.raises(_lib.LETKFError):
        footprint(**dict(base, m=1))


def test_server_rejects_invalid_parameters(lib):
    out = ctypes.c_void_p(99)
    for bad in [dict(max_systems=0), dict(slots=9), dict(max_pending=0), dict(max_batch=33)]:
        p = _lib.letkf_server_params()
        p.device, p.max_systems, p.slots, p.max_pending, p.max_batch = 0, 4, 2, 8, 8
        for k, v in bad.items():
            setattr(p, k, v)
        assert lib.letkf_server_create(ctypes.byref(p), ctypes.byref(out)) == _lib.LETKF_EINVAL
        assert out.value is None
    assert lib.letkf_server_destroy(None) == _lib.LETKF_OK


def _plan(**kw):
    from paper_1310_5954_gb300.letkf import make_params
    p, keep = make_params(path="fused", precision="mixed", ar1_a=0.99, sigma=0.1, **kw)
    return _lib.letkf_fused_plan(p)


ELT = dict(n_sub=80, obstruction=0.28, m=100, dom_sub=4, halo=2)


@pytest.mark.parametrize("kw,q,n", [
    (dict(n_sub=8, m=20, dom_sub=4, halo=1), 32, 4),       # every domain of a 20-member system
    (ELT, 32, 16),                                          # the 16 edge domains with p_loc <= 24
    (dict(ELT, simt_q_max=-1), 0, 0),                       # off
    (dict(ELT, simt_q_max=24), 24, 16),
    (dict(ELT, simt_q_max=64), 64, 40),
    (dict(n_sub=40, obstruction=0.14, m=50, dom_sub=4, halo=2, simt_q_max=64), 64, 92),
    (dict(ELT, m=150), 0, 0),                               # the dual form stays on the tensor cores
])
def test_fused_plan_simt_threshold(lib, kw, q, n):
    smem, simt_q, n_simt = _plan(**kw)
    assert (simt_q, n_simt) == (q, n)
    assert 0 < smem <= 227 * 1024


def test_fused_plan_lowers_the_threshold_to_fit_shared_memory(lib):
    # every ELT domain would be q <= 100: the five q x q FP32 iteration matrices alone exceed what
    # is left of 227 KB, so the threshold drops until the workspace fits
    smem, q, n = _plan(**dict(ELT, simt_q_max=128))
    assert 64 <= q < 100 and n >= 40 and smem <= 227 * 1024


def test_fused_plan_rejects_other_paths_and_null_outputs(lib):
    from paper_1310_5954_gb300.letkf import make_params
    p, keep = make_params(n_sub=8, m=20, ar1_a=0.99, sigma=0.1, dom_sub=4, halo=1, path="plain")
    one = ctypes.c_int()
    assert lib.letkf_fused_plan(ctypes.byref(p), ctypes.byref(one), ctypes.byref(one), ctypes.byref(one)) == _lib.LETKF_EINVAL
    p.path = _lib.LETKF_PATH_FUSED
    assert lib.letkf_fused_plan(ctypes.byref(p), None, ctypes.byref(one), ctypes.byref(one)) == _lib.LETKF_EINVAL
    assert lib.letkf_fused_plan(None, ctypes.byref(one), ctypes.byref(one), ctypes.byref(one)) == _lib.LETKF_EINVAL


def test_headers_are_plain_c(tmp_path):
    # the boundary is a C ABI: both headers compile as strict C99 (and as C++)
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "h.c"
    src.write_text('#include "letkf.h"\n#include "letkf_serve.h"\nint main(void) { letkf_params p = {0}; (void)p; return 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, "-fsyntax-only", str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("n,obs,b,h,off", [(8, 0.0, 4, 1, 2), (40, 0.14, 4, 2, 2), (80, 0.28, 4, 2, 2),
                                           (13, 0.2, 4, 2, 3), (40, 0.14, 4, 2, 0), (10, 0.0, 3, 1, 1)])
def test_domain_tables_match_the_oracle_also_on_a_shifted_grid(lib, n, obs, b, h, off):
    """The library's domains (letkf_domain_tables) equal the oracle's, for the block grid shifted by
    dom_offset too (the second partition of Sect. 5)."""
    from oracle import geometry
    from paper_1310_5954_gb300.letkf import make_params
    p, keep = make_params(n_sub=n, m=20, ar1_a=0.9, sigma=0.1, dom_sub=b, halo=h, obstruction=obs, q_white=0.1,
                          precision="fp32", path="fused", dom_offset=off)
    tab = _lib.letkf_domain_tables(p)
    g = geometry.make_geometry(n, obs)
    doms = {(d.I, d.J): d for d in geometry.make_domains(g, b, h, offset=off)}
    nb = tab["blocks_per_side"]
    assert tab["n_dom"] == len(doms) and tab["n_act"] == g.n_act
    for k in range(tab["n_dom"]):
        d = doms[divmod(int(tab["block"][k]), nb)]
        own = tab["own"][tab["own_off"][k]:tab["own_off"][k + 1]]
        obs_sub = tab["obs_sub"][tab["obs_off"][k]:tab["obs_off"][k + 1]]
        assert np.array_equal(own, d.owned_act) and np.array_equal(obs_sub, d.obs_sub), k


def test_domain_offset_outside_the_block_is_refused(lib):
    from paper_1310_5954_gb300.letkf import make_params
    for off in (-1, 4):
        p, keep = make_params(n_sub=8, m=20, ar1_a=0.9, sigma=0.1, dom_sub=4, halo=1, q_white=0.1,
                              precision="fp32", path="fused", dom_offset=off)
        out = ctypes.c_void_p(1234)
        assert lib.letkf_create(ctypes.byref(p), ctypes.byref(out)) == _lib.LETKF_EINVAL


@pytest.mark.parametrize("m", [128, 160, 200, 256])
def test_fused_plan_dual_form_fits_shared_memory(lib, m):
    # the observation-space form at ELT geometry over its whole ensemble range: operands, the
    # halo anomalies' rows staged beside them and the epilogue's rows of P3 within one CTA's
    # 227 KB; its footprint grows with m
    smem, q, n = _plan(**dict(ELT, m=m))
    assert (q, n) == (0, 0)
    assert 0 < smem <= 227 * 1024
    if m > 128:
        assert smem >= _plan(**dict(ELT, m=128))[0]
