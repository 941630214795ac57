"""The C ABI library loads and exports every declared entry point (no GPU needed)."""

import ctypes
import os

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
    for s in range(-8, 1):
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
                                 dict(precision=_lib.LETKF_PREC_FP64, m=200), dict(dom_sub=12, halo=2)])
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
