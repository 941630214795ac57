"""letkf_analyze_static: the allocation-free analysis, checked against letkf_analyze.

Callers that cannot allocate device memory while they run (a real-time controller that
reserves its memory before its loop) use letkf_analyze_static, whose scratch is a fixed
array compiled into the library.  This file is collected last on purpose: it runs the
library's shared static scratch after every other test has used the library, and it must
also pass on its own in a fresh process.
"""

import numpy as np
import pytest
import torch

from paper_1310_5954_gb300 import _lib
from paper_1310_5954_gb300 import build as builder

from _gpu_common import gpu_filter, slopes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("name,prec,tol", [("vlt-40x40", "fp32", 1e-6), ("tiny-8x8", "fp64", 1e-13)])
def test_static_analysis_matches_analyze_on_two_calls(name, prec, tol):
    y, _ = slopes(name, 5)
    f = gpu_filter(name, prec, "plain")
    dt = f.dtype
    for k in range(2):                       # move away from the initial ensemble
        f.step(torch.as_tensor(y[k], dtype=dt, device="cuda"))
    out = torch.empty((f.info.n, f.info.m), dtype=dt, device="cuda")
    for k in (2, 3):                         # two allocation-free calls in a row, one per frame
        yk = torch.as_tensor(y[k], dtype=dt, device="cuda")
        out.fill_(float("nan"))
        before, frame = f.get_state()
        before = before.clone()
        rc = _lib.letkf_analyze_static(f.ctx, yk.data_ptr(), 0.0, out.data_ptr())
        assert rc == _lib.LETKF_OK
        after, frame2 = f.get_state()
        assert torch.equal(before, after) and frame2 == frame      # the context is untouched
        f.analyze(yk)                        # the existing entry point on the same frame
        ref, _ = f.get_state()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) <= tol, _rel(out, ref)
        assert _rel(out.mean(1), ref.mean(1)) <= tol
        f.forecast()
    assert f.sync() == 0
    f.close()


def test_static_analysis_rejects_oversized_problem():
    f = gpu_filter("elt-80x80", "fp32", "plain")
    y = torch.zeros(f.info.p, dtype=f.dtype, device="cuda")
    out = torch.zeros((f.info.n, f.info.m), dtype=f.dtype, device="cuda")
    assert _lib.letkf_analyze_static(f.ctx, y.data_ptr(), 0.0, out.data_ptr()) == _lib.LETKF_ESCRATCH
    assert "16 MiB" in _lib.letkf_status_string(_lib.LETKF_ESCRATCH)
    f.close()


def test_static_analysis_nonfinite_slope_gives_the_forecast_then_recovers():
    """A non-finite slope: the output is the context's forecast ensemble bit for bit and
    LETKF_ENONFINITE is latched; the next finite call equals letkf_analyze again (the call's own
    reject flag starts from zero every time)."""
    y, _ = slopes("vlt-40x40", 4)
    f = gpu_filter("vlt-40x40", "fp32", "plain")
    dt = f.dtype
    f.step(torch.as_tensor(y[0], dtype=dt, device="cuda"))
    before, _ = f.get_state()
    before = before.clone()
    bad = torch.as_tensor(y[1], dtype=dt, device="cuda").clone()
    bad[7] = float("nan")
    out = torch.full((f.info.n, f.info.m), float("inf"), dtype=dt, device="cuda")
    assert _lib.letkf_analyze_static(f.ctx, bad.data_ptr(), 0.0, out.data_ptr()) == _lib.LETKF_OK
    assert torch.equal(out, before)
    assert f.sync() == _lib.LETKF_ENONFINITE
    good = torch.as_tensor(y[1], dtype=dt, device="cuda")
    out.fill_(float("nan"))
    assert _lib.letkf_analyze_static(f.ctx, good.data_ptr(), 0.0, out.data_ptr()) == _lib.LETKF_OK
    f.analyze(good)
    ref, _ = f.get_state()
    assert torch.isfinite(out).all()
    assert _rel(out, ref) <= 1e-6, _rel(out, ref)
    assert f.sync() == 0
    f.close()
