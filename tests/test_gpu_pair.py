"""Two local ETKFs run together with two domain partitions (Sect. 5), on the GPU.

letkf_step_pair analyses both filters' domains in one fused launch and returns the mean of their
predictions.  Checked against two FP64 oracle filters (the second with its block grid shifted by
half a block and its own seed) averaged the same way, and against the two filters stepped alone
(batching changes no bit)."""

import numpy as np
import pytest
import torch

from oracle import etkf, geometry
from paper_1310_5954_gb300 import LETKF, LETKFPair, _lib
from paper_1310_5954_gb300 import build as builder

from _gpu_common import model, rel, slopes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


def _kw(name, prec, m=None):
    w, g, doms, L, Ls = model(name, m)
    return dict(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
                obstruction=w.obstruction, q_sqrt=L, p0_sqrt=Ls, precision=prec, seed=w.seed,
                obs_block=w.obs_block)


def _oracle_pair(name, m=None):
    w, g, doms, L, Ls = model(name, m)
    doms_b = geometry.make_domains(g, w.dom_sub, w.halo, offset=w.dom_sub // 2)
    mk = lambda d, seed: etkf.OracleFilter(g, d, w.m, w.ar1_a, w.sigma, seed=seed, L=L, L_stat=Ls,
                                           obs_block=w.obs_block)
    return mk(doms, w.seed), mk(doms_b, w.seed + 1)


# free-running bounds: tiny FP32 as a single filter (2e-4, its domains on the CUDA cores); the
# 40x40 system's cold-start frames (cond ~3e3) carry the tensor-core Newton-Schulz rounding
# 4 sqrt(kappa) 2^-16 ~ 3.4e-3 into the predictions (FP32 5e-3); mixed 2e-2 as for one filter
@pytest.mark.parametrize("name,prec,n,tol", [("tiny-8x8", "fp32", 20, 2e-4), ("tiny-8x8", "mixed", 20, 2e-2),
                                             ("vlt-40x40", "mixed", 12, 2e-2), ("vlt-40x40", "fp32", 12, 5e-3)])
def test_pair_matches_two_averaged_oracle_filters(name, prec, n, tol):
    y, _ = slopes(name, n)
    p = LETKFPair(**_kw(name, prec))
    oa, ob = _oracle_pair(name)
    worst = 0.0
    for k in range(n):
        xp = p.step(torch.as_tensor(y[k], dtype=torch.float32, device="cuda")).cpu().numpy().astype(np.float64)
        yk = y[k].astype(np.float32).astype(np.float64)
        xo = 0.5 * (oa.step(yk) + ob.step(yk))
        worst = max(worst, rel(xp, xo))
    assert worst < tol, worst
    assert p.sync() == 0
    p.close()


def test_pair_equals_its_two_filters_stepped_alone():
    """Batching the two filters changes no bit: each keeps the state it has when stepped alone, and
    the pair's output is the mean of the two predictions rounded once."""
    name, n = "vlt-40x40", 6
    y, _ = slopes(name, n)
    kw = _kw(name, "mixed")
    p = LETKFPair(**kw)
    a = LETKF(**dict(kw, path="fused"))
    b = LETKF(**dict(kw, path="fused", dom_offset=kw["dom_sub"] // 2, seed=kw["seed"] + 1))
    for k in range(n):
        yk = torch.as_tensor(y[k], dtype=torch.float32, device="cuda")
        xp = p.step(yk)
        pa, pb = a.step(yk), b.step(yk)
        assert torch.equal(xp, 0.5 * (pa + pb)), k
    for mine, alone in ((p.a, a), (p.b, b)):
        x1, f1 = mine.get_state()
        x2, f2 = alone.get_state()
        assert torch.equal(x1, x2) and f1 == f2 == n
    assert p.sync() == 0 and a.sync() == 0 and b.sync() == 0
    for f in (p, a, b):
        f.close()


def test_pair_rejects_a_nonfinite_frame_in_both_filters():
    name = "tiny-8x8"
    y, _ = slopes(name, 4)
    p = LETKFPair(**_kw(name, "fp32"))
    p.step(torch.as_tensor(y[0], dtype=torch.float32, device="cuda"))
    xa0, xb0 = p.a.get_state()[0].clone(), p.b.get_state()[0].clone()
    bad = torch.as_tensor(y[1], dtype=torch.float32, device="cuda").clone()
    bad[5] = float("inf")
    out = p.step(bad)
    assert p.a.sync() == _lib.LETKF_ENONFINITE and p.b.sync() == _lib.LETKF_ENONFINITE
    assert torch.equal(p.a.get_state()[0], xa0) and torch.equal(p.b.get_state()[0], xb0)
    na = p.info.n_act
    # member means summed in another order than torch's: FP32 rounding of values up to ~20
    assert torch.allclose(out, 0.5 * (xa0[:na].mean(1) + xb0[:na].mean(1)), rtol=1e-5, atol=1e-5)
    p.step(torch.as_tensor(y[2], dtype=torch.float32, device="cuda"))
    assert p.sync() == 0
    p.close()


def test_pair_argument_checks():
    kw = _kw("tiny-8x8", "fp32")
    a = LETKF(**dict(kw, path="fused"))
    pl = LETKF(**dict(kw, path="plain"))
    y = torch.zeros(a.info.p, dtype=torch.float32, device="cuda")
    out = torch.zeros(a.info.n_act, dtype=torch.float32, device="cuda")
    lib = _lib.load()
    assert lib.letkf_step_pair(a.ctx, a.ctx, y.data_ptr(), 0.0, out.data_ptr()) == _lib.LETKF_EINVAL   # same context
    assert lib.letkf_step_pair(a.ctx, pl.ctx, y.data_ptr(), 0.0, out.data_ptr()) == _lib.LETKF_EINVAL  # plain path
    a.close()
    pl.close()
