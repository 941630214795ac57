"""Fault handling on the GPU, injected from the host (nothing faults, traps or hangs the device):

* skipped domains (letkf_set_domain_mask): the analysis equals the FP64 oracle's over the other
  domains, and the skipped domains' actuators keep their forecast bit for bit; restoring the mask
  gives back the unmasked filter bit for bit;
* the serving loop: frames beyond a system's queue depth are refused (LETKF_EBUSY) and the rest
  served; a system released while others run leaves their results unchanged (bit for bit against
  each stepped alone).
"""

import numpy as np
import pytest
import torch

from oracle import etkf
from paper_1310_5954_gb300 import LETKF, Server, _lib
from paper_1310_5954_gb300 import build as builder

from _gpu_common import gpu_filter, model, oracle_filter, rel, slopes

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-4, "mixed": 5e-3, "fp64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


def _t(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.mark.parametrize("name,prec,path", [("tiny-8x8", "fp64", "plain"), ("vlt-40x40", "fp32", "plain"),
                                            ("vlt-40x40", "fp32", "fused"), ("vlt-40x40", "mixed", "fused"),
                                            ("elt-80x80", "mixed", "fused")])
def test_skipped_domains_keep_their_forecast(name, prec, path):
    w, g, doms, L, Ls = model(name)
    y, _ = slopes(name, 2)
    f = gpu_filter(name, prec, path)
    o = oracle_filter(name)
    rng = np.random.default_rng(41)
    active = rng.random(len(doms)) > 0.3
    active[0] = False
    f.set_domain_mask(active)
    dt = f.dtype
    xf = o.X.astype(np.float32).astype(np.float64) if dt == torch.float32 else o.X.copy()
    f.set_state(_t(xf, dt), 0)
    f.analyze(_t(y[0], dt))
    xa, _ = f.get_state()
    xa = xa.cpu().numpy().astype(np.float64)
    yk = y[0].astype(np.float32).astype(np.float64) if dt == torch.float32 else y[0]
    ref = etkf.letkf_analysis(xf, yk, o.C, w.sigma, [d for d, a in zip(doms, active) if a], g.n_act, g.n_subv)
    assert rel(xa.mean(axis=1), ref.mean(axis=1)) < TOL[prec]
    skipped = np.concatenate([d.rows(g.n_act) for d, a in zip(doms, active) if not a])
    assert np.array_equal(xa[skipped], xf[skipped].astype(np.float32 if dt == torch.float32 else np.float64))
    assert f.sync() == 0
    f.close()


@pytest.mark.parametrize("prec,path", [("fp32", "plain"), ("mixed", "fused")])
def test_mask_restored_is_bitwise(prec, path):
    y, _ = slopes("vlt-40x40", 3)
    a = gpu_filter("vlt-40x40", prec, path)
    b = gpu_filter("vlt-40x40", prec, path)
    mask = np.ones(a.info.n_domains, dtype=bool)
    mask[::3] = False
    b.set_domain_mask(mask)
    b.set_domain_mask(None)
    for k in range(3):
        pa = a.step(_t(y[k])).cpu().numpy()
        pb = b.step(_t(y[k])).cpu().numpy()
        assert np.array_equal(pa, pb)
    assert a.sync() == 0 and b.sync() == 0
    a.close()
    b.close()


def _kw(name):
    w, g, doms, L, Ls = model(name)
    return dict(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
                obstruction=w.obstruction, p0_sqrt=Ls, q_sqrt=L, precision="mixed", path="fused", seed=w.seed,
                obs_block=w.obs_block)


def _alone(name, ys):
    f = LETKF(**_kw(name))
    out = np.stack([f.step(torch.as_tensor(y, device="cuda")).cpu().numpy() for y in ys])
    assert f.sync() == 0
    f.close()
    return out


def test_queue_overflow_is_refused():
    depth = 4
    ys = np.ascontiguousarray(slopes("tiny-8x8", 10)[0][:10], dtype=np.float32)
    srv = Server(slots=1, max_pending=depth)
    sid = srv.admit(**_kw("tiny-8x8"))
    out = srv.set_output(sid, 10)
    codes = [srv.submit(sid, ys[k]) for k in range(10)]       # nothing pumped: the queue fills
    assert codes[:depth] == [_lib.LETKF_OK] * depth
    assert all(c == _lib.LETKF_EBUSY for c in codes[depth:])
    srv.drain()
    info = srv.info()
    srv.close()
    assert info["frames_done"] == depth
    assert np.array_equal(out[:depth], _alone("tiny-8x8", ys[:depth]))


def test_release_while_others_run():
    n = 6
    ya = np.ascontiguousarray(slopes("tiny-8x8", n)[0][:n], dtype=np.float32)
    yb = np.ascontiguousarray(slopes("vlt-40x40", n)[0][:n], dtype=np.float32)
    srv = Server(slots=2, max_pending=16)
    a = srv.admit(**_kw("tiny-8x8"))
    b = srv.admit(**_kw("vlt-40x40"))
    out_a = srv.set_output(a, n)
    srv.set_output(b, n)
    for k in range(3):
        srv.submit(a, ya[k])
        srv.submit(b, yb[k])
        srv.pump()
    srv.drain()
    srv.release(b)                     # the client of b goes away between frames
    for k in range(3, n):
        assert srv.submit(a, ya[k]) == _lib.LETKF_OK
        srv.pump()
    srv.drain()
    srv.close()
    assert np.array_equal(out_a, _alone("tiny-8x8", ya))
