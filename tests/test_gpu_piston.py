"""Differential-piston removal on the GPU (letkf_piston; Sect. 3.1, Sect. 5) against the FP64 oracle
(oracle.piston), through the C ABI.

* The correction itself: two contexts stepped on the same frames, one without correction and one
  correcting the output only (the output mode leaves the ensemble untouched, so both see the same
  raw prediction x_hat); the difference of their outputs must be P delta with delta the oracle's
  least-squares pistons of that x_hat and y, within the a-priori rounding bound of the
  computation in the state's precision.
* The in-loop mode, free-running, against the oracle's in-loop filter, within the free-running
  bounds of each precision.
* A rejected frame passes through uncorrected, and systems with and without correction served in
  one mix give, bit for bit, what each gives alone.
"""

import numpy as np
import pytest
import torch

from oracle import piston
from oracle.fried import fried_matrix
from paper_1310_5954_gb300 import LETKF, Server, _lib
from paper_1310_5954_gb300 import build as builder

from _gpu_common import gpu_filter, model, oracle_filter, rel, slopes

pytestmark = pytest.mark.gpu

UNIT = {torch.float32: 2.0 ** -24, torch.float64: 2.0 ** -53}


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


def _bound(name, K, y, x, g, u):
    """First-order bound on |delta_gpu - delta| for delta = K g, g_l = sum over the domain's E
    boundary entries of (y - D x) weighted by exact coefficients (|w| <= 1): each residual carries
    at most 4 roundings of operands bounded by |y| + 2|x|; K is stored rounded and the product
    sums n_dom terms."""
    w, gm, doms, _, _ = model(name)
    D = fried_matrix(gm)
    owner = np.argmax(piston.ownership(gm, doms), axis=1)
    E = np.zeros(len(doms), dtype=int)
    for k in range(gm.n_subv):
        own = set(owner[np.nonzero(D[k])[0]])
        if len(own) > 1:
            for o in own:
                E[o] += 1
    kinf = np.abs(K).sum(axis=1).max()
    tol_g = 4 * u * E.max() * (np.abs(y).max() + 2 * np.abs(x).max())
    return kinf * (tol_g + u * len(doms) * np.abs(g).max()) + 1e-300


@pytest.mark.parametrize("name,prec,path,frames", [
    ("tiny-8x8", "fp64", "plain", 3), ("tiny-8x8", "fp32", "plain", 3), ("tiny-8x8", "fp32", "fused", 3),
    ("tiny-8x8", "mixed", "fused", 3), ("vlt-40x40", "fp32", "plain", 2), ("vlt-40x40", "mixed", "fused", 2),
    ("elt-80x80", "mixed", "fused", 1)])
def test_correction_matches_oracle(name, prec, path, frames):
    w, g, doms, _, _ = model(name)
    y, _ = slopes(name, frames)
    raw = gpu_filter(name, prec, path)
    cor = gpu_filter(name, prec, path, piston="output")
    from paper_1310_5954_gb300.letkf import make_params
    p, keep = make_params(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
                          obstruction=w.obstruction, piston="output")
    K = _lib.letkf_piston_operator(p)
    D = fried_matrix(g)
    P = piston.ownership(g, doms)
    u = UNIT[raw.dtype]
    for k in range(frames):
        yk = torch.as_tensor(y[k], dtype=raw.dtype, device="cuda")
        xr = raw.step(yk).cpu().numpy().astype(np.float64)
        xc = cor.step(yk).cpu().numpy().astype(np.float64)
        yk64 = yk.cpu().numpy().astype(np.float64)
        delta = piston.differential_pistons(xr, yk64, g, doms)
        gsum = (D @ P).T @ (yk64 - D @ xr)
        tol = _bound(name, K, yk64, xr, gsum, u)
        err = np.abs((xc - xr) - P @ delta).max()
        assert err <= tol, (k, err, tol)
        assert np.abs(delta).max() > 100 * tol      # the correction is not vacuous
    xa, _ = raw.get_state()
    xb, _ = cor.get_state()
    assert torch.equal(xa, xb)                        # output mode leaves the ensemble alone
    assert raw.sync() == 0 and cor.sync() == 0
    raw.close()
    cor.close()


@pytest.mark.parametrize("name,prec,path,frames,tol", [
    ("tiny-8x8", "fp64", "plain", 20, 1e-9), ("tiny-8x8", "fp32", "plain", 20, 2e-4),
    ("tiny-8x8", "fp32", "fused", 20, 2e-4), ("tiny-8x8", "mixed", "fused", 20, 2e-2),
    ("vlt-40x40", "mixed", "fused", 8, 2e-2)])
def test_in_loop_free_running_matches_oracle(name, prec, path, frames, tol):
    y, _ = slopes(name, frames)
    f = gpu_filter(name, prec, path, piston="in_loop")
    o = oracle_filter(name, piston="in_loop")
    worst = 0.0
    for k in range(frames):
        yk = torch.as_tensor(y[k], dtype=f.dtype, device="cuda")
        xp = f.step(yk).cpu().numpy().astype(np.float64)
        xo = o.step(yk.cpu().numpy().astype(np.float64))
        worst = max(worst, rel(xp, xo))
    assert worst < tol, worst
    assert f.sync() == 0
    f.close()


@pytest.mark.parametrize("prec,path", [("fp32", "plain"), ("mixed", "fused")])
def test_rejected_frame_passes_through(prec, path):
    y, _ = slopes("tiny-8x8", 3)
    ys = [y[0].copy(), y[1].copy(), y[2].copy()]
    ys[1][5] = np.nan
    f0 = gpu_filter("tiny-8x8", prec, path)
    f1 = gpu_filter("tiny-8x8", prec, path, piston="in_loop")
    x0 = f0.step(torch.as_tensor(ys[0], dtype=f0.dtype, device="cuda"))
    f1.step(torch.as_tensor(ys[0], dtype=f1.dtype, device="cuda"))
    s1, _ = f1.get_state()
    # the rejected frame: the prediction is the mean of the unchanged first instant, uncorrected,
    # and the ensemble is left as it was
    xb0 = f0.step(torch.as_tensor(ys[1], dtype=f0.dtype, device="cuda")).cpu().numpy()
    xb1 = f1.step(torch.as_tensor(ys[1], dtype=f1.dtype, device="cuda")).cpu().numpy()
    s1b, _ = f1.get_state()
    assert torch.equal(s1, s1b)
    first = s1[: f1.info.n_act].double().mean(dim=1).cpu().numpy()
    np.testing.assert_allclose(xb1, first, rtol=0, atol=1e-5 * max(1.0, np.abs(first).max()))
    assert np.isfinite(xb0).all() and np.isfinite(xb1).all()
    assert f0.sync() == _lib.LETKF_ENONFINITE and f1.sync() == _lib.LETKF_ENONFINITE
    f0.close()
    f1.close()


def _kw(name, m, mode):
    w, g, doms, L, Ls = model(name, m)
    return dict(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
                obstruction=w.obstruction, p0_sqrt=Ls, q_sqrt=L, precision="mixed", path="fused", seed=w.seed,
                obs_block=w.obs_block, piston=mode)


def test_served_mix_equals_alone():
    systems = [("tiny-8x8", None, "in_loop"), ("vlt-40x40", None, "output"), ("tiny-8x8", 150, "in_loop"),
               ("vlt-40x40", None, "off")]
    n = 8
    ys = [np.ascontiguousarray(slopes(nm, n)[0][:n], dtype=np.float32) for nm, _, _ in systems]
    srv = Server(slots=2, max_pending=16)
    ids = [srv.admit(**_kw(nm, m, mode)) for nm, m, mode in systems]
    outs = [srv.set_output(i, n) for i in ids]
    for k in range(n):
        for s, i in enumerate(ids):
            assert srv.submit(i, ys[s][k]) == _lib.LETKF_OK
        if k % 3 != 2:
            srv.pump()
    srv.drain()
    states = [srv.state(i)[0].cpu().numpy() for i in ids]
    srv.close()
    for s, (nm, m, mode) in enumerate(systems):
        f = LETKF(**_kw(nm, m, mode))
        preds = np.stack([f.step(torch.as_tensor(ys[s][k], device="cuda")).cpu().numpy() for k in range(n)])
        x, _ = f.get_state()
        assert f.sync() == 0
        f.close()
        assert np.array_equal(outs[s], preds), (nm, mode, np.abs(outs[s] - preds).max())
        assert np.array_equal(states[s], x.cpu().numpy())
