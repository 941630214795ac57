"""The transform itself, per domain, against the FP64 oracle: the mean weights
w_bar = [(m-1)I + G]^-1 Y'^T R^-1 d and T = sqrt(m-1) [(m-1)I + G]^(-1/2) of Sect. 2.2-2.3 as the
fused kernel computed them (letkf_set_capture), at the cold start (frames 0 and 1, where
cond((m-1)I + G) reaches ~1e4) and in steady state, for every form of the analysis (m x m and
observation-space, tensor cores and CUDA cores) and both precisions.

Bounds, from the arithmetic (kappa = cond((m-1)I + G) of the domain, from the oracle):
* T, Gram accurate to FP32 (FP32 precision; mixed precision with the conditioning bound s > 8,
  whose Gram is split; the CUDA-core forms): relative Frobenius error <= 4 sqrt(kappa) 2^-16 + 3e-5.
  The Newton-Schulz iterates hold entries from 1 to sqrt(kappa) and every split-BF16 product
  rounds at 2^-16 relative to its largest entries.
* T, Gram from single-BF16 operands (mixed precision, s <= 8): <= 2e-3.  Rounding the slopes to
  BF16 (2^-9) moves G/(m-1) by at most ~2^-8 (s - 1) in norm, and the iteration stops once the
  update lands under that rounding.
* w_bar (refined against the exact FP32 slopes): relative error <= 4 kappa 2^-24 + 2e-5.
The conditioning bound s = 1 + ||G||_F/(m-1) the kernel reports must match the oracle's to 1 %.
"""

import functools

import numpy as np
import pytest
import torch

from oracle import etkf
from paper_1310_5954_gb300 import _lib
from paper_1310_5954_gb300 import build as builder
from paper_1310_5954_gb300.letkf import make_params

from _gpu_common import gpu_filter, model, oracle_filter, rel, slopes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


STEADY = {"tiny-8x8": 30, "vlt-40x40": 20, "elt-80x80": 12}


@functools.lru_cache(maxsize=None)
def _states(name, m):
    """Forecast ensembles of the oracle at frames 0, 1 and a steady-state frame (FP32-rounded, as
    both sides see them), with the frame indices."""
    n = STEADY[name] if m is None else 12
    y, _ = slopes(name, n + 1)
    o = oracle_filter(name, m=m)
    out = []
    for k in range(n + 1):
        if k in (0, 1, n):
            out.append((k, o.X.astype(np.float32).astype(np.float64)))
        if k < n:
            o.step(y[k].astype(np.float32).astype(np.float64))
    return tuple(out), y


def _library_index(w, m):
    """Library domain number of each oracle domain (by block index)."""
    p, keep = make_params(n_sub=w.n_sub, m=m or w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub,
                          halo=w.halo, obstruction=w.obstruction, q_white=0.1, precision="mixed", path="fused")
    tab = _lib.letkf_domain_tables(p)
    nb = tab["blocks_per_side"]
    return {int(b): k for k, b in enumerate(tab["block"])}, nb


def _picks(g, doms):
    """An interior domain (most slopes), an edge domain (fewest), and the obstruction-rim domain
    (partly observed, block centre nearest the pupil centre)."""
    pl = np.array([d.obs_sub.size for d in doms])
    obs = np.flatnonzero(pl > 0)
    centre = (g.n_sub - 1) / 2.0
    b = np.array([[d.I, d.J] for d in doms], dtype=float)
    dist = np.hypot((b[:, 0] + 0.5) * 4 - 0.5 - centre, (b[:, 1] + 0.5) * 4 - 0.5 - centre)
    partial = obs[pl[obs] < pl.max()]
    picks = {int(obs[np.argmax(pl[obs])]), int(obs[np.argmin(pl[obs])])}
    if partial.size:
        picks.add(int(partial[np.argmin(dist[partial])]))
    return sorted(picks)


CASES = [("tiny-8x8", None, 0), ("tiny-8x8", None, -1), ("vlt-40x40", None, 0), ("vlt-40x40", None, -1),
         ("vlt-40x40", None, 64), ("elt-80x80", None, 0), ("vlt-40x40", 200, 0), ("tiny-8x8", 150, 0)]


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
@pytest.mark.parametrize("name,m,simt", CASES)
def test_transform_and_mean_weights_per_domain(name, m, simt, prec):
    w, g, doms, L, Ls = model(name, m)
    states, y = _states(name, m)
    lib_of, nb = _library_index(w, m)
    f = gpu_filter(name, prec, "fused", m=m, simt_q_max=simt)
    mm = f.info.m
    C = etkf.sparse_observation(g, w.obs_block)
    forms, worst = set(), []
    for k, xf in states:
        Y = C @ xf
        ybar = Y.mean(1)
        Yp = Y - ybar[:, None]
        yk = y[k].astype(np.float32).astype(np.float64)
        for di in _picks(g, doms):
            d = doms[di]
            orows = d.obs_rows(g.n_subv)
            w_o, T_o = etkf.ensemble_transform(Yp[orows], yk[orows] - ybar[orows], w.sigma)
            G = Yp[orows].T @ Yp[orows] / w.sigma ** 2
            lam = np.linalg.eigvalsh((mm - 1) * np.eye(mm) + G)
            kappa = lam[-1] / lam[0]
            s_o = 1.0 + np.linalg.norm(G) / (mm - 1)
            f.capture_transform(lib_of[d.I * nb + d.J])
            f.set_state(_t(xf), k)
            f.analyze(_t(y[k]))
            c = f.captured()
            f.capture_transform(None)
            forms.add(c["form"])
            tag = f"{name} m={mm} {prec} simt={simt} frame {k} domain {di} ({c['form']}, kappa {kappa:.3g})"
            assert abs(c["s"] / s_o - 1) < 1e-2, (tag, c["s"], s_o)
            single_bf16 = prec == "mixed" and c["form"].endswith("tensor") and c["s"] <= 8.0
            tol_T = 2e-3 if single_bf16 else 4 * np.sqrt(kappa) * 2.0 ** -16 + 3e-5
            tol_w = 4 * kappa * 2.0 ** -24 + 2e-5
            eT, ew = rel(c["T"], T_o), rel(c["wbar"], w_o)
            worst.append((eT / tol_T, ew / tol_w, tag, eT, ew))
            assert eT < tol_T, (tag, "T", eT, tol_T)
            assert ew < tol_w, (tag, "w_bar", ew, tol_w)
    assert f.sync() == 0
    f.close()
    # every form this configuration is meant to take was exercised
    want = {("tiny-8x8", 0): {"mm/simt"}, ("tiny-8x8", -1): {"mm/tensor"},
            ("vlt-40x40", 0): {"mm/tensor", "dual/simt"}, ("vlt-40x40", -1): {"mm/tensor"},
            ("vlt-40x40", 64): {"mm/simt", "dual/simt"}, ("elt-80x80", 0): {"mm/tensor", "dual/simt"}}
    assert forms == (want[(name, simt)] if m is None else {"dual/tensor"}), forms


def test_capture_argument_checks():
    f = gpu_filter("tiny-8x8", "fp32", "fused")
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert _lib.load().letkf_set_capture(f.ctx, 0, buf.data_ptr(), 16) == _lib.LETKF_EINVAL     # too small
    assert _lib.load().letkf_set_capture(f.ctx, f.info.n_domains, buf.data_ptr(), 1 << 20) == _lib.LETKF_EINVAL
    assert _lib.load().letkf_set_capture(f.ctx, -1, None, 0) == _lib.LETKF_OK                    # off
    f.close()
    p = gpu_filter("tiny-8x8", "fp32", "plain")
    assert _lib.load().letkf_set_capture(p.ctx, 0, buf.data_ptr(), 1 << 20) == _lib.LETKF_ESTATE
    p.close()
