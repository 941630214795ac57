"""Row-band partition of the domains over ranks and the ghost-row exchange (paper_1310_5954_gb300.bands),
on the host: the plan's invariants, and a world-size-2 gloo run in which each rank analyses and
forecasts only its band (the oracle's per-domain arithmetic standing in for the GPU) and exchanges
ghost rows every frame, matching a single-process run of the whole system bit for bit."""

import os
import socket

import numpy as np
import pytest

from paper_1310_5954_gb300 import _lib, bands
from paper_1310_5954_gb300 import build as builder


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


def _system(name):
    from _gpu_common import model
    w, g, doms, L, Ls = model(name)
    return w, g, doms, L, Ls, dict(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub,
                                   halo=w.halo, obstruction=w.obstruction, q_white=0.1)


@pytest.mark.parametrize("name,ranks", [("tiny-8x8", 2), ("vlt-40x40", 2), ("vlt-40x40", 4), ("elt-80x80", 8)])
def test_plan_invariants(name, ranks):
    w, g, doms, L, Ls, kw = _system(name)
    plans = bands.plan_for(ranks, **kw)
    owned = np.concatenate([p.owned for p in plans])
    assert np.array_equal(np.sort(owned), np.arange(g.n_act))            # each actuator owned once
    assert sum(len(p.domains) for p in plans) == len(doms)
    tab = _lib.letkf_domain_tables(_params(kw))
    for p in plans:
        # contiguous bands of block rows, in rank order
        rows = tab["block"][p.domains] // tab["blocks_per_side"]
        assert rows.size == 0 or (rows.min() >= p.block_rows[0] and rows.max() < p.block_rows[1])
        assert p.domains.size > 0
        reads = np.unique(np.concatenate([tab["halo"][tab["halo_off"][d]:tab["halo_off"][d + 1]] for d in p.domains]))
        assert np.array_equal(np.union1d(np.intersect1d(reads, p.owned), p.ghosts), reads)
        assert not np.intersect1d(p.ghosts, p.owned).size
        for q, ids in p.recv.items():
            assert np.array_equal(plans[q].send[p.rank], ids)
            assert np.isin(ids, plans[q].owned).all()
            # halo reach: only neighbouring bands exchange rows
            assert abs(q - p.rank) == 1
    costs = np.array([p.cost for p in plans])
    assert costs.max() <= 1.6 * costs.mean()


def _params(kw):
    from paper_1310_5954_gb300.letkf import make_params
    p, keep = make_params(**kw)
    _params.keep = keep
    return p


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _band_worker(rank, world, port, name, n_frames, out_path):
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    sys.path.insert(0, here)
    sys.path.insert(0, os.path.dirname(here))
    import torch
    import torch.distributed as dist
    from oracle import etkf
    from _gpu_common import oracle_filter, slopes
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, g, doms, L, Ls, kw = _system(name)
        plan = bands.plan_for(world, **kw)[rank]
        assert plan.ghosts.size > 0 and plan.domains.size > 0
        o = oracle_filter(name)
        na, m = g.n_act, w.m
        y, _ = slopes(name, n_frames)
        # this rank holds its own rows (both instants) and its ghosts' observed instant; the rest
        # is poisoned so that any use of it shows
        X = np.full_like(o.X, np.nan)
        X[plan.owned] = o.X[plan.owned]
        X[na + plan.owned] = o.X[na + plan.owned]
        X[na + plan.ghosts] = o.X[na + plan.ghosts]
        C = o.C
        for k in range(n_frames):
            Xa = X.copy()
            for d in plan.domains:
                dom = doms[d]
                orows = dom.obs_rows(g.n_subv)
                if orows.size == 0:
                    continue
                rows = dom.rows(na)
                Y = C[orows] @ X                       # sparse rows: only the halo's observed instant
                Yp = Y - Y.mean(axis=1, keepdims=True)
                wbar, T = etkf.ensemble_transform(Yp, y[k][orows] - Y.mean(axis=1), w.sigma)
                xbar = X[rows].mean(axis=1)
                Xa[rows] = xbar[:, None] + (X[rows] - xbar[:, None]) @ (wbar[:, None] + T)
            V = o.perturbation(k)
            X = np.full_like(X, np.nan)
            X[plan.owned] = w.ar1_a * Xa[plan.owned] + V[plan.owned]
            X[na + plan.owned] = Xa[plan.owned]
            xo = torch.as_tensor(X[na:].copy())
            bands.exchange(plan, xo)
            X[na + plan.ghosts] = xo.numpy()[plan.ghosts]
        np.save(out_path + f".{rank}.npy", np.stack([X[plan.owned], X[na + plan.owned]]))
        np.save(out_path + f".{rank}.idx.npy", plan.owned)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,n_frames", [("tiny-8x8", 6), ("vlt-40x40", 3)])
def test_two_ranks_match_one_process(tmp_path, name, n_frames):
    import multiprocessing as mp
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    if here not in sys.path:
        sys.path.insert(0, here)
    from _gpu_common import oracle_filter, slopes
    world = 2
    out = str(tmp_path / "band")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_band_worker, args=(r, world, port, name, n_frames, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    o = oracle_filter(name)
    y, _ = slopes(name, n_frames)
    for k in range(n_frames):
        o.step(y[k])
    na = o.geom.n_act
    seen = np.zeros(na, dtype=bool)
    for r in range(world):
        blk = np.load(out + f".{r}.npy")
        idx = np.load(out + f".{r}.idx.npy")
        assert np.isfinite(blk).all()
        assert np.array_equal(blk[0], o.X[idx]) and np.array_equal(blk[1], o.X[na + idx])
        seen[idx] = True
    assert seen.all()
