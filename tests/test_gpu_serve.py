"""The serving loop (include/letkf_serve.h) on the GPU.

Batching must not change any result: each system's domains are analysed by the same kernel
code whatever else shares the launch, so every frame's prediction and the final ensemble of a
system served in a mix must equal, bit for bit, those of the same system stepped alone through
letkf_step.  Also: admission by device footprint, a rejected frame inside a mix, the footprint
formula against the allocator, and the real-time replay's records.
"""

import numpy as np
import pytest
import torch

from paper_1310_5954_gb300 import LETKF, LETKFError, Server, _lib, footprint
from paper_1310_5954_gb300 import build as builder

from _gpu_common import model, slopes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


def _kw(name, dense_noise=True, m=None):
    w, g, doms, L, Ls = model(name, m)
    kw = dict(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
              obstruction=w.obstruction, p0_sqrt=Ls, precision="mixed", path="fused", seed=w.seed,
              obs_block=w.obs_block)
    if dense_noise:
        kw["q_sqrt"] = L
    else:
        kw["q_white"] = 0.05
    return kw


# systems of different sizes and ensemble sizes (one of m >= 128, in the dual form); one draws
# white process noise inline
SYSTEMS = [("tiny-8x8", True, None), ("vlt-40x40", True, None), ("tiny-8x8", False, None), ("tiny-8x8", True, 150)]
FRAMES = 12


def _frames(name):
    y, _ = slopes(name, FRAMES)
    return np.ascontiguousarray(y[:FRAMES], dtype=np.float32)


def _alone(name, dense, m, ys, bad_frame=None):
    f = LETKF(**_kw(name, dense, m))
    preds = []
    for k in range(len(ys)):
        y = ys[k].copy()
        if bad_frame == k:
            y[3] = np.nan
        preds.append(f.step(torch.as_tensor(y, device="cuda")).cpu().numpy())
    st = f.sync()
    x, frame = f.get_state()
    x = x.cpu().numpy()
    f.close()
    return np.stack(preds), x, frame, st


def _serve(ys_list, pattern, bad=None):
    srv = Server(slots=2, max_pending=16)
    ids, outs = [], []
    for name, dense, m in SYSTEMS:
        sid = srv.admit(**_kw(name, dense, m))
        ids.append(sid)
        outs.append(srv.set_output(sid, FRAMES))
    sent = [0] * len(SYSTEMS)
    for burst in pattern:          # burst: frames to submit per system before the next pump
        for s, n in enumerate(burst):
            for _ in range(n):
                if sent[s] < FRAMES:
                    y = ys_list[s][sent[s]].copy()
                    if bad is not None and bad == (s, sent[s]):
                        y[3] = np.nan
                    assert srv.submit(ids[s], y) == _lib.LETKF_OK
                    sent[s] += 1
        srv.pump()
    for s in range(len(SYSTEMS)):
        while sent[s] < FRAMES:
            assert srv.submit(ids[s], ys_list[s][sent[s]]) == _lib.LETKF_OK
            sent[s] += 1
    srv.drain()
    states = [srv.state(i) for i in ids]
    info = srv.info()
    recs = srv.records()
    srv.close()
    return outs, [(x.cpu().numpy(), fr) for x, fr in states], info, recs


PATTERN = [(1, 1, 1, 1), (2, 0, 1, 0), (0, 3, 0, 2), (1, 1, 2, 1), (3, 1, 0, 0), (0, 0, 3, 3), (2, 2, 2, 2)]


def test_batched_frames_equal_alone():
    ys_list = [_frames(name) for name, _, _ in SYSTEMS]
    outs, states, info, recs = _serve(ys_list, PATTERN)
    assert info["frames_done"] == FRAMES * len(SYSTEMS)
    assert info["batched_systems"] > info["batches"], "no batch held more than one system"
    assert max(r["batch_systems"] for r in recs) >= 2
    for s, (name, dense, m) in enumerate(SYSTEMS):
        preds, x, frame, st = _alone(name, dense, m, ys_list[s])
        assert st == 0
        assert np.array_equal(outs[s], preds), (name, np.abs(outs[s] - preds).max())
        assert np.array_equal(states[s][0], x) and states[s][1] == frame == FRAMES
    for r in recs:
        assert r["status"] == _lib.LETKF_OK
        assert r["t_arrival_ns"] <= r["t_launch_ns"] <= r["t_done_ns"]
    # frames of one system complete in order
    for s in range(len(SYSTEMS)):
        fr = [r["frame"] for r in recs if r["system"] == s]
        assert fr == list(range(FRAMES))


def test_rejected_frame_inside_a_mix():
    ys_list = [_frames(name) for name, _, _ in SYSTEMS]
    outs, states, info, recs = _serve(ys_list, PATTERN, bad=(1, 4))
    bad = [r for r in recs if r["status"] != _lib.LETKF_OK]
    assert [(r["system"], r["frame"], r["status"]) for r in bad] == [(1, 4, _lib.LETKF_ENONFINITE)]
    for s, (name, dense, m) in enumerate(SYSTEMS):
        preds, x, frame, st = _alone(name, dense, m, ys_list[s], bad_frame=4 if s == 1 else None)
        assert st == (_lib.LETKF_ENONFINITE if s == 1 else 0)
        assert np.array_equal(outs[s], preds)
        assert np.array_equal(states[s][0], x)


def test_admission_by_footprint():
    ka, kb = _kw("tiny-8x8"), _kw("vlt-40x40")
    fa, fb = footprint(**ka), footprint(**kb)
    assert fb > 1 << 20 > fa
    # room for one tiny and one vlt system (plus the server's per-system y and x_hat buffers)
    srv = Server(hbm_budget=fa + fb + (64 << 10), slots=1)
    a = srv.admit(**ka)
    b = srv.admit(**kb)
    with pytest.raises(LETKFError) as e:
        srv.admit(**kb)
    assert e.value.status == _lib.LETKF_EBUSY
    assert srv.info()["hbm_used"] <= srv.info()["hbm_budget"] and srv.info()["systems"] == 2
    srv.release(b)
    c = srv.admit(**kb)
    assert srv.info()["systems"] == 2 and c != a
    srv.close()


@pytest.mark.parametrize("cfg", [
    ("tiny-8x8", dict(precision="fp64", path="plain")),
    ("vlt-40x40", dict(precision="fp32", path="plain")),
    ("vlt-40x40", dict(precision="mixed", path="fused")),
    ("tiny-8x8", dict(precision="fp32", path="fused", q_sqrt=None, q_white=0.1)),
    ("tiny-8x8", dict(precision="mixed", path="fused", m=150)),
])
def test_footprint_equals_allocated_bytes(cfg):
    name, over = cfg
    kw = _kw(name)
    kw.update(over)
    f = LETKF(**kw)
    assert f.info.device_bytes == footprint(**kw)
    f.close()


def test_replay_runs_a_trace_in_real_time():
    ys_list = [_frames(name) for name, _, _ in SYSTEMS]
    srv = Server(slots=2, max_pending=32)
    ids = [srv.admit(**_kw(name, dense, m)) for name, dense, m in SYSTEMS]
    sys_ids, t_ns, ys = [], [], []
    for k in range(FRAMES):
        for s in range(len(SYSTEMS)):
            sys_ids.append(ids[s])
            t_ns.append(k * 1_000_000 + s * 250_000)     # 1 kHz per system, staggered
            ys.append(ys_list[s][k])
    refused = srv.replay(sys_ids, t_ns, ys)
    assert refused == 0
    recs = srv.records()
    assert len(recs) == FRAMES * len(SYSTEMS)
    lat = np.array([r["t_done_ns"] - r["t_arrival_ns"] for r in recs])
    assert (lat > 0).all() and np.median(lat) < 50_000_000
    srv.close()


def _overlapping_pairs(recs):
    """Pairs of batches in different stream slots whose device-clock intervals intersect."""
    batches = {}
    for r in recs:
        batches[(r["slot"], r["t_dev_start_ns"], r["t_dev_end_ns"])] = True
    b = sorted(batches)
    return [(x, y) for i, x in enumerate(b) for y in b[i + 1:]
            if x[0] != y[0] and max(x[1], y[1]) < min(x[2], y[2])]


def test_admission_while_frames_are_in_flight_and_overlap_on_the_device():
    """Continuous batching: a system's frame is launched into the second stream slot while another
    system's batch is still on the GPU, and a third system is admitted while a batch is outstanding
    (no drain).  The two slots' batches overlap on the device clock (CUDA events), and every
    system's predictions and final ensemble equal those of the same system stepped alone, bit for
    bit."""
    systems = [("elt-80x80", True, None), ("tiny-8x8", True, None), ("tiny-8x8", False, None)]
    ys = [_frames(name) for name, _, _ in systems]
    srv = Server(slots=2, max_pending=16)
    ids = [srv.admit(**_kw(*systems[0])), srv.admit(**_kw(*systems[1]))]
    outs = [srv.set_output(i, FRAMES) for i in ids]
    in_flight_at_admission = -1
    sent_c = 0
    for k in range(FRAMES):
        assert srv.submit(ids[0], ys[0][k]) == _lib.LETKF_OK
        srv.pump()                                   # the large system's frame k on one slot
        assert srv.submit(ids[1], ys[1][k]) == _lib.LETKF_OK
        srv.pump()                                   # the small one's, while that batch runs
        if k == 3:
            in_flight_at_admission = srv.info()["frames_in_flight"]
            ids.append(srv.admit(**_kw(*systems[2])))
            outs.append(srv.set_output(ids[2], FRAMES))
        if len(ids) == 3:
            assert srv.submit(ids[2], ys[2][sent_c]) == _lib.LETKF_OK
            sent_c += 1
            srv.pump()
    while sent_c < FRAMES:
        assert srv.submit(ids[2], ys[2][sent_c]) == _lib.LETKF_OK
        sent_c += 1
    srv.drain()
    states = [srv.state(i) for i in ids]
    recs = srv.records()
    srv.close()
    assert in_flight_at_admission >= 1, "nothing was in flight when the third system was admitted"
    assert all(r["status"] == _lib.LETKF_OK for r in recs) and len(recs) == 3 * FRAMES
    for r in recs:
        assert 0 <= r["t_dev_start_ns"] < r["t_dev_end_ns"]
    pairs = _overlapping_pairs(recs)
    assert pairs, "no two batches of different slots overlapped on the device"
    for s, (name, dense, m) in enumerate(systems):
        preds, x, frame, st = _alone(name, dense, m, ys[s])
        assert st == 0
        assert np.array_equal(outs[s], preds), (name, np.abs(outs[s] - preds).max())
        assert np.array_equal(states[s][0].cpu().numpy(), x) and states[s][1] == frame == FRAMES
        assert [r["frame"] for r in recs if r["system"] == ids[s]] == list(range(FRAMES))
