"""Closed-loop comparison of the control laws on the paper's 8 m case (Sect. 3, Sect. 3.1-3.2).

16x16 Fried system (241 actuators), three frozen-flow layers, 500 Hz, two-step delay (the slopes
of frame k see the phase of frame k - 1 and the prediction x_hat(k+1|k) corrects frame k + 1), a
deformable mirror with coupling 0.3, and the coherent energy of the fine-grid residual as the
figure of merit (paper_1310_5954_gb300.closed_loop).  The filters run on pseudo-open-loop slopes,
which in this linear loop are the open-loop slopes.  Compared with the Kalman filter on the
Riccati gain (the optimal control law of Sect. 2.1, FP64 on the host) the GPU filters must show
what Figs. 2 and 3 report: the global ETKF's loss of coherent energy shrinks as its ensemble
grows (Fig. 2, at two noise levels), the local ETKF loses less than the global one at the same
ensemble size, and removing the differential pistons lowers the local ETKF's loss (Fig. 3).  The
figures' values are not in the paper, so these are the qualitative pins.  On this system (4x4
subaperture domains, halo 2: 50 local state rows, up to 128 slopes) the local filter needs about
100 members: with 50, even with the pistons removed in the loop, it keeps little coherent energy,
and without that correction it diverges (so does the FP64 oracle, at 20 or 50 members).
"""

import functools

import numpy as np
import pytest
import torch

from oracle import fried, geometry, kf
from paper_1310_5954_gb300 import LETKF, _lib
from paper_1310_5954_gb300 import build as builder
from paper_1310_5954_gb300.closed_loop import DeformableMirror, coherent_energy
from synth import TruthStream, workload

pytestmark = pytest.mark.gpu

N_FRAMES, BURN = 1200, 200


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


@functools.lru_cache(maxsize=None)
def _case(sigma, name="scao-8m", n_frames=N_FRAMES):
    w = workload(name)
    w.sigma = sigma
    g = geometry.make_geometry(w.n_sub, w.obstruction)
    L = w.process_noise_sqrt(g.act_rc)
    Ls = w.stationary_sqrt(g.act_rc)
    ts = TruthStream(w)
    fr = ts.frames(0, n_frames)
    s = fr["slopes"]
    y = np.ascontiguousarray(np.concatenate([s[:, 0][:, g.sub_valid], s[:, 1][:, g.sub_valid]], axis=1))
    dm = DeformableMirror(g.sub_valid, g.act_valid, w.q)
    phi_next = np.stack([ts.phase_fine(k + 1)[dm.pupil] for k in range(BURN, n_frames)]).astype(np.float32)
    # the Kalman filter on the Riccati gain, same AR(1) model and noise
    A = kf.ar1_companion(g.n_act, w.ar1_a)
    C = fried.observation_matrix(g, w.obs_block)
    H = kf.kalman_gain(kf.dare(A, C, kf.process_covariance(L), sigma ** 2 * np.eye(g.p)), C, sigma ** 2 * np.eye(g.p))
    x = np.zeros(g.n)
    kfp = []
    for k in range(n_frames):
        x = kf.kf_predict(x, y[k], A, C, H)
        kfp.append(x[: g.n_act].copy())
    return w, g, L, Ls, y, dm, phi_next, np.array(kfp)


def _ec(case, preds):
    _, _, _, _, _, dm, phi_next, _ = case
    pred = np.asarray(preds, dtype=np.float64)[BURN:]
    if not np.isfinite(pred).all():
        return 0.0                          # a diverged law corrects nothing
    var = []
    for a in range(0, len(pred), 100):
        e = phi_next[a:a + 100].astype(np.float64) - dm.correction(pred[a:a + 100])
        e -= e.mean(axis=1, keepdims=True)
        var.append(np.mean(e * e, axis=1))
    return coherent_energy(np.concatenate(var))


@functools.lru_cache(maxsize=None)
def _run(sigma, path, m, piston="off", name="scao-8m", n_frames=N_FRAMES):
    case = _case(sigma, name, n_frames)
    w, g, L, Ls, y, _, _, _ = case
    prec = "fp32" if path == "global" else "mixed"
    f = LETKF(n_sub=w.n_sub, m=m, ar1_a=w.ar1_a, sigma=sigma, dom_sub=w.dom_sub, halo=w.halo,
              obstruction=w.obstruction, q_sqrt=L, p0_sqrt=Ls, precision=prec, path=path, seed=w.seed,
              obs_block=w.obs_block, piston=piston)
    yd = torch.as_tensor(y, dtype=torch.float32, device="cuda")
    preds = torch.stack([f.step(yd[k]) for k in range(n_frames)]).cpu().numpy()
    status = f.sync()
    f.close()
    ec = _ec(case, preds)
    # a filter that stays on track reports no error; one that diverges (the global ETKF with too
    # few members) may overflow into the Newton-Schulz iteration's sweep limit
    assert status == 0 or (path == "global" and ec < 0.05 * _ec(case, case[7])), (path, m, piston, status)
    return ec


def _loss(sigma, ec, name="scao-8m", n_frames=N_FRAMES):
    case = _case(sigma, name, n_frames)
    ec_kf = _ec(case, case[7])
    return (ec_kf - ec) / ec_kf


@pytest.mark.parametrize("sigma", [0.1, 0.3])
def test_global_etkf_approaches_the_kf_as_members_grow(sigma):
    losses = [_loss(sigma, _run(sigma, "global", m)) for m in (200, 800, 3200)]
    print(f"\nsigma {sigma}: EC(KF) {_ec(_case(sigma), _case(sigma)[7]):.4f}; global ETKF loss at m = 200, 800, "
          f"3200: {', '.join(f'{x:.4f}' for x in losses)}")
    assert losses[0] > losses[1] > losses[2]
    assert losses[2] < 0.25 * losses[0]
    assert losses[2] > -0.01          # the optimal law is not beaten by more than the statistics


def test_local_etkf_beats_the_global_one_and_piston_removal_helps():
    sigma = 0.1
    ec_kf = _ec(_case(sigma), _case(sigma)[7])
    rows = {}
    for m in (100, 200):
        rows[m] = (_loss(sigma, _run(sigma, "fused", m)), _loss(sigma, _run(sigma, "fused", m, "output")),
                   _loss(sigma, _run(sigma, "fused", m, "in_loop")), _loss(sigma, _run(sigma, "global", m)))
    in_loop_50 = _loss(sigma, _run(sigma, "fused", 50, "in_loop"))
    print(f"\nsigma {sigma}: EC(KF) {ec_kf:.4f}; loss vs KF by m: local / local + piston output / "
          f"local + piston in loop / global")
    for m, r in rows.items():
        print(f"  m = {m}: " + " / ".join(f"{x:.4f}" for x in r))
    print(f"  m = 50, local + piston in loop: {in_loop_50:.4f}")
    for m, (loc, out, inl, glob) in rows.items():
        assert loc < glob, m                 # Fig. 3: local better than global at equal m
        assert min(out, inl) < loc, m        # removing the differential pistons lowers the loss
    assert rows[200][0] < rows[100][0]       # and the local loss falls with m
    assert rows[200][2] < rows[100][2] < in_loop_50


def test_16m_local_etkf_with_piston_removal_within_3_percent_at_197_members():
    """Sect. 3.2, Fig. 3 (16 m, 32x32, 877 actuators): the local ETKF does better than the global one
    at the same ensemble size, removing the differential pistons lowers its loss, and with 197
    members the loss against the KF falls under 3 %.  The paper reaches 3 % with a post-processing
    method it does not describe; the least-squares correction of the output alone (the reading used
    here) measured 6.2 %, the same correction applied inside the loop 1.1 % (sigma = 0.1)."""
    sigma, name, n = 0.1, "scao-16m", 1000
    case = _case(sigma, name, n)
    ec_kf = _ec(case, case[7])
    loss = {mode: _loss(sigma, _run(sigma, "fused", 197, mode, name, n), name, n) for mode in ("off", "output", "in_loop")}
    glob = _loss(sigma, _run(sigma, "global", 197, "off", name, n), name, n)
    print(f"\n16 m, sigma {sigma}: EC(KF) {ec_kf:.4f}; loss vs KF at m = 197: local {loss['off']:.4f}, "
          f"local + piston output {loss['output']:.4f}, local + piston in loop {loss['in_loop']:.4f}, global {glob:.4f}")
    assert loss["off"] < glob
    assert loss["output"] < loss["off"] and loss["in_loop"] < loss["off"]
    assert loss["in_loop"] < 0.03
