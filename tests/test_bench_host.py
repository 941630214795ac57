"""Host legs of bench.py at the frame counts a short run uses (--steps 20 --warmup 5).

The benchmark generates W + K + 1 truth frames: W + K filter steps, plus the truth of the frame
after the last one, which scores the last prediction.  The oracle's timed sample must therefore
stop at W + K predictions even when its time budget would let it run every slope frame.
"""

import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


def test_residual_rms_refuses_more_predictions_than_truth():
    bench = _bench()
    phi = np.zeros((6, 4))
    bench.residual_rms(np.zeros((5, 4)), phi, 0)
    with pytest.raises(ValueError):
        bench.residual_rms(np.zeros((6, 4)), phi, 0)


@pytest.mark.parametrize("warmup,steps", [(5, 20), (3, 2)])
def test_cpu_baseline_scores_every_frame_of_a_short_run(warmup, steps):
    """The oracle finishes every frame inside its budget: it stops at W + K predictions and the
    residual of its sample (and of the same number of GPU-side predictions) is computable."""
    from oracle import geometry
    from synth import workload
    bench = _bench()
    w = workload("tiny-8x8")
    g = geometry.make_geometry(w.n_sub, w.obstruction)
    L = w.process_noise_sqrt(g.act_rc)
    Ls = w.stationary_sqrt(g.act_rc)
    _, y, phi = bench.workload_inputs("tiny-8x8", warmup + steps, g.sub_valid, g.act_valid)
    assert len(y) == len(phi) == warmup + steps + 1
    fps, preds, nfr, _ = bench.cpu_baseline("tiny-8x8", y, 600.0, L, Ls)
    assert nfr == len(preds) == warmup + steps and fps > 0
    burn = min(50, (warmup + steps) // 4)
    nb = min(burn, max(nfr - 2, 0))
    r = bench.residual_rms(preds, phi, nb)
    assert np.isfinite(r) and r > 0
    # the in-loop piston oracle leg takes the same path
    _, preds_pl, nfr_pl, _ = bench.cpu_baseline("tiny-8x8", y, 600.0, L, Ls, piston="in_loop")
    assert nfr_pl == warmup + steps
    assert np.isfinite(bench.residual_rms(preds_pl, phi, nb))


def test_traffic_record_matches_kernel_source_workload_and_precision(tmp_path, monkeypatch):
    # roofline.traffic comes from the committed ncu record only for the same kernel source (its
    # hash), workload and precision; anything else reports no traffic rather than a stale figure
    import hashlib
    import json
    bench = _bench()
    src = tmp_path / "paper_1310_5954_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_text("kernel source")
    sha = hashlib.sha256(b"kernel source").hexdigest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"source": "k.cu", "source_sha256": sha, "dram_bytes_per_launch": 1234}
    (prof / "traffic.json").write_text(json.dumps({"fk:wl:mixed": rec}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("fk", "wl", "mixed") == 1234
    assert bench._traffic("fk", "wl", "fp32") is None
    assert bench._traffic("fk", "other", "mixed") is None
    (src / "k.cu").write_text("kernel source, changed")
    assert bench._traffic("fk", "wl", "mixed") is None
