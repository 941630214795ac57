#!/usr/bin/env python3
"""Benchmark of the local ETKF frame update on GB300.

One step = one filter frame of the whole hot path (slope check, process-noise draw,
observed anomalies, local Gram / eigensolve / weights per domain, transform,
AR(1) forecast, x_hat(k+1|k) output) for the ELT-class workload: 80 x 80
subapertures, 28 % obstruction, m = 100 members, 332 domains of 4 x 4
subapertures with a 2-subaperture halo.  Inputs are seeded synthetic von Karman
frozen-flow frames (see synth/).

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the same
workload instead (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LETKF frames/s and p99 frame latency, tuned vs plain, at matched residual RMS"
FP32_ALU_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="elt-80x80")
    ap.add_argument("--path", default="fused", choices=["fused", "plain"])
    ap.add_argument("--precision", default=None, choices=[None, "mixed", "fp32", "fp64"])
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-path comparison run")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--flush-mb", type=int, default=256)
    ap.add_argument("--profile-steps", type=int, default=30)
    ap.add_argument("--no-serving", action="store_true", help="skip the two serving-loop legs")
    ap.add_argument("--graph", action="store_true", help="fused path: each step as one CUDA graph launch")
    ap.add_argument("--no-autotune", action="store_true", help="fused path: default launch tuning")
    ap.add_argument("--mix-seconds", type=float, default=2.0, help="arrival window of the serving mix")
    ap.add_argument("--ns-frames", type=int, default=10000, help="frames of the non-stationary serving run")
    ap.add_argument("--no-piston", action="store_true", help="skip the differential-piston leg")
    ap.add_argument("--no-global", action="store_true", help="skip the global-ETKF (m = 1024) leg")
    ap.add_argument("--no-pair", action="store_true", help="skip the two-partition leg")
    ap.add_argument("--global-steps", type=int, default=200, help="timed steps of the global-ETKF leg")
    ap.add_argument("--oracle-probe", type=float, default=0.0,
                    help="(internal) time the oracle alone for this many seconds and print frames/s")
    ap.add_argument("--global-only", action="store_true",
                    help="run only the global-ETKF leg and print its JSON object (profiling)")
    ap.add_argument("--piston-frames", type=int, default=600, help="frames of the differential-piston leg")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampler of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        under = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(under), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_inputs(wname, n_frames, sub_valid, act_valid):
    """Seeded truth frames compressed with the filter's own geometry (valid subapertures/actuators)."""
    from synth import TruthStream, workload
    w = workload(wname)
    fr = TruthStream(w).frames(0, n_frames + 1)
    y = np.ascontiguousarray(np.concatenate([fr["slopes"][:, 0][:, sub_valid], fr["slopes"][:, 1][:, sub_valid]], axis=1))
    phi = fr["phi_act"][:, act_valid]
    return w, y, phi


def residual_rms(xpred, phi, burn):
    """sqrt of the mean over frames >= burn of ||phi_true(k+1) - x_hat(k+1|k)||^2 / n_act, piston removed.

    Frame k's prediction is scored by the truth of frame k + 1, so at most len(phi) - 1 predictions
    can be scored; more is a caller error."""
    if len(xpred) > len(phi) - 1:
        raise ValueError(f"{len(xpred)} predictions but truth for only {len(phi) - 1} of them")
    e = phi[1:len(xpred) + 1] - xpred
    e = e - e.mean(axis=1, keepdims=True)
    e = e[burn:]
    return float(math.sqrt(np.mean(np.sum(e * e, axis=1) / e.shape[1])))


def make_filter(w, path, precision, L, Ls, seed_offset=0, piston="off"):
    from paper_1310_5954_gb300 import LETKF
    return LETKF(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
                 obstruction=w.obstruction, q_sqrt=L, p0_sqrt=Ls, precision=precision, path=path,
                 seed=w.seed + seed_offset, obs_block=w.obs_block, piston=piston)


def run_device(f, y_dev, K, W, flush, torch):
    """W warm-up steps, then K timed steps, each bracketed by CUDA events on the filter's stream,
    with L2 flushed (a write larger than L2) before each timed step.  Returns per-step ms and all
    predictions (W + K, n_act) on the host."""
    st = f.stream
    preds = torch.empty((W + K, f.info.n_act), dtype=f.dtype, device=f.device)
    with torch.cuda.stream(st):
        for k in range(W):          # the same sequence as a timed step (flush, step), untimed
            flush.fill_(float(k & 7))
            f.step(y_dev[k], out=preds[k])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(st):
        for k in range(K):
            flush.fill_(float(k & 7))
            ev[k][0].record(st)
            f.step(y_dev[W + k], out=preds[W + k])
            ev[k][1].record(st)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = [a.elapsed_time(b) for a, b in ev]
    return ms, preds.double().cpu().numpy(), wall


def run_e2e(f, y_host, K, W, torch):
    """Through the public API with host buffers: per frame, pinned host -> device copy of the
    slopes, the step, and a device -> host read of x_hat(k+1|k); the frame is complete when
    the prediction is on the host."""
    st = f.stream
    p = f.info.p
    y_dev = torch.empty(p, dtype=f.dtype, device=f.device)
    out_dev = torch.empty(f.info.n_act, dtype=f.dtype, device=f.device)
    out_host = torch.empty(f.info.n_act, dtype=f.dtype, pin_memory=True)
    lat = []
    with torch.cuda.stream(st):
        for k in range(W):
            y_dev.copy_(y_host[k], non_blocking=True)
            f.step(y_dev, out=out_dev)
            out_host.copy_(out_dev, non_blocking=True)
            st.synchronize()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(K):
            t = time.perf_counter()
            y_dev.copy_(y_host[W + k], non_blocking=True)
            f.step(y_dev, out=out_dev)
            out_host.copy_(out_dev, non_blocking=True)
            st.synchronize()
            lat.append((time.perf_counter() - t) * 1e3)
        wall = time.perf_counter() - t0
    return K / wall, lat, p * y_dev.element_size(), f.info.n_act * out_dev.element_size()


def stage_profile(f, y_dev, steps, flush, torch):
    f.profile(True)
    with torch.cuda.stream(f.stream):
        for k in range(steps):
            flush.fill_(float(k & 7))
            f.step(y_dev[k % y_dev.shape[0]])
    return f.profile(False)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _global_roofline(tflops):
    """The global path's frame against the tensor peak (measured burst, else the fallback)."""
    pk = peaks().get("bf16_tflops")
    src = "MEASURED_PEAKS.json bf16_tflops (burst), of measured"
    if not pk:
        pk, src = 1900.0, "fallback 1.9 PFLOP/s bf16 burst, of fallback"
    return {"bound": "tensor", "achieved": tflops, "peak": pk, "unit": "TFLOP/s", "frac": tflops / pk,
            "peak_source": src}


def _traffic(kernel, workload, precision):
    """DRAM bytes per launch from the committed ncu summary of this kernel on this workload and
    precision (key "kernel:workload:precision"), or None when there is none or the kernel source
    changed since the counters were taken (the summary records its hash)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(f"{kernel}:{workload}:{precision}")
        src = os.path.join(ROOT, "paper_1310_5954_gb300", "csrc", rec["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        return rec["dram_bytes_per_launch"] if h == rec["source_sha256"] else None
    except Exception:
        return None


def roofline(f, prof, sms, sm_max_mhz, workload=None):
    """Roofline of the dominant stage (largest summed CUDA-event time over the profiled steps).

    Algorithmic work of one frame (per-unit counts):
      dense contractions  2 m^2 (sum p_loc + sum n_loc)  (local Gram and ensemble transform)
      eigensolve / inverse square root  11 m^3 per observing domain (the dense symmetric
      eigensolver count: 9 m^3 for eigenvalues and vectors, 2 m^3 to form T)
    The fused kernel runs all of it on the tensor cores, so it is measured against the BF16
    tensor peak (MEASURED_PEAKS.json, burst, of measured); the plain path's eigensolve stage
    runs on the FP32 ALUs, measured against 152 SMs x 128 lanes x 2 flop x max SM clock."""
    name, (ms, launches) = max(prof.items(), key=lambda kv: kv[1][0])
    per_launch_ms = ms / max(launches, 1)
    info = f.info
    m = info.m
    contraction = 2.0 * m * m * (info.sum_p_loc + info.sum_n_loc)
    eigen = 11.0 * m ** 3 * info.n_domains_observing
    if name == "fused_analysis_forecast":
        flops = contraction + eigen
        pk = peaks().get("bf16_tflops", 1900.0)
        achieved = flops / (per_launch_ms * 1e-3) / 1e12
        return {"kernel": "fused_kernel", "bound": "tensor", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": achieved / pk, "traffic": _traffic("fused_kernel", workload, f.precision), "per_launch_ms": per_launch_ms,
                "work_per_launch_flop": flops,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured"}
    if name == "eigensolve_weights":
        flops = eigen
        pk = sms * FP32_ALU_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
        achieved = flops / (per_launch_ms * 1e-3) / 1e12
        return {"kernel": "plain_eig", "bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": achieved / pk, "traffic": None, "per_launch_ms": per_launch_ms, "work_per_launch_flop": flops,
                "peak_source": f"{sms} SMs x {FP32_ALU_LANES_PER_SM} FP32 lanes x 2 x {sm_max_mhz:.0f} MHz (derived)"}
    bytes_ = 8.0 * info.n * m * (2 if f.precision == "fp64" else 1)
    pk = peaks().get("hbm_gbs", 6800.0)
    achieved = bytes_ / (per_launch_ms * 1e-3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": pk, "unit": "GB/s",
            "frac": achieved / pk, "traffic": None, "per_launch_ms": per_launch_ms, "work_per_launch_bytes": bytes_,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs, of measured"}


def cpu_baseline(wname, y, seconds, L, Ls, piston="off"):
    """The FP64 oracle as it stands, on this host's cores, over the first frames of the workload.

    y holds one more frame than can be scored (the truth of frame k + 1 scores frame k), so the
    oracle steps at most len(y) - 1 frames, whatever the time budget."""
    from oracle import etkf, geometry
    from synth import workload
    w = workload(wname)
    g = geometry.make_geometry(w.n_sub, w.obstruction)
    doms = geometry.make_domains(g, w.dom_sub, w.halo)
    o = etkf.OracleFilter(g, doms, w.m, w.ar1_a, w.sigma, seed=w.seed, L=L, L_stat=Ls, piston=piston)
    preds = []
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds and len(preds) < len(y) - 1:
        preds.append(o.step(y[len(preds)]))
    dt = time.perf_counter() - t0
    return len(preds) / dt, np.array(preds), len(preds), dt


def piston_leg(w, path, precision, L, Ls, y, phi, n_frames, flush, tuning, torch):
    """Differential pistons between domains (Sect. 3.1, Sect. 5): the same frames through the filter
    without correction, with the output corrected, and with the correction in the loop; per mode the
    per-step time (CUDA events, L2 flushed before each step), the residual RMS after a burn-in of
    half the frames, and the two correction kernels' share of the step."""
    n = min(n_frames, len(y) - 1)      # the truth of frame k + 1 scores frame k's prediction
    burn = n // 2
    out = {"frames": n, "burn_in": burn, "modes": {}}
    preds_in_loop = None
    for mode in ("off", "output", "in_loop"):
        f = make_filter(w, path, precision, L, Ls, 0, piston=mode)
        if path == "fused" and tuning:
            f.set_tuning(**tuning)
        ydev = torch.as_tensor(y[:n], dtype=f.dtype, device=f.device).contiguous()
        ms, preds, _ = run_device(f, ydev, n - 3, 3, flush, torch)
        rec = {"frames_per_s": (n - 3) / (sum(ms) / 1e3), "p50_ms": float(np.percentile(ms, 50)),
               "p99_ms": float(np.percentile(ms, 99)), "residual_rms": residual_rms(preds, phi, burn)}
        if mode != "off":
            prof = stage_profile(f, ydev, 30, flush, torch)
            if "differential_pistons" in prof:
                rec["piston_kernels_ms_per_step"] = prof["differential_pistons"][0] / 30
        rec["device_status"] = f.sync()
        f.close()
        out["modes"][mode] = rec
        if mode == "in_loop":
            preds_in_loop = preds
    return out, preds_in_loop


def pair_leg(w, precision, L, Ls, y, phi, K, W, flush, torch, single_rms, burn, oracle_seconds):
    """Two local ETKFs run together with two domain partitions (Sect. 5): the second filter's block
    grid shifted by half a block, its own seed; the output is the mean of the two predictions
    (letkf_step_pair, both filters' domains in one fused launch).  Per-step time (CUDA events, L2
    flushed before each step) and residual RMS on the headline frames next to the single filter's;
    the FP64 oracle's pair (two oracle filters averaged) on the first frames, bounded in time."""
    from paper_1310_5954_gb300 import LETKFPair
    p = LETKFPair(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
                  obstruction=w.obstruction, q_sqrt=L, p0_sqrt=Ls, precision=precision, seed=w.seed,
                  obs_block=w.obs_block)
    ydev = torch.as_tensor(y, dtype=p.dtype, device=p.device).contiguous()
    ms, preds, _ = run_device(p, ydev, K, W, flush, torch)
    status = p.sync()
    p.close()
    out = {"workload": f"{w.name}: two filters, block grids offset by {w.dom_sub // 2} subapertures, seeds "
                       f"{w.seed} and {w.seed + 1}, output the mean prediction",
           "frames_per_s": K / (sum(ms) / 1e3), "p50_ms": float(np.percentile(ms, 50)),
           "p99_ms": float(np.percentile(ms, 99)),
           "residual_rms": {"frames": W + K, "burn_in": burn, "pair": residual_rms(preds, phi, burn),
                            "single": single_rms},
           "device_status": status}
    if oracle_seconds > 0:
        from oracle import etkf, geometry
        g = geometry.make_geometry(w.n_sub, w.obstruction)
        mk = lambda off, seed: etkf.OracleFilter(g, geometry.make_domains(g, w.dom_sub, w.halo, offset=off), w.m,
                                                 w.ar1_a, w.sigma, seed=seed, L=L, L_stat=Ls, obs_block=w.obs_block)
        oa, ob = mk(0, w.seed), mk(w.dom_sub // 2, w.seed + 1)
        op = []
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < oracle_seconds and len(op) < len(y) - 1:
            k = len(op)
            op.append(0.5 * (oa.step(y[k]) + ob.step(y[k])))
        nf = len(op)
        nb = min(burn, max(nf - 2, 0))
        out["oracle_first_frames"] = {"frames": nf, "burn_in": nb, "oracle_pair": residual_rms(np.array(op), phi, nb),
                                      "gpu_pair": residual_rms(preds[:nf], phi, nb),
                                      "seconds": time.perf_counter() - t0}
    return out


def global_leg(steps, warmup, flush, torch, workers=16):
    """Global ETKF (Sect. 2.2: one domain, the whole pupil) at ELT scale with 1024 members on the
    tiled tensor-core GEMM: per-step time (CUDA events, L2 flushed before each step), the stage
    times, the algorithmic FP32 work per frame (Gram, Newton-Schulz products, transform, noise
    draw) and its rate; the tensor-core work is three split-BF16 products per FP32 product."""
    from paper_1310_5954_gb300 import LETKF
    from synth import compressed_frames, workload
    w = workload("etkf-elt-m1024")
    sv, av = _geometry(w)
    act_rc = np.argwhere(av)
    L = w.process_noise_sqrt(act_rc)
    Ls = w.stationary_sqrt(act_rc)
    n_fr = warmup + steps
    y, phi, _ = compressed_frames(w, 0, n_fr + 1, sv, av, workers)
    f = LETKF(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, obstruction=w.obstruction, q_sqrt=L, p0_sqrt=Ls,
              precision="fp32", path="global", seed=w.seed, obs_block=w.obs_block)
    ydev = torch.as_tensor(y[:n_fr], dtype=torch.float32, device=f.device).contiguous()
    ms, preds, _ = run_device(f, ydev, steps, warmup, flush, torch)
    ns_steps, s_bound = f.global_stats()
    prof = stage_profile(f, ydev, 20, flush, torch)
    status = f.sync()
    m, n, p, na = f.info.m, f.info.n, f.info.p, f.info.n_act
    lower = bool(np.allclose(L, np.tril(L)))
    work = {"gram": 2.0 * (m + 1) ** 2 * p, "newton_schulz": 2.0 * m ** 3 * (1 + 3 * max(ns_steps - 1, 0)),
            "transform": 2.0 * n * m * m, "noise": 2.0 * na * na * m / (2.0 if lower else 1.0)}
    tot = sum(work.values())
    t_med = float(np.median(ms)) / 1e3
    f.close()
    burn = n_fr // 2
    return {"workload": f"{w.name}: 80x80, 28% obstruction, one domain (n={n}, p={p}), m={m}, FP32 "
                        f"(split-BF16 tensor-core products)",
            "frames_per_s": steps / (sum(ms) / 1e3), "p50_ms": float(np.median(ms)), "p99_ms": float(np.percentile(ms, 99)),
            "stages_ms_per_step": {k: v[0] / 20 for k, v in prof.items()},
            "newton_schulz_steps_last_frame": ns_steps, "spectral_bound_last_frame": s_bound,
            "fp32_work_gflop_per_frame": {k: v / 1e9 for k, v in work.items()},
            "fp32_work_tflops_at_p50": tot / t_med / 1e12,
            "bf16_tensor_tflops_at_p50": 3.0 * tot / t_med / 1e12,
            # the whole frame against the tensor peak: the tensor-core work (three BF16 products
            # per FP32 product) over the frame's p50 time
            "roofline": _global_roofline(3.0 * tot / t_med / 1e12),
            "residual_rms": {"frames": n_fr, "burn_in": burn, "gpu": residual_rms(preds, phi, burn)},
            "device_status": status}


def etkf_vs_letkf(w, L, Ls, y, phi, burn, letkf_rms, torch):
    """Sect. 3.1 (Fig. 3): at the same ensemble size the local ETKF beats the global ETKF.  The
    global path with the local filter's ensemble size, run over the same frames as the headline
    leg, residual RMS next to the local filter's."""
    from paper_1310_5954_gb300 import LETKF
    f = LETKF(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, obstruction=w.obstruction, q_sqrt=L, p0_sqrt=Ls,
              precision="fp32", path="global", seed=w.seed, obs_block=w.obs_block)
    ydev = torch.as_tensor(y, dtype=torch.float32, device=f.device).contiguous()
    n = len(y) - 1
    preds = torch.empty((n, f.info.n_act), dtype=torch.float32, device=f.device)
    for k in range(n):
        f.step(ydev[k], out=preds[k])
    status = f.sync()
    f.close()
    p = preds.double().cpu().numpy()
    finite = np.isfinite(p).all(axis=1)
    out = {"m": w.m, "frames": n, "burn_in": burn, "local_etkf_residual_rms": letkf_rms, "device_status": status}
    if finite.all():
        out["global_etkf_residual_rms"] = residual_rms(p, phi, burn)
    else:   # the unlocalised filter diverged: report where, not a non-finite number
        out["global_etkf_residual_rms"] = None
        out["global_etkf_first_nonfinite_frame"] = int(np.argmin(finite))
    return out


def _geometry(w):
    """Valid subaperture / actuator masks as the library computes them (a small probe context)."""
    from paper_1310_5954_gb300 import LETKF
    # the masks do not depend on the domains: any valid decomposition serves
    probe = LETKF(n_sub=w.n_sub, m=4, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=4, halo=0,
                  obstruction=w.obstruction, q_white=0.1, precision="fp32", path="plain")
    sv, av = probe.geometry()
    probe.close()
    return sv, av


def _lat_stats(lat_ms):
    lat = np.asarray(lat_ms, dtype=np.float64)
    if lat.size == 0:
        return {"frames": 0}
    return {"frames": int(lat.size), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max())}


def _replay_mix(srv, systems, seconds, rate_scale, n_cycle, seed):
    """Seeded Poisson arrivals (each system at rate_scale x its rate) replayed in real time."""
    rng = np.random.default_rng(seed)
    ev = []
    for s in systems:
        rate = s["rate"] * rate_scale
        t = rng.exponential(1.0 / rate)
        k = 2
        while t < seconds:
            ev.append((t, s["sid"], k % n_cycle))
            k += 1
            t += rng.exponential(1.0 / rate)
    ev.sort()
    by_sid = {s["sid"]: s for s in systems}
    info0 = srv.info()
    t0 = time.perf_counter()
    refused = srv.replay([e[1] for e in ev], [int(e[0] * 1e9) for e in ev], [by_sid[e[1]]["y"][e[2]] for e in ev])
    wall = time.perf_counter() - t0
    recs = srv.records()
    info = srv.info()
    lat = {}
    for r in recs:
        lat.setdefault(r["system"], []).append((r["t_done_ns"] - r["t_arrival_ns"]) / 1e6)
    by_size = {}
    for s in systems:
        by_size.setdefault(f"{s['w'].n_sub}x{s['w'].n_sub}", []).extend(lat.get(s["sid"], []))
    all_lat = [v for l in lat.values() for v in l]
    batches = info["batches"] - info0["batches"]
    return {"rate_scale": rate_scale, "arrival_window_s": seconds, "wall_s": wall, "offered_frames": len(ev),
            "refused_frames": refused, "offered_frames_per_s": len(ev) / seconds,
            "served_frames_per_s": len(recs) / wall,
            "mean_batch_systems": (info["batched_systems"] - info0["batched_systems"]) / max(batches, 1),
            "latency_all": _lat_stats(all_lat),
            "latency_by_size": {k: _lat_stats(v) for k, v in
                                sorted(by_size.items(), key=lambda kv: int(kv[0].split("x")[0]))}}


def serving_mix_leg(seconds, n_cycle=32, workers=8):
    """16 AO systems of mixed sizes and ensemble sizes served together (synth.serving_mix): every
    system's ensemble resident on the device, frames arriving as seeded Poisson streams, batched
    continuously by the library's server.  Each system's slopes cycle over its first n_cycle truth
    frames (the work per frame does not depend on the data).

    First each system's frame alone through the server gives its service time; their sum weighted
    by the arrival rates is the offered load in GPU-seconds per second.  The mix then runs at its
    nominal rates (overloaded when that load exceeds 1: frames beyond a 16-deep queue per system are
    refused) and at rates scaled to 80 % of the measured capacity, where the latencies mean
    something."""
    from paper_1310_5954_gb300 import Server
    from synth import compressed_frames, serving_mix
    mix = serving_mix()
    srv = Server(slots=2, max_pending=16, max_batch=32)
    systems = []
    t_setup = time.perf_counter()
    for e in mix:
        w = e["workload"]
        sv, av = _geometry(w)
        L = w.process_noise_sqrt(np.argwhere(av))
        sid = srv.admit(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
                        obstruction=w.obstruction, q_sqrt=L, precision="mixed", seed=w.seed, obs_block=w.obs_block)
        del L
        y, _, _ = compressed_frames(w, 0, n_cycle, sv, av, workers)
        systems.append({"sid": sid, "w": w, "rate": e["rate_hz"], "y": [np.ascontiguousarray(r) for r in y]})
    setup_s = time.perf_counter() - t_setup
    # each system alone: two warm-up frames, then 10 frames one at a time (launch -> completion)
    per_system = []
    load = 0.0
    for s in systems:
        for k in range(2):
            srv.submit(s["sid"], s["y"][k])
            srv.drain()
        srv.records()
        for k in range(10):
            srv.submit(s["sid"], s["y"][k % n_cycle])
            srv.drain()
        svc = [(r["t_done_ns"] - r["t_launch_ns"]) / 1e6 for r in srv.records()]
        t_ms = float(np.median(svc))
        load += s["rate"] * t_ms * 1e-3
        per_system.append({"system": s["w"].name, "rate_hz": s["rate"], "service_ms_alone": t_ms})
    nominal = _replay_mix(srv, systems, seconds, 1.0, n_cycle, 1310595444)
    scale = min(1.0, 0.8 / load) if load > 0 else 1.0
    sustained = _replay_mix(srv, systems, seconds, scale, n_cycle, 1310595445)
    out = {"workload": "serving mix: 16 systems, sizes {16,32,40,64,80,100}^2 subapertures, m in {20,50,100,200}, "
                       "Poisson arrivals at 500 Hz - 2 kHz per system, mixed precision, fused path, 2 stream slots",
           "offered_load_gpu_s_per_s": load, "nominal_rates": nominal, "rates_at_80pct_capacity": sustained,
           "per_system": per_system, "hbm_used_bytes": srv.info()["hbm_used"], "setup_s": setup_s,
           "data": f"synthetic: each system's slopes cycle over its first {n_cycle} seeded truth frames"}
    srv.close()
    return out


def nonstationary_leg(n_frames, workers=16, oracle_seconds=15.0):
    """The non-stationary ELT system (r0 halves at frame 3000, wind 10 -> 25 m/s rotating 90 deg
    over frames 6000-7000, noise 0.1 -> 0.3 rad at 8000) fed through the serving loop at a fixed
    1 kHz arrival: per-frame latency, and the residual phase RMS per phase of the schedule; the
    FP64 oracle runs the first frames for the residual comparison (bounded time)."""
    from paper_1310_5954_gb300 import Server
    from synth import compressed_frames, workload
    w = workload("elt-80x80-nonstationary")
    sv, av = _geometry(w)
    act_rc = np.argwhere(av)
    L = w.process_noise_sqrt(act_rc)
    Ls = w.stationary_sqrt(act_rc)
    t_gen = time.perf_counter()
    y, phi, sig = compressed_frames(w, 0, n_frames + 1, sv, av, workers)
    gen_s = time.perf_counter() - t_gen
    srv = Server(slots=2, max_pending=1024, max_batch=1)
    sid = srv.admit(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma_at(0), dom_sub=w.dom_sub, halo=w.halo,
                    obstruction=w.obstruction, q_sqrt=L, p0_sqrt=Ls, precision="mixed", seed=w.seed,
                    obs_block=w.obs_block)
    pred = srv.set_output(sid, n_frames)
    ys = [np.ascontiguousarray(y[k]) for k in range(n_frames)]
    t0 = time.perf_counter()
    refused = srv.replay([sid] * n_frames, [k * 1_000_000 for k in range(n_frames)], ys, sigma=sig[:n_frames])
    wall = time.perf_counter() - t0
    recs = srv.records()
    srv.close()
    lat = np.array([(r["t_done_ns"] - r["t_arrival_ns"]) / 1e6 for r in recs if r["frame"] >= 100])
    e = phi[1:n_frames + 1].astype(np.float64) - pred.astype(np.float64)
    e -= e.mean(axis=1, keepdims=True)
    rms_k = np.sqrt(np.mean(e * e, axis=1))
    phases = [(100, 3000, "stationary"), (3000, 6000, "r0 halved"), (6000, 7000, "wind ramp + rotation"),
              (7000, 8000, "25 m/s"), (8000, n_frames, "noise 0.3 rad")]
    rms = {}
    for a, b, nm in phases:
        if b > a and a < n_frames:
            rms[f"{a}-{min(b, n_frames)} {nm}"] = float(np.sqrt(np.mean(rms_k[a:min(b, n_frames)] ** 2)))
    out = {"workload": f"{w.name}: 80x80, m={w.m}, 1 kHz fixed arrival through the serving loop",
           "frames": n_frames, "refused_frames": refused, "wall_s": wall, "served_frames_per_s": len(recs) / wall,
           "latency_after_frame_100": _lat_stats(lat), "residual_rms_by_phase": rms, "frame_generation_s": gen_s}
    inputs = {"w": w, "y": y, "phi": phi, "sigma": sig, "L": L, "Ls": Ls, "pred": pred}
    return out, inputs


def cpu_baseline_nonstationary(inp, seconds):
    """cpu_baseline leg, second part: the FP64 oracle on the first frames of the non-stationary
    run (bounded time), residual RMS next to the served GPU filter's on the same frames."""
    from oracle import etkf, geometry
    w = inp["w"]
    g = geometry.make_geometry(w.n_sub, w.obstruction)
    doms = geometry.make_domains(g, w.dom_sub, w.halo)
    o = etkf.OracleFilter(g, doms, w.m, w.ar1_a, w.sigma_at(0), seed=w.seed, L=inp["L"], L_stat=inp["Ls"])
    y, phi, sig = inp["y"], inp["phi"], inp["sigma"]
    op = []
    t1 = time.perf_counter()
    while time.perf_counter() - t1 < seconds and len(op) < len(inp["pred"]):
        k = len(op)
        op.append(o.step(y[k].astype(np.float64), sigma=float(sig[k])))
    nf = len(op)
    burn = nf // 2

    def rms(p):
        e = phi[1:nf + 1].astype(np.float64) - p
        e = e - e.mean(axis=1, keepdims=True)
        return float(np.sqrt(np.mean(e[burn:] ** 2)))
    return {"frames": nf, "burn_in": burn, "oracle": rms(np.array(op)),
            "gpu": rms(inp["pred"][:nf].astype(np.float64)), "seconds": time.perf_counter() - t1}


def oracle_probe(wname, seconds):
    """The oracle alone on the first frames of the workload for a bounded time (run in a child
    process whose BLAS thread count the parent sets)."""
    from oracle import geometry
    from synth import workload
    w = workload(wname)
    g = geometry.make_geometry(w.n_sub, w.obstruction)
    L = w.process_noise_sqrt(g.act_rc)
    Ls = w.stationary_sqrt(g.act_rc)
    _, y, _ = workload_inputs(wname, 64, g.sub_valid, g.act_valid)
    fps, _, nfr, dt = cpu_baseline(wname, y, seconds, L, Ls)
    print(json.dumps({"frames_per_s": fps, "frames": nfr, "seconds": dt}))


def oracle_single_thread(wname, seconds):
    """cpu_baseline at one thread: the same oracle in a child process with every BLAS / OpenMP
    thread pool limited to one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--workload", wname, "--oracle-probe", str(seconds)],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"unavailable": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else "probe failed"}
    return json.loads(r.stdout.strip().splitlines()[-1])


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.oracle_probe > 0:
        return oracle_probe(args.workload, args.oracle_probe)
    if args.impl == "reference":
        return reference_main(args, world, rank)
    import torch
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1310_5954_gb300 import LETKF  # noqa: F401
    if args.global_only:
        flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device=dev)
        print(json.dumps(global_leg(args.global_steps, 5, flush, torch)))
        return
    from synth import workload
    precision = args.precision or ("mixed" if args.path == "fused" else "fp32")
    w = workload(args.workload)
    K, W = args.steps, args.warmup
    # geometry from the library itself (what the filter will use)
    probe = LETKF(n_sub=w.n_sub, m=4, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
                  obstruction=w.obstruction, q_white=0.1, precision="fp32", path="plain")
    sub_valid, act_valid = probe.geometry()
    probe.close()
    act_rc = np.argwhere(act_valid)
    L = w.process_noise_sqrt(act_rc)
    Ls = w.stationary_sqrt(act_rc)
    w, y, phi = workload_inputs(args.workload, W + K, sub_valid, act_valid)
    flush = torch.empty(args.flush_mb * (1 << 20) // 4, dtype=torch.float32, device=dev)

    def timed(path, prec, seed_offset):
        f = make_filter(w, path, prec, L, Ls, seed_offset)
        ydev = torch.as_tensor(y, dtype=f.dtype, device=dev).contiguous()
        if path == "fused":
            if args.graph:
                f.set_graph(True)
            elif not args.no_autotune:
                tuned[path] = f.autotune(ydev[0], frames=20)
        if world > 1:
            dist.barrier()
        ms, preds, wall = run_device(f, ydev, K, W, flush, torch)
        prof = stage_profile(f, ydev, args.profile_steps, flush, torch)
        status = f.sync()
        return f, ms, preds, wall, prof, ydev, status

    tuned = {}
    clocks = Clocks(local)
    f, ms, preds, wall, prof, ydev, status = timed(args.path, precision, rank)
    clk = clocks.stop()
    tot = sum(ms) / 1e3
    if world > 1:
        t = torch.tensor([tot], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot = float(t.item())
    value = world * K / tot
    sm_max = clk.get("sm_max_mhz") or 2070.0
    roof = roofline(f, prof, torch.cuda.get_device_properties(dev).multi_processor_count, sm_max, args.workload)
    # end to end through the public API, host buffers
    y_host = torch.as_tensor(y, dtype=f.dtype).pin_memory()
    fe = make_filter(w, args.path, precision, L, Ls, rank)
    if args.path == "fused":
        if args.graph:
            fe.set_graph(True)
        elif args.path in tuned:
            fe.set_tuning(**tuned[args.path]["tuning"])
    e2e_fps, e2e_lat, h2d, d2h = run_e2e(fe, y_host, K, W, torch)
    fe.close()
    burn = min(50, (W + K) // 4)
    out = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * tot / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "bf16+f32", "fp32": "f32", "fp64": "f64"}[precision], "data": "synthetic",
        "impl": "gpu",
        "config": {"workload": f"{w.name}: {w.n_sub}x{w.n_sub} subapertures, {int(w.obstruction * 100)}% "
                               f"obstruction, m={w.m}, {f.info.n_domains} domains {w.dom_sub}x{w.dom_sub}+halo "
                               f"{w.halo}, n={f.info.n}, p={f.info.p}",
                   "path": args.path, "precision": precision,
                   "cuda_graph": args.path == "fused" and (args.graph or
                                                            bool(tuned.get(args.path, {}).get("tuning", {}).get("graph"))),
                   "launch_tuning": tuned.get(args.path),
                   "l2": f"flushed before every timed step ({args.flush_mb} MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "roofline": roof,
        # main-stream stages (profiled) plus the side stream's noise draw for the next frame: in
        # mixed precision normals, tensor-core product and partial-sum kernels; in FP32 the normals
        # kernel (the GEMM is cuBLAS's)
        "gpu_launches": int(K * sum(v[1] for v in prof.values()) / max(args.profile_steps, 1))
                        + (K * (3 if precision == "mixed" else 1) if args.path == "fused" else 0),
        "stages_ms_per_step": {k: v[0] / args.profile_steps for k, v in prof.items()},
        "clocks": clk, "device_status": status,
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "p50_ms": float(np.percentile(e2e_lat, 50)), "p99_ms": float(np.percentile(e2e_lat, 99))},
        "residual_rms": {"frames": W + K, "burn_in": burn, args.path: residual_rms(preds, phi, burn)},
        # the paper's only timing (Sect. 4), on other hardware and another workload: context only
        "paper_context": {"one_domain_update_s": 0.005, "loop_budget_s": 0.002,
                          "hardware": "Intel Xeon W3565, 4 cores (CPU, precision not stated)",
                          "workload": "40 m telescope, 69 domains, m = 197, n_max = 162, p_max = 242",
                          "this_run_frame_s": tot / K},
    }
    f.close()
    if world == 1 and not args.no_compare:
        other = "plain" if args.path == "fused" else None
        if other:
            fp, msp, predp, _, profp, _, stp = timed(other, "fp32", 0)
            out["plain"] = {"value": K / (sum(msp) / 1e3), "ms_per_step": sum(msp) / K,
                            "p50_ms": float(np.percentile(msp, 50)), "p99_ms": float(np.percentile(msp, 99)),
                            "stages_ms_per_step": {k: v[0] / args.profile_steps for k, v in profp.items()},
                            "device_status": stp}
            out["residual_rms"]["plain"] = residual_rms(predp, phi, burn)
            out["speedup_vs_plain"] = out["value"] / out["plain"]["value"]
            fp.close()
    preds_pl = None
    if rank == 0 and world == 1 and not args.no_piston:
        out["piston_removal"], preds_pl = piston_leg(w, args.path, precision, L, Ls, y, phi, args.piston_frames,
                                                     flush, tuned.get(args.path, {}).get("tuning"), torch)
    if rank == 0 and world == 1 and not args.no_pair and args.path == "fused":
        out["two_partitions"] = pair_leg(w, precision, L, Ls, y, phi, K, W, flush, torch,
                                         out["residual_rms"][args.path], burn,
                                         0.0 if args.no_cpu_baseline else args.cpu_seconds / 2)
    if rank == 0 and world == 1 and not args.no_global:
        out["global_etkf"] = global_leg(args.global_steps, 5, flush, torch)
        out["global_etkf"]["same_m_as_local"] = etkf_vs_letkf(w, L, Ls, y, phi, burn,
                                                              out["residual_rms"][args.path], torch)
    ns_inputs = None
    if rank == 0 and world == 1 and not args.no_serving:
        out["serving_mix"] = serving_mix_leg(args.mix_seconds)
        out["serving_nonstationary"], ns_inputs = nonstationary_leg(args.ns_frames)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fps, opreds, nfr, dt = cpu_baseline(args.workload, y, args.cpu_seconds, L, Ls)
        out["cpu_baseline"] = {"value": fps, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"first {nfr} frames of {w.name}, FP64 numpy/LAPACK oracle, {dt:.1f} s",
                               "single_thread": oracle_single_thread(args.workload, args.cpu_seconds / 2)}
        nb = min(burn, max(nfr - 2, 0))
        out["residual_rms"]["oracle_first_frames"] = {"frames": nfr, "burn_in": nb,
                                                      "oracle": residual_rms(opreds, phi, nb),
                                                      args.path: residual_rms(preds[:nfr], phi, nb)}
        if "plain" in out:
            out["residual_rms"]["oracle_first_frames"]["plain"] = residual_rms(predp[:nfr], phi, nb)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and preds_pl is not None:
        # the oracle's in-loop filter on the first frames, next to the GPU's in-loop run
        _, opl, nfr, dt = cpu_baseline(args.workload, y, args.cpu_seconds / 2, L, Ls, piston="in_loop")
        nb = min(burn, max(nfr - 2, 0))
        out["piston_removal"]["oracle_first_frames"] = {"frames": nfr, "burn_in": nb, "seconds": dt,
                                                        "oracle_in_loop": residual_rms(opl, phi, nb),
                                                        "gpu_in_loop": residual_rms(preds_pl[:nfr], phi, nb)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and ns_inputs is not None:
        out["serving_nonstationary"]["oracle_first_frames"] = cpu_baseline_nonstationary(ns_inputs, 15.0)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def reference_main(args, world, rank):
    """The oracle as it stands on the host cores (rank 0 only): W + K frames of the same workload,
    each frame one step, stopped early after a bounded time budget."""
    if rank != 0:
        return
    from oracle import geometry
    from synth import workload
    w = workload(args.workload)
    g = geometry.make_geometry(w.n_sub, w.obstruction)
    L = w.process_noise_sqrt(g.act_rc)
    Ls = w.stationary_sqrt(g.act_rc)
    _, y, _ = workload_inputs(args.workload, args.warmup + args.steps, g.sub_valid, g.act_valid)
    from oracle import etkf
    doms = geometry.make_domains(g, w.dom_sub, w.halo)
    o = etkf.OracleFilter(g, doms, w.m, w.ar1_a, w.sigma, seed=w.seed, L=L, L_stat=Ls)
    for k in range(args.warmup):
        o.step(y[k])
    budget = 150.0
    t0 = time.perf_counter()
    done = 0
    for k in range(args.steps):
        o.step(y[args.warmup + k])
        done += 1
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    fps = done / dt
    out = {"metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world, "steps": done,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / done, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"{w.name}: {w.n_sub}x{w.n_sub} subapertures, m={w.m}, {len(doms)} domains",
                      "path": "oracle"},
           "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"{done} frames after {args.warmup} warm-up frames"
                                      + (" (stopped at the time budget)" if done < args.steps else "")},
           "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
