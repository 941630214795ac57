"""Shared set-up of the GPU parity tests: one workload, seen by the CUDA path and by the oracle.

Both sides get the same seeded inputs from `synth` (slopes, process-noise and
stationary covariance factors) and the same Philox seed; each side builds its
own geometry and draws its own normals.
"""

import functools

import numpy as np

from oracle import etkf, geometry
from synth import TruthStream, workload


@functools.lru_cache(maxsize=None)
def model(name, m=None, **over):
    w = workload(name)
    for k, v in over.items():
        setattr(w, k, v)
    if m is not None:
        w.m = m
    g = geometry.make_geometry(w.n_sub, w.obstruction)
    doms = geometry.make_domains(g, w.dom_sub, w.halo)
    L = w.process_noise_sqrt(g.act_rc)
    Ls = w.stationary_sqrt(g.act_rc)
    return w, g, doms, L, Ls


@functools.lru_cache(maxsize=None)
def slopes(name, n_frames, **over):
    w, g, _, _, _ = model(name, **over)
    fr = TruthStream(w).frames(0, n_frames + 1)
    y = np.concatenate([fr["slopes"][:, 0][:, g.sub_valid], fr["slopes"][:, 1][:, g.sub_valid]], axis=1)
    return np.ascontiguousarray(y), np.ascontiguousarray(fr["phi_act"][:, g.act_valid])


def oracle_filter(name, m=None, piston="off", **over):
    w, g, doms, L, Ls = model(name, m, **over)
    return etkf.OracleFilter(g, doms, w.m, w.ar1_a, w.sigma, seed=w.seed, L=L, L_stat=Ls, obs_block=w.obs_block,
                             a2=w.ar2_a, piston=piston)


def gpu_filter(name, precision, path, m=None, piston="off", simt_q_max=0, **over):
    from paper_1310_5954_gb300 import LETKF
    w, g, doms, L, Ls = model(name, m, **over)
    return LETKF(n_sub=w.n_sub, m=w.m, ar1_a=w.ar1_a, sigma=w.sigma, dom_sub=w.dom_sub, halo=w.halo,
                 obstruction=w.obstruction, q_sqrt=L, p0_sqrt=Ls, precision=precision, path=path,
                 seed=w.seed, obs_block=w.obs_block, ar2_a=w.ar2_a, piston=piston, simt_q_max=simt_q_max)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def domain_errors(xa, xo, doms, n_act):
    """Per domain: relative L2 error of its owned rows' analysis mean and of their anomalies
    (members minus that mean), GPU against oracle, over both state instants."""
    out = []
    for d in doms:
        r = d.rows(n_act)
        ma, mo = xa[r].mean(1), xo[r].mean(1)
        out.append((rel(ma, mo), rel(xa[r] - ma[:, None], xo[r] - mo[:, None])))
    return out


def assert_domainwise(xa, xo, doms, n_act, tol_mean, tol_anom, tag=""):
    """Every domain within the bounds; a failure names the worst domain (block, slopes, rows)."""
    xa = np.asarray(xa, dtype=np.float64)
    xo = np.asarray(xo, dtype=np.float64)
    errs = domain_errors(xa, xo, doms, n_act)
    for which, tol, name in ((0, tol_mean, "analysis mean"), (1, tol_anom, "anomalies")):
        k = max(range(len(errs)), key=lambda i: errs[i][which])
        d = doms[k]
        assert errs[k][which] < tol, (
            f"{tag}: {name} of domain {k} (block {d.I},{d.J}, p_loc {2 * d.obs_sub.size}, "
            f"n_loc {2 * d.owned_act.size}) off by {errs[k][which]:.3e} relative (bound {tol:.1e})")
    return errs
