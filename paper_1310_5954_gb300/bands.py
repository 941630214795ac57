"""Row-band partition of one AO system's domains over ranks (one GPU each), and the per-frame
exchange of ghost rows.

Domains are independent within a frame (Sect. 2.3): a domain's analysis reads the observed
instant of the actuators at the corners of its observed subapertures (its halo), and updates only
the actuators it owns.  Cutting the pupil into contiguous bands of block rows, one band per rank,
each rank updates and forecasts its own actuators, and the only data that crosses ranks is, once
per frame after the forecast, the observed-instant rows of the halo actuators that a neighbouring
band owns.  The plan is computed on the host from the library's domain tables
(letkf_domain_tables); the exchange uses torch.distributed point-to-point messages.
"""

from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

from . import _lib


@dataclasses.dataclass
class BandPlan:
    rank: int
    n_ranks: int
    block_rows: tuple            # [first, end) block rows of this band
    domains: np.ndarray          # domain indices (library numbering)
    owned: np.ndarray            # valid actuators this rank updates (rows of both instants)
    ghosts: np.ndarray           # halo actuators of its domains owned by other ranks
    send: Dict[int, np.ndarray]  # rank -> own actuators that rank reads, in its receive order
    recv: Dict[int, np.ndarray]  # rank -> ghost actuators received from that rank
    cost: float                  # load estimate of the band


def domain_cost(tables: dict, m: int) -> np.ndarray:
    """Load estimate of each domain: the m^3 transform of an observing domain (Sect. 2.3 cost
    O(m^3 + m^2 (n + p))) plus its m^2 (n_loc + p_loc) products; a domain without observation
    only copies its rows."""
    n_loc = 2 * np.diff(tables["own_off"])
    p_loc = 2 * np.diff(tables["obs_off"])
    return np.where(p_loc > 0, float(m) ** 3 + float(m) ** 2 * (n_loc + p_loc), float(m) * n_loc)


def partition(tables: dict, n_ranks: int, m: int) -> List[BandPlan]:
    """Contiguous bands of block rows, one per rank, balanced by domain_cost (each band ends at the
    block row where the running cost comes closest to its share of the total)."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    bps = int(tables["blocks_per_side"])
    block_row = tables["block"] // bps
    cost = domain_cost(tables, m)
    row_cost = np.bincount(block_row, weights=cost, minlength=bps)
    cum = np.cumsum(row_cost)
    total = cum[-1]
    # band r ends at the block row whose running cost is closest to r / n_ranks of the total,
    # keeping at least one block row per band while rows remain
    cuts = [0]
    for r in range(1, n_ranks):
        target = total * r / n_ranks
        c = int(np.argmin(np.abs(cum - target))) + 1
        c = max(c, cuts[-1] + 1)
        c = min(c, bps - (n_ranks - r)) if bps >= n_ranks else min(max(c, cuts[-1]), bps)
        cuts.append(c)
    cuts.append(bps)
    own_off, own = tables["own_off"], tables["own"]
    halo_off, halo = tables["halo_off"], tables["halo"]
    n_act = int(tables["n_act"])
    owner = np.full(n_act, -1, dtype=np.int64)
    dom_rank = np.searchsorted(np.array(cuts[1:]), block_row, side="right")
    for d in range(len(block_row)):
        owner[own[own_off[d]:own_off[d + 1]]] = dom_rank[d]
    if (owner < 0).any():
        raise RuntimeError("an actuator has no owning domain")
    plans = []
    need = []
    for r in range(n_ranks):
        doms = np.nonzero(dom_rank == r)[0]
        owned = np.sort(np.concatenate([own[own_off[d]:own_off[d + 1]] for d in doms])) if doms.size else \
            np.zeros(0, dtype=np.int64)
        reads = np.unique(np.concatenate([halo[halo_off[d]:halo_off[d + 1]] for d in doms])) if doms.size else \
            np.zeros(0, dtype=np.int64)
        ghosts = reads[owner[reads] != r]
        need.append(ghosts)
        plans.append(BandPlan(rank=r, n_ranks=n_ranks, block_rows=(cuts[r], cuts[r + 1]), domains=doms,
                              owned=owned, ghosts=ghosts, send={}, recv={}, cost=float(cost[doms].sum())))
    for r in range(n_ranks):
        g = need[r]
        for q in np.unique(owner[g]):
            ids = g[owner[g] == q]
            plans[r].recv[int(q)] = ids
            plans[int(q)].send[r] = ids
    return plans


def plan_for(n_ranks: int, **system) -> List[BandPlan]:
    """partition() of the system described by LETKF's keyword arguments."""
    from .letkf import make_params
    p, keep = make_params(**system)
    return partition(_lib.letkf_domain_tables(p), n_ranks, int(system["m"]))


def exchange(plan: BandPlan, x_obs, group: Optional[object] = None) -> None:
    """After the forecast: send the observed-instant rows of own actuators to the ranks whose
    halos read them and receive this rank's ghost rows, in place.  x_obs is a torch tensor whose
    row j is valid actuator j's observed instant (n_act x m, on the rank's device)."""
    import torch
    import torch.distributed as dist
    reqs = []
    bufs = []
    for q in sorted(set(plan.send) | set(plan.recv)):
        if q in plan.send:
            idx = torch.as_tensor(plan.send[q], dtype=torch.int64, device=x_obs.device)
            out = x_obs.index_select(0, idx).contiguous()
            bufs.append(out)
            reqs.append(dist.isend(out, dst=q, group=group))
        if q in plan.recv:
            inb = torch.empty((len(plan.recv[q]),) + tuple(x_obs.shape[1:]), dtype=x_obs.dtype, device=x_obs.device)
            bufs.append((q, inb))
            reqs.append(dist.irecv(inb, src=q, group=group))
    for r in reqs:
        r.wait()
    for b in bufs:
        if isinstance(b, tuple):
            q, inb = b
            x_obs.index_copy_(0, torch.as_tensor(plan.recv[q], dtype=torch.int64, device=x_obs.device), inb)
