"""Differential pistons between domains (Sect. 3.1, Fig. 3 discussion; Sect. 5) in FP64.

Test infrastructure only: the CUDA library never imports this module.

The local ETKF updates each domain separately, so the whole-pupil estimate stitched from the
domain estimates carries a different piston error on each domain.  The paper removes these
"differential pistons" with a post-processing step whose method it does not give, and names
removing them inside the loop as the next step.  Reading used here:

  * one piston delta_l per domain l, added to every actuator it owns: x' = x + P delta, with
    P (n_act x n_dom) the ownership indicator;
  * delta is the least-squares fit of the slope residual of the estimate,
        delta = argmin || (y - D x) - D P delta ||^2,
    where only subapertures whose corners belong to more than one domain carry information
    (a piston common to all four corners of a subaperture gives it zero slope);
  * the fit fixes delta only up to one constant per connected group of domains; the constant is
    chosen so that the correction adds no piston to the estimate: sum over the group's owned
    actuators of delta = 0;
  * "output" mode corrects only the reported prediction x_hat(k+1|k) with the frame's slopes y_k;
    "in_loop" mode also adds the same P delta to every member of both phase instants of the
    forecast ensemble, so that the next analysis starts from the corrected ensemble.

The least-squares problem is solved here by the SVD-based minimum-norm solution followed by the
gauge projection.
"""

from __future__ import annotations

from typing import List

import numpy as np
import scipy.sparse.csgraph as csgraph

from .fried import fried_matrix
from .geometry import Domain, Geometry


def ownership(geom: Geometry, domains: List[Domain]) -> np.ndarray:
    """P (n_act x n_dom): P[j, l] = 1 when domain l owns actuator j."""
    P = np.zeros((geom.n_act, len(domains)))
    for l, d in enumerate(domains):
        P[d.owned_act, l] = 1.0
    if not np.all(P.sum(axis=1) == 1.0):
        raise ValueError("every actuator must be owned by exactly one domain")
    return P


def domain_groups(geom: Geometry, domains: List[Domain]) -> np.ndarray:
    """Connected groups of domains: two domains are linked when a subaperture has corners in both."""
    DP = fried_matrix(geom) @ ownership(geom, domains)
    A = (np.abs(DP).T @ np.abs(DP)) > 0
    _, labels = csgraph.connected_components(A, directed=False)
    return labels


def differential_pistons(x: np.ndarray, y: np.ndarray, geom: Geometry, domains: List[Domain]) -> np.ndarray:
    """delta (n_dom): least-squares pistons of the slope residual y - D x, no piston added per group."""
    D = fried_matrix(geom)
    P = ownership(geom, domains)
    DP = D @ P
    r = np.asarray(y, dtype=np.float64) - D @ np.asarray(x, dtype=np.float64)
    delta = np.linalg.lstsq(DP, r, rcond=None)[0]
    n_own = P.sum(axis=0)
    for g in np.unique(labels := domain_groups(geom, domains)):
        sel = labels == g
        delta[sel] -= np.dot(n_own[sel], delta[sel]) / n_own[sel].sum()
    return delta


def remove_differential_pistons(x: np.ndarray, y: np.ndarray, geom: Geometry,
                                domains: List[Domain]) -> np.ndarray:
    """x + P delta (the corrected whole-pupil estimate)."""
    return np.asarray(x, dtype=np.float64) + ownership(geom, domains) @ differential_pistons(x, y, geom, domains)
