"""Fried-geometry Shack-Hartmann operator D and the observation matrix C (Sect. 3).

The paper emulates the sensor by a matrix D that takes differences of the phase
at the subaperture edges (Sect. 3).  Reading used (scaling and sign are not
printed): for subaperture (r, c) with corner phases a(r,c), a(r,c+1), a(r+1,c),
a(r+1,c+1), the x-slope is the mean of the two horizontal edge differences and
the y-slope the mean of the two vertical ones,
    s_x = [(a(r,c+1) - a(r,c)) + (a(r+1,c+1) - a(r+1,c))] / 2,
    s_y = [(a(r+1,c) - a(r,c)) + (a(r+1,c+1) - a(r,c+1))] / 2,
in radians of phase difference per pitch.

The state holds two phase instants (Sect. 2.1).  Reading used for which instant
the slopes see: C = [0 D] (obs_block = 1, one-frame sensor delay) or [D 0]
(obs_block = 0).
"""

from __future__ import annotations

import numpy as np

from .geometry import Geometry


def fried_matrix(geom: Geometry) -> np.ndarray:
    """Dense D, shape (p, n_act): rows are x-slopes then y-slopes of the valid subapertures."""
    ns, na = geom.n_subv, geom.n_act
    D = np.zeros((2 * ns, na))
    for k, (r, c) in enumerate(geom.sub_rc):
        i00 = geom.act_index[r, c]
        i01 = geom.act_index[r, c + 1]
        i10 = geom.act_index[r + 1, c]
        i11 = geom.act_index[r + 1, c + 1]
        D[k, i01] += 0.5
        D[k, i11] += 0.5
        D[k, i00] -= 0.5
        D[k, i10] -= 0.5
        D[ns + k, i10] += 0.5
        D[ns + k, i11] += 0.5
        D[ns + k, i00] -= 0.5
        D[ns + k, i01] -= 0.5
    return D


def observation_matrix(geom: Geometry, obs_block: int = 1) -> np.ndarray:
    """C (p x n): the slopes observe one of the state's two phase instants."""
    D = fried_matrix(geom)
    Z = np.zeros_like(D)
    return np.hstack([Z, D]) if obs_block == 1 else np.hstack([D, Z])
