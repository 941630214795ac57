"""Pupil geometry and domain decomposition (Sect. 3 set-up; Sect. 2.3, Fig. 1).

Readings of the paper used here:
* A subaperture is valid when at least half of its area lies inside the annular
  pupil [obstruction * R, R], R = N/2 pitches, centred on the grid (Sect. 3: a
  sensor "with a transmission factor equal to 0.5").  The area fraction is the
  share of a 20 x 20 grid of midpoints that fall inside, compared in exact
  integer arithmetic for the outer edge.  This reproduces the paper's counts:
  241 valid actuators for 16 x 16 and 877 actuators / 812 subapertures
  (p = 1624, n = 1754) for 32 x 32 (Sect. 3 and Sect. 3.2).
* Fried geometry: actuators sit on subaperture corners; an actuator is valid
  when it is a corner of at least one valid subaperture (Sect. 3, Fig. 1).
* Estimation domains (Sect. 2.3): the subaperture grid is cut into b x b blocks;
  block (I, J) owns the actuators with floor(r/b) = I and floor(c/b) = J, the last
  actuator row/column folding into the last block.  Its observation region is
  the valid subapertures in rows [bI-h, b(I+1)+h) x columns [bJ-h, b(J+1)+h),
  clipped to the grid, both slope directions.  Blocks owning no valid actuator
  are dropped.

Index conventions: row r is y, column c is x; valid actuators and valid
subapertures are numbered in row-major grid order.  The state x stacks two
phase instants on the valid actuators ([block 1; block 2], n = 2 n_act); the
slope vector y stacks all x-slopes then all y-slopes (p = 2 n_sub_valid).
"""

from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

_SAMPLES = 20  # midpoint samples per subaperture side


def subaperture_mask(n_sub: int, obstruction: float = 0.0) -> np.ndarray:
    """Valid-subaperture mask (N x N, row-major [r, c]) by the half-illumination rule."""
    q = _SAMPLES
    s = 2 * np.arange(q) + 1                      # midpoint numerators, unit 1/(2q) pitch
    R2 = (q * n_sub) ** 2                         # outer radius^2 in those units
    rin2 = (obstruction * q * n_sub) ** 2
    mask = np.zeros((n_sub, n_sub), dtype=bool)
    for r in range(n_sub):
        b = 2 * q * r + s[:, None] - q * n_sub    # y numerators
        for c in range(n_sub):
            a = 2 * q * c + s[None, :] - q * n_sub
            d2 = a * a + b * b
            inside = (d2 <= R2) & (d2 >= rin2)
            mask[r, c] = 2 * int(inside.sum()) >= q * q
    return mask


def actuator_mask(sub_valid: np.ndarray) -> np.ndarray:
    """Valid actuators ((N+1) x (N+1)): corners of at least one valid subaperture."""
    n = sub_valid.shape[0]
    act = np.zeros((n + 1, n + 1), dtype=bool)
    act[:-1, :-1] |= sub_valid
    act[:-1, 1:] |= sub_valid
    act[1:, :-1] |= sub_valid
    act[1:, 1:] |= sub_valid
    return act


@dataclasses.dataclass
class Geometry:
    n_sub: int
    sub_valid: np.ndarray        # (N, N) bool
    act_valid: np.ndarray        # (N+1, N+1) bool
    sub_rc: np.ndarray           # (n_subv, 2) row, col of valid subapertures
    act_rc: np.ndarray           # (n_act, 2)
    act_index: np.ndarray        # (N+1, N+1) valid index or -1
    sub_index: np.ndarray        # (N, N) valid index or -1

    @property
    def n_act(self) -> int:
        return int(self.act_rc.shape[0])

    @property
    def n_subv(self) -> int:
        return int(self.sub_rc.shape[0])

    @property
    def n(self) -> int:          # state dimension, two phase instants
        return 2 * self.n_act

    @property
    def p(self) -> int:          # observation dimension, two slope directions
        return 2 * self.n_subv


def make_geometry(n_sub: int, obstruction: float = 0.0, sub_valid: np.ndarray = None) -> Geometry:
    if sub_valid is None:
        sub_valid = subaperture_mask(n_sub, obstruction)
    sub_valid = np.asarray(sub_valid, dtype=bool)
    act_valid = actuator_mask(sub_valid)
    sub_rc = np.argwhere(sub_valid)
    act_rc = np.argwhere(act_valid)
    act_index = -np.ones(act_valid.shape, dtype=np.int64)
    act_index[act_valid] = np.arange(act_rc.shape[0])
    sub_index = -np.ones(sub_valid.shape, dtype=np.int64)
    sub_index[sub_valid] = np.arange(sub_rc.shape[0])
    return Geometry(n_sub, sub_valid, act_valid, sub_rc, act_rc, act_index, sub_index)


@dataclasses.dataclass
class Domain:
    I: int
    J: int
    owned_act: np.ndarray        # valid actuator indices owned (row-major)
    obs_sub: np.ndarray          # valid subaperture indices in the observation region

    def rows(self, n_act: int) -> np.ndarray:
        """State rows updated by this domain: owned actuators in both blocks."""
        return np.concatenate([self.owned_act, self.owned_act + n_act])

    def obs_rows(self, n_subv: int) -> np.ndarray:
        """Observation rows: x-slopes then y-slopes of the region's subapertures."""
        return np.concatenate([self.obs_sub, self.obs_sub + n_subv])


def make_domains(geom: Geometry, dom_sub: int, halo: int, offset: int = 0) -> List[Domain]:
    """Domain decomposition of Sect. 2.3 under the reading in the module docstring.

    offset shifts the block grid by that many subapertures along both axes (block I spans
    subaperture rows [b I - offset, b (I + 1) - offset)), giving the second partition of the
    two-partition variant of Sect. 5; offset 0 is the partition described above."""
    n = geom.n_sub
    b = dom_sub
    if not 0 <= offset < b:
        raise ValueError("offset must lie in [0, dom_sub)")
    nb = -(-(n + offset) // b)
    last = (n - 1 + offset) // b          # block of the last subaperture row; row n folds into it
    doms = []
    for I in range(nb):
        for J in range(nb):
            owned = []
            for r in range(n + 1):
                if min((r + offset) // b, last) != I:
                    continue
                for c in range(n + 1):
                    if min((c + offset) // b, last) != J:
                        continue
                    if geom.act_valid[r, c]:
                        owned.append(geom.act_index[r, c])
            if not owned:
                continue
            obs = []
            for r in range(max(0, b * I - offset - halo), min(n, b * (I + 1) - offset + halo)):
                for c in range(max(0, b * J - offset - halo), min(n, b * (J + 1) - offset + halo)):
                    if geom.sub_valid[r, c]:
                        obs.append(geom.sub_index[r, c])
            doms.append(Domain(I, J, np.array(sorted(owned), dtype=np.int64),
                               np.array(sorted(obs), dtype=np.int64)))
    return doms
