"""Shack-Hartmann sensor emulated on a fine phase grid (Sect. 3 set-up).

The paper generates the true phase on a grid several points per subaperture
finer than the actuator pitch and feeds the control law with sensor slopes.
Here each subaperture spans q x q fine pixels; its slope in a direction is the
phase difference across one pitch, averaged (trapezoid rule) along the two edges
normal to that direction.  Units: radians of phase difference per pitch.  With
q = 1 this collapses to the four-corner difference of the Fried geometry; the
workloads use q = 4, so the filter's model sees the sensor through aliasing just
as a real system does.
"""

from __future__ import annotations

import numpy as np


class FineGridSensor:
    """Slopes and actuator-point phase of an N x N subaperture sensor, q fine samples per pitch."""

    def __init__(self, n_sub: int, q: int = 4):
        if q < 1:
            raise ValueError("q must be >= 1")
        self.n_sub = int(n_sub)
        self.q = int(q)
        self.n_fine = self.n_sub * self.q + 1
        w = np.ones(self.q + 1)
        w[0] = w[-1] = 0.5
        self._w = w / self.q  # trapezoid weights along an edge, summing to 1

    def fine_coords(self, pitch: float):
        """Metric coordinates (x, y) of the fine grid; x runs along columns."""
        t = np.arange(self.n_fine, dtype=np.float64) * (pitch / self.q)
        return np.meshgrid(t, t, indexing="xy")

    def measure(self, phi_fine: np.ndarray):
        """Return (slopes_x, slopes_y, phi_act) for one fine phase map.

        phi_fine: (N q + 1, N q + 1), rows = y, columns = x.
        slopes_x, slopes_y: (N, N) per subaperture (row r, column c), every subaperture.
        phi_act: (N + 1, N + 1) phase at the actuator points (the subaperture corners).
        """
        q, n = self.q, self.n_sub
        f = np.asarray(phi_fine, dtype=np.float64)
        # edge values: column differences across one pitch on every fine row
        left = f[:, 0:n * q:q]          # (Nq+1, N): x = c*q
        right = f[:, q:n * q + 1:q]     # x = (c+1)*q
        dx = right - left               # (Nq+1, N)
        # trapezoid average over the q+1 fine rows of each subaperture
        sx = np.zeros((n, n))
        for i in range(q + 1):
            sx += self._w[i] * dx[i:i + n * q:q, :][:n, :]
        top = f[0:n * q:q, :]
        bot = f[q:n * q + 1:q, :]
        dy = bot - top                  # (N, Nq+1)
        sy = np.zeros((n, n))
        for i in range(q + 1):
            sy += self._w[i] * dy[:, i:i + n * q:q][:, :n]
        phi_act = f[::q, ::q]
        return sx, sy, np.ascontiguousarray(phi_act)
