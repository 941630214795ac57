"""Seeded synthetic AO inputs shared by the GPU path's callers and the oracle's tests.

This package generates what the paper's simulations feed to the control law
(Sect. 3): von Karman turbulence under Taylor frozen flow, a Shack-Hartmann
sensor emulated on a fine phase grid, white slope noise, and the von Karman
phase covariance used to build the process-noise model.  It holds none of the
filter's arithmetic (no state-space model, no Fried operator, no analysis):
both the CUDA path and the FP64 oracle consume its outputs unchanged.
"""

from .turbulence import (VKScreen, vk_phase_covariance, vk_structure_function_kolmogorov,
                         actuator_covariance_lag_table)
from .wfs import FineGridSensor
from .workloads import Workload, WORKLOADS, workload, serving_mix, TruthStream, compressed_frames, yule_walker_ar2

__all__ = [
    "VKScreen", "vk_phase_covariance", "vk_structure_function_kolmogorov",
    "actuator_covariance_lag_table", "FineGridSensor", "Workload", "WORKLOADS", "workload",
    "serving_mix", "TruthStream", "compressed_frames", "yule_walker_ar2",
]
