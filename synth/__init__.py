"""Seeded synthetic inputs shared by the oracle checks and the CUDA path.

This package holds no arithmetic of the reconstruction method (no wave
propagation, no wavelet transform, no solver): only phantoms, speed maps,
sensor layouts, noise and the workload descriptions built from them.
"""
from .phantoms import blobs, vessels2d, vessel_tree3d, speed_map  # noqa: F401
from .sensors import circle, arc, fibonacci_sphere, line  # noqa: F401
from .workloads import Workload, workload, batched_workloads, add_noise, WORKLOADS  # noqa: F401
