"""Seeded, synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This package generates *inputs only*: surface meshes (curved P2 triangles on
spheres and spheroids), plane-wave excitations, the seeded multi-body
workload and tabulated material data (the paper's silver optical constants).  It contains none of the solver's arithmetic (no frames, kernels,
quadrature, Morton ordering or linear algebra), so that the CUDA library and
the oracle can both consume the same arrays without sharing any method code.
"""

from .meshes import icosphere_p2, spheroid_p2, mesh_counts
from .excitation import plane_wave, fibonacci_directions, fibonacci_plane_waves
from .configs import WORKLOADS, multibody_mesh, multibody_spec, workload
from .materials import SILVER_JC, eps_silver

__all__ = [
    "icosphere_p2",
    "spheroid_p2",
    "mesh_counts",
    "plane_wave",
    "fibonacci_directions",
    "fibonacci_plane_waves",
    "WORKLOADS",
    "workload",
    "multibody_mesh",
    "multibody_spec",
    "SILVER_JC",
    "eps_silver",
]
