"""Seeded synthetic workloads shared by the tests, the oracle checks and the bench.

This package only *generates inputs* (charge densities on a mesh, macroparticle
samples, geometry/grid descriptions).  It contains none of the solver's
arithmetic, so that the CPU oracle and the CUDA path share nothing but their
inputs.
"""
from .bunches import (  # noqa: F401
    Geometry,
    Grid,
    mesh_axes,
    gaussian_bunch,
    uniform_ellipsoid,
    random_density,
    workload_fp64_ordinary_16,
    workload_igf_64,
    workload_throughput_128,
    workload_batched_96,
    workload_differentiable_128,
    particle_normals,
)
