"""Seeded synthetic inputs shared by the oracle-based tests, the CUDA-path tests and the benchmark.

This module holds no arithmetic of the DG method itself. It only produces the
inputs the C-ABI and the oracle both consume:

* split-square periodic triangle meshes (vertex ids of identified vertices plus
  unwrapped corner coordinates),
* initial velocities sampled at the equispaced element lattice points,
* the fixed time step a run uses (the convective/viscous CFL bound of the
  paper's introduction, eq. (2), with constants the paper leaves open),
* the named workloads (mesh size, degree, viscosity, initial data, steps).

Random numbers come from numpy's PCG64 generator with explicit seeds.
"""
from .mesh import split_square_mesh, lattice_points, n_lattice
from .fields import (taylor_green, advected_taylor_green, double_shear_layer,
                     random_spectrum_velocity, sample_lattice, constant_field)
from .workloads import Workload, WORKLOADS, cfl_dt, make_workload

__all__ = [
    "split_square_mesh", "lattice_points", "n_lattice", "taylor_green", "advected_taylor_green",
    "double_shear_layer", "random_spectrum_velocity", "sample_lattice", "constant_field",
    "Workload", "WORKLOADS", "cfl_dt", "make_workload",
]
