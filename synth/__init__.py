"""Seeded synthetic inputs shared by the oracle-based tests, the CUDA-path tests and the benchmark.

This module holds no arithmetic of the DG method itself. It only produces the
inputs the C-ABI and the oracle both consume:

* split-square periodic triangle meshes (vertex ids of identified vertices plus
  unwrapped corner coordinates), channels open in x, and the kind (wall, inflow,
  outflow) of boundary edges by their position,
* initial velocities sampled at the equispaced element lattice points, and boundary
  data sampled at the equispaced points of each triangle edge,
* the fixed time step a run uses (the convective/viscous CFL bound of the
  paper's introduction, eq. (2), with constants the paper leaves open),
* the named workloads (mesh size, degree, viscosity, initial data, steps),
* periodic Kuhn-split cube meshes of tetrahedra and 3-D fields (the ABC flow) at the
  tetrahedral lattice points.

Random numbers come from numpy's PCG64 generator with explicit seeds.
"""
from .mesh import split_square_mesh, lattice_points, n_lattice, channel_mesh, boundary_kinds_by_x, edge_points
from .fields import (taylor_green, advected_taylor_green, double_shear_layer,
                     random_spectrum_velocity, sample_lattice, sample_edges, constant_field)
from .workloads import Workload, WORKLOADS, cfl_dt, make_workload
from .mesh3 import kuhn_cube_mesh, lattice_points3, n_lattice3, abc_flow, sample_lattice3

__all__ = [
    "split_square_mesh", "lattice_points", "n_lattice", "channel_mesh", "boundary_kinds_by_x", "edge_points",
    "sample_edges", "taylor_green", "advected_taylor_green",
    "double_shear_layer", "random_spectrum_velocity", "sample_lattice", "constant_field",
    "Workload", "WORKLOADS", "cfl_dt", "make_workload",
    "kuhn_cube_mesh", "lattice_points3", "n_lattice3", "abc_flow", "sample_lattice3",
]
