"""Named synthetic workloads and the fixed time step of a run.

All workloads are doubly periodic split-square meshes. Where the paper ran on
unstructured meshes of the same domains (Example 1a, Example 2 in Sec. 4) these
structured meshes stand in for them.
"""
from dataclasses import dataclass, field as dfield
import numpy as np

from .mesh import split_square_mesh
from .fields import (taylor_green, double_shear_layer, random_spectrum_velocity,
                     sample_lattice, advected_taylor_green)


@dataclass
class Workload:
    name: str
    N: int
    k: int
    nu: float
    L: float
    ic: str
    steps: int
    seed: int = 0
    alpha: float = 2.0
    cC: float = 0.1
    cB: float = 0.05
    notes: str = ""
    extra: dict = dfield(default_factory=dict)


WORKLOADS = {
    # Taylor-Green on [0,2pi]^2, 8x8 split squares, BDM_2, nu = 1e-2, 100 steps.
    "tgv_n8_k2": Workload("tgv_n8_k2", 8, 2, 1e-2, 2 * np.pi, "tgv", 100),
    # Double shear layer on [0,2pi]^2, 256x256 split squares, BDM_3, nu = 1e-4, 2000 steps.
    "shear_n256_k3": Workload("shear_n256_k3", 256, 3, 1e-4, 2 * np.pi, "shear", 2000),
    # Random-spectrum Euler flow on the unit square, 1024x1024 split squares, BDM_2, nu = 0.
    "spectrum_n1024_k2": Workload("spectrum_n1024_k2", 1024, 2, 0.0, 1.0, "spectrum", 20, seed=0),
    # Gradient workload: 128x128 unit square, BDM_2, nu = 1e-3, 200 steps.
    "adjoint_n128_k2": Workload("adjoint_n128_k2", 128, 2, 1e-3, 1.0, "spectrum", 200, seed=3),
}


def cfl_dt(tri_coords, k, vmax, nu, cC=0.1, cB=0.05):
    """dt = min(cC h/(k^2 vmax), cB h^2/(k^4 nu)), h = max element diameter (paper Sec. 1, eq. (2)).

    The paper leaves cC and cB open ("sufficiently small"); the defaults are the
    values this project uses for every workload.
    """
    X = np.asarray(tri_coords)
    e = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 1], X[:, 0] - X[:, 2]], axis=1)
    h = float(np.sqrt((e ** 2).sum(-1)).max())
    c = cC * h / (k * k * max(vmax, 1e-300))
    if nu > 0:
        c = min(c, cB * h * h / (k ** 4 * nu))
    return c


def make_workload(w, N=None, k=None):
    """Build (tri_vertex_ids, tri_coords, lattice velocity, dt) for a named or given workload."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    N = w.N if N is None else N
    k = w.k if k is None else k
    vid, X = split_square_mesh(N, L=w.L)
    if w.ic == "tgv":
        f = taylor_green(w.L)
    elif w.ic == "shear":
        f = double_shear_layer()
    elif w.ic == "spectrum":
        f = random_spectrum_velocity(w.seed, L=w.L)
    elif w.ic == "advected_tgv":
        f = advected_taylor_green(L=w.L)
    else:
        raise ValueError(w.ic)
    grid = (k * N, w.L) if w.ic == "spectrum" and k * N > 64 else None
    vals = sample_lattice(f, X, k, grid=grid)
    vmax = float(np.sqrt((vals ** 2).sum(-1)).max())
    dt = cfl_dt(X, k, vmax, w.nu, w.cC, w.cB)
    return vid, X, vals, dt
