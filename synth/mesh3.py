"""Periodic tetrahedral meshes of the cube and 3-D initial fields (inputs only, no method arithmetic).

Cube (i, j, l) of an N x N x N grid on [0, L]^3 is cut into the six tetrahedra of its Kuhn
(Freudenthal) triangulation: for each ordering (a, b, c) of the three axes, the tetrahedron
with vertices 0, e_a, e_a + e_b, e_a + e_b + e_c (the cube's main diagonal is shared by all six),
listed so that the orientation is positive. Neighbouring cubes triangulate their common face
the same way, so the mesh is conforming. Element ids 6 (cube) + permutation index, cube =
(l N + j) N + i. The periodic vertex id of grid point (i, j, l) is the point taken mod N;
coordinates are unwrapped.
"""
import itertools

import numpy as np

_PERMS = list(itertools.permutations(range(3)))


def kuhn_cube_mesh(N, L=2.0 * np.pi):
    """Return (tet_vertex_ids [6N^3, 4] int64, tet_coords [6N^3, 4, 3] float64). N >= 2."""
    N = int(N)
    if N < 2:
        raise ValueError("N must be >= 2 (a face's three vertices must have distinct periodic ids)")
    h = L / N
    n = 6 * N ** 3
    vid = np.empty((n, 4), dtype=np.int64)
    X = np.empty((n, 4, 3), dtype=np.float64)
    t = 0
    for l in range(N):
        for j in range(N):
            for i in range(N):
                base = np.array([i, j, l])
                for p in _PERMS:
                    corners = [np.zeros(3, dtype=np.int64)]
                    c = np.zeros(3, dtype=np.int64)
                    for a in p:
                        c = c.copy()
                        c[a] += 1
                        corners.append(c)
                    P = [base + c for c in corners]
                    # positive orientation: det[v1-v0, v2-v0, v3-v0] > 0, else swap v2 and v3
                    d = np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], 1).astype(float))
                    if d < 0:
                        P[2], P[3] = P[3], P[2]
                    for v in range(4):
                        g = P[v]
                        vid[t, v] = (g[0] % N) + N * ((g[1] % N) + N * (g[2] % N))
                        X[t, v] = g * h
                    t += 1
    return vid, X


def n_lattice3(m):
    """Points of the degree-m tetrahedral lattice (1, the centroid, for m = 0)."""
    return (m + 1) * (m + 2) * (m + 3) // 6


def lattice_points3(tet_coords, m):
    """Equispaced points v0 + (i/m)(v1-v0) + (j/m)(v2-v0) + (l/m)(v3-v0), l = 0..m, j = 0..m-l,
    i = 0..m-l-j (i fastest); the centroid for m = 0. Returns [n_tet, n_lattice3(m), 3]."""
    X = np.asarray(tet_coords, dtype=np.float64)
    v0 = X[:, 0]
    if m == 0:
        return X.mean(axis=1)[:, None, :]
    pts = []
    for l in range(m + 1):
        for j in range(m + 1 - l):
            for i in range(m + 1 - l - j):
                pts.append(v0 + (i / m) * (X[:, 1] - v0) + (j / m) * (X[:, 2] - v0) + (l / m) * (X[:, 3] - v0))
    return np.stack(pts, axis=1)


def abc_flow(A=1.0, B=0.7, C=0.4):
    """Arnold-Beltrami-Childress field on [0, 2 pi]^3: curl u = u, divergence free; an exact
    Navier-Stokes solution decaying as exp(-nu t) (the convective term is a gradient)."""
    def f(x, y, z):
        return (A * np.sin(z) + C * np.cos(y), B * np.sin(x) + A * np.cos(z), C * np.sin(y) + B * np.cos(x))
    return f


def sample_lattice3(field, tet_coords, k):
    """field at the degree-k lattice points: [n_tet, n_lattice3(k), 3]."""
    P = lattice_points3(tet_coords, k)
    u = field(P[..., 0], P[..., 1], P[..., 2])
    return np.stack([np.broadcast_to(c, P.shape[:-1]) for c in u], -1).astype(np.float64)
