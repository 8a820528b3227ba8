"""Split-square periodic triangulations and the element lattice convention.

Square (i, j) of an N x N grid on [x0, x0+L]^2 is cut along its SW-NE diagonal:
lower triangle (i,j),(i+1,j),(i+1,j+1) and upper triangle (i,j),(i+1,j+1),(i,j+1),
both counter-clockwise; element ids 2*(j*N+i) + {0, 1}. Periodic vertex id of
grid point (i, j) is (i mod N) + N*(j mod N). Coordinates are unwrapped, so an
element next to the periodic seam keeps its true shape.
"""
import numpy as np


def split_square_mesh(N, L=2.0 * np.pi, origin=(0.0, 0.0), periodic=True):
    """Return (tri_vertex_ids [2N^2,3] int64, tri_coords [2N^2,3,2] float64).

    periodic: vertices on opposite sides of the square are identified (a torus); otherwise
    every vertex has its own id and the square's edges are walls (boundary facets).
    """
    N = int(N)
    if N < 1:
        raise ValueError("N must be >= 1")
    h = L / N
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")  # j rows, i columns
    i = i.reshape(-1)
    j = j.reshape(-1)
    corners_lo = [(0, 0), (1, 0), (1, 1)]
    corners_up = [(0, 0), (1, 1), (0, 1)]
    n_tri = 2 * N * N
    vid = np.empty((n_tri, 3), dtype=np.int64)
    X = np.empty((n_tri, 3, 2), dtype=np.float64)
    cell = j * N + i
    for which, corners in enumerate((corners_lo, corners_up)):
        t = 2 * cell + which
        for c, (di, dj) in enumerate(corners):
            if periodic:
                vid[t, c] = ((i + di) % N) + N * ((j + dj) % N)
            else:
                vid[t, c] = (i + di) + (N + 1) * (j + dj)
            X[t, c, 0] = origin[0] + (i + di) * h
            X[t, c, 1] = origin[1] + (j + dj) * h
    return vid, X


def n_lattice(m):
    """Number of points of the degree-m element lattice (1 point, the centroid, for m = 0)."""
    return (m + 1) * (m + 2) // 2


def lattice_points(tri_coords, m):
    """Equispaced lattice points v0 + (i/m)(v1-v0) + (j/m)(v2-v0), j = 0..m, i = 0..m-j.

    For m = 0 the single point is the centroid. Returns [n_tri, n_lattice(m), 2].
    """
    X = np.asarray(tri_coords, dtype=np.float64)
    v0, v1, v2 = X[:, 0, :], X[:, 1, :], X[:, 2, :]
    if m == 0:
        return ((v0 + v1 + v2) / 3.0)[:, None, :]
    pts = []
    for jj in range(m + 1):
        for ii in range(m + 1 - jj):
            pts.append(v0 + (ii / m) * (v1 - v0) + (jj / m) * (v2 - v0))
    return np.stack(pts, axis=1)


def channel_mesh(Nx, Ny, Lx, Ly, periodic_y=True, origin=(0.0, 0.0)):
    """Split-square triangulation of the rectangle [x0, x0+Lx] x [y0, y0+Ly] with Nx x Ny squares.

    periodic_y: the bottom and top edges are identified (a periodic channel), so the only
    boundary edges are x = x0 and x = x0 + Lx; otherwise every edge of the rectangle is a
    boundary edge. Element ids 2*(j*Nx+i) + {0, 1} as in split_square_mesh.
    """
    Nx, Ny = int(Nx), int(Ny)
    hx, hy = Lx / Nx, Ly / Ny
    i, j = np.meshgrid(np.arange(Nx), np.arange(Ny), indexing="xy")
    i = i.reshape(-1)
    j = j.reshape(-1)
    corners_lo = [(0, 0), (1, 0), (1, 1)]
    corners_up = [(0, 0), (1, 1), (0, 1)]
    n_tri = 2 * Nx * Ny
    vid = np.empty((n_tri, 3), dtype=np.int64)
    X = np.empty((n_tri, 3, 2), dtype=np.float64)
    cell = j * Nx + i
    for which, corners in enumerate((corners_lo, corners_up)):
        t = 2 * cell + which
        for c, (di, dj) in enumerate(corners):
            jj = (j + dj) % Ny if periodic_y else (j + dj)
            vid[t, c] = (i + di) + (Nx + 1) * jj
            X[t, c, 0] = origin[0] + (i + di) * hx
            X[t, c, 1] = origin[1] + (j + dj) * hy
    return vid, X


def boundary_kinds_by_x(tri_coords, x_in, x_out, tol=1e-9):
    """Kind of every triangle edge [n_tri, 3] (int8): 1 on the line x = x_in (inflow), 2 on
    x = x_out (outflow), 0 elsewhere (walls, or interior edges, whose kind is not used). Edge e
    of a triangle is the one opposite its vertex e."""
    X = np.asarray(tri_coords, dtype=np.float64)
    out = np.zeros(X.shape[:2], dtype=np.int8)
    for e in range(3):
        a, b = X[:, (e + 1) % 3], X[:, (e + 2) % 3]
        on_in = (np.abs(a[:, 0] - x_in) < tol) & (np.abs(b[:, 0] - x_in) < tol)
        on_out = (np.abs(a[:, 0] - x_out) < tol) & (np.abs(b[:, 0] - x_out) < tol)
        out[on_in, e] = 1
        out[on_out, e] = 2
    return out


def edge_points(tri_coords, k):
    """The k+1 equispaced points of every triangle edge in the triangle's counter-clockwise
    direction: edge e from vertex (e+1)%3 to vertex (e+2)%3. Returns [n_tri, 3, k+1, 2]."""
    X = np.asarray(tri_coords, dtype=np.float64)
    t = np.arange(k + 1) / k
    pts = np.empty((X.shape[0], 3, k + 1, 2))
    for e in range(3):
        a, b = X[:, (e + 1) % 3], X[:, (e + 2) % 3]
        pts[:, e] = a[:, None, :] + t[None, :, None] * (b - a)[:, None, :]
    return pts
