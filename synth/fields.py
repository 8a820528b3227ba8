"""Initial velocity fields sampled at the element lattice points.

Each field is a callable (x, y) -> (u1, u2) on numpy arrays. The random-spectrum
field is represented by its Fourier coefficients so it can be evaluated exactly
either by a direct trigonometric sum or, when the sample points lie on a uniform
grid, by an inverse FFT of the same coefficients.
"""
import numpy as np

from .mesh import lattice_points, edge_points


def taylor_green(L=2.0 * np.pi):
    """u = (sin kx cos ky, -cos kx sin ky) with k = 2*pi/L (divergence free, periodic on [0,L]^2)."""
    kap = 2.0 * np.pi / L

    def f(x, y):
        return np.sin(kap * x) * np.cos(kap * y), -np.cos(kap * x) * np.sin(kap * y)
    f.kappa = kap
    return f


def advected_taylor_green(U=(1.0, 0.0), L=2.0 * np.pi, t=0.0, nu=0.0):
    """Galilean translate of the Taylor-Green vortex: U + TG(x - U t) * exp(-2 nu k^2 t)."""
    tg = taylor_green(L)
    kap = tg.kappa
    damp = np.exp(-2.0 * nu * kap * kap * t)

    def f(x, y):
        a, b = tg(x - U[0] * t, y - U[1] * t)
        return U[0] + damp * a, U[1] + damp * b
    return f


def double_shear_layer(rho=np.pi / 15.0, delta=0.05):
    """Double shear layer on [0, 2pi]^2 (Example 2 of the paper, Sec. 4)."""
    def f(x, y):
        u1 = np.where(y <= np.pi, np.tanh((y - np.pi / 2.0) / rho), np.tanh((1.5 * np.pi - y) / rho))
        u2 = delta * np.sin(x)
        return u1, u2
    return f


def constant_field(c=(0.3, -0.7)):
    def f(x, y):
        return np.full_like(x, c[0]), np.full_like(x, c[1])
    return f


class RandomSpectrum:
    """Divergence-free field u = (d psi/dy, -d psi/dx) on the periodic square [0,L]^2.

    psi = sum over half-plane integer vectors m, 0 < |m| <= kmax, of
    |m|^-3 [a_m cos(2 pi m.x/L) + b_m sin(2 pi m.x/L)], a_m, b_m ~ N(0,1) from PCG64(seed),
    then u is scaled to unit RMS over the square (computed from the coefficients).
    """

    def __init__(self, seed, kmax=32, L=1.0, slope=3.0):
        self.L = float(L)
        modes = []
        for mx in range(0, kmax + 1):
            for my in range(-kmax, kmax + 1):
                if mx == 0 and my <= 0:
                    continue
                if mx * mx + my * my <= kmax * kmax:
                    modes.append((mx, my))
        self.modes = np.array(modes, dtype=np.int64)
        rng = np.random.Generator(np.random.PCG64(seed))
        a = rng.standard_normal(len(modes))
        b = rng.standard_normal(len(modes))
        mag = np.sqrt((self.modes ** 2).sum(axis=1).astype(np.float64))
        sig = mag ** (-slope)
        # psi = Re[ c_m exp(2 pi i m.x / L) ], c_m = sig (a - i b)
        c = sig * (a - 1j * b)
        w = 2.0 * np.pi / self.L
        self.c1 = c * (1j * w * self.modes[:, 1])      # d/dy
        self.c2 = -c * (1j * w * self.modes[:, 0])     # -d/dx
        ms = 0.5 * (np.abs(self.c1) ** 2 + np.abs(self.c2) ** 2).sum()
        self.scale = 1.0 / np.sqrt(ms)

    def __call__(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        shp = x.shape
        xf, yf = x.reshape(-1), y.reshape(-1)
        out1 = np.empty(xf.size)
        out2 = np.empty(xf.size)
        w = 2.0 * np.pi / self.L
        step = 4096
        for s in range(0, xf.size, step):
            ph = w * (np.outer(xf[s:s + step], self.modes[:, 0]) + np.outer(yf[s:s + step], self.modes[:, 1]))
            e = np.exp(1j * ph)
            out1[s:s + step] = (e @ self.c1).real
            out2[s:s + step] = (e @ self.c2).real
        return (self.scale * out1).reshape(shp), (self.scale * out2).reshape(shp)

    def on_grid(self, M):
        """Exact values on the M x M grid x = p L / M (arrays indexed [px, py])."""
        kmax = int(np.abs(self.modes).max())
        if M <= 2 * kmax:
            raise ValueError("grid too coarse for the spectrum")
        out = []
        for c in (self.c1, self.c2):
            A = np.zeros((M, M), dtype=np.complex128)
            np.add.at(A, (self.modes[:, 0] % M, self.modes[:, 1] % M), c)
            out.append(self.scale * (np.fft.ifft2(A) * (M * M)).real)
        return out


def random_spectrum_velocity(seed, kmax=32, L=1.0):
    return RandomSpectrum(seed, kmax=kmax, L=L)


def sample_lattice(field, tri_coords, k, grid=None):
    """Velocity values at the degree-k lattice points: [n_tri, n_lattice(k), 2] float64.

    ``grid`` = (M, L) asks for evaluation through ``field.on_grid(M)`` when every
    lattice point sits on the grid x = p L / M (true for split-square meshes with
    M = k N); points are wrapped periodically into [0, L).
    """
    P = lattice_points(tri_coords, k)
    if grid is not None and hasattr(field, "on_grid"):
        M, L = grid
        g = P / (L / M)
        gi = np.rint(g)
        if np.abs(g - gi).max() < 1e-6:
            gi = gi.astype(np.int64) % M
            u1, u2 = field.on_grid(M)
            vals = np.empty(P.shape)
            vals[..., 0] = u1[gi[..., 0], gi[..., 1]]
            vals[..., 1] = u2[gi[..., 0], gi[..., 1]]
            return vals
    u1, u2 = field(P[..., 0], P[..., 1])
    return np.stack([u1, u2], axis=-1)


def sample_edges(field, tri_coords, k):
    """field at the k+1 equispaced points of every triangle edge (counter-clockwise direction):
    [n_tri, 3, k+1, 2], the boundary-data format of the inflow condition."""
    P = edge_points(tri_coords, k)
    a, b = field(P[..., 0], P[..., 1])
    return np.stack([np.broadcast_to(a, P.shape[:-1]), np.broadcast_to(b, P.shape[:-1])], -1).astype(np.float64)
