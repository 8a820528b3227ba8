"""Plain FP64 oracle of the divergence-free DG method on tetrahedra, d = 3 (test infrastructure only).

The method of Secs. 2.1-2.4 and 3 is stated for d = 2, 3. This module is its three-dimensional
form on closed (periodic) tetrahedral meshes, written the same plain way as the two-dimensional
oracle and sharing no code with the CUDA path:

* spaces (eq. (4)): broken [P^k]^3 velocities, broken P^{k-1} pressures, P^k multipliers on the
  triangular faces; Bernstein polynomials in barycentric coordinates (element and face);
* L(u) (eq. (6)): the upwind convection form eq. (7) and the SIPG viscous form eq. (18) with
  penalty alpha k^2 / h_F, h_F the larger diameter of the face's two tetrahedra;
* the hybrid-mixed system eq. (12), condensed per element and solved by a sparse LU with one
  multiplier pinned (the constant multiplier is the kernel on a closed mesh), and the
  uncondensed saddle system as an independent route;
* SSP-RK3 (eq. (8)) in the paper's stage form;
* the pressure: (w, lam) of eq. (12) with the functional L(u) alone, mean-free (eq. (4e)).

Faces. A face is parametrised in canonical coordinates (s, t): x = p0 + s (p1 - p0) + t (p2 - p0)
with p0, p1, p2 its vertices in increasing periodic vertex id. Both sides of a face evaluate at
the same canonical points, and the multiplier basis is a function of (s, t). The face rule is the
one choice both this oracle and the CUDA path must share: the upwind flux switches with the sign
of u.n inside a face. It is the collapsed rule with q = ceil((3k+1)/2) Gauss-Legendre points in
a and q Gauss-Jacobi (weight 1 - b) points in b, s = a (1 - b), t = b; its weights sum to 1/2.
"""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import roots_jacobi

RK3_STAGES = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))  # Sec. 2.3, eq. (8)


# ---------------------------------------------------------------- quadrature
def gauss_legendre_01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_jacobi1_01(n):
    """n-point Gauss rule on [0, 1] for the weight (1 - b): exact for (1 - b) p(b), deg p <= 2n - 1."""
    x, w = roots_jacobi(n, 1.0, 0.0)
    return 0.5 * (x + 1.0), 0.25 * w


def face_rule(k):
    """The shared face rule on the reference triangle {s, t >= 0, s + t <= 1} (module docstring)."""
    q = int(math.ceil((3 * k + 1) / 2.0))
    a, wa = gauss_legendre_01(q)
    b, wb = gauss_jacobi1_01(q)
    A, B = np.meshgrid(a, b, indexing="ij")
    WA, WB = np.meshgrid(wa, wb, indexing="ij")
    st = np.stack([(A * (1.0 - B)).ravel(), B.ravel()], axis=1)
    return st, (WA * WB).ravel()


def tet_rule(degree):
    """Collapsed Gauss-Legendre rule on the reference tetrahedron {xi >= 0, sum xi <= 1}:
    xi1 = a (1 - b)(1 - c), xi2 = b (1 - c), xi3 = c, Jacobian (1 - b)(1 - c)^2; n = degree // 2 + 2
    points per direction. Weights sum to 1/6."""
    n = degree // 2 + 2
    a, wa = gauss_legendre_01(n)
    A, B, C = np.meshgrid(a, a, a, indexing="ij")
    WA, WB, WC = np.meshgrid(wa, wa, wa, indexing="ij")
    xi = np.stack([(A * (1 - B) * (1 - C)).ravel(), (B * (1 - C)).ravel(), C.ravel()], axis=1)
    w = (WA * WB * WC * (1 - B) * (1 - C) ** 2).ravel()
    return xi, w


def bernstein3(deg):
    """Barycentric exponents (i0, i1, i2, i3) with sum deg."""
    if deg < 0:
        return []
    out = []
    for l in range(deg + 1):
        for j in range(deg + 1 - l):
            for i in range(deg + 1 - l - j):
                out.append((deg - i - j - l, i, j, l))
    return out


def bernstein2(deg):
    return [(deg - i - j, i, j) for j in range(deg + 1) for i in range(deg + 1 - j)]


def _multinom(e):
    n = sum(e)
    c = math.factorial(n)
    for x in e:
        c //= math.factorial(x)
    return float(c)


# ------------------------------------------------------------------ topology
class Topology3:
    """Tetrahedra, their faces, and the canonical face parametrisation (module docstring).

    Local face e of a tetrahedron is the one opposite its vertex e. Every face must have two sides
    (closed mesh); two element faces are the same face when their periodic vertex ids and the
    face's edge vectors (in canonical order) agree.
    """

    def __init__(self, tet_vertex_ids, tet_coords):
        vid = np.asarray(tet_vertex_ids, dtype=np.int64)
        X = np.asarray(tet_coords, dtype=np.float64)
        n = vid.shape[0]
        if vid.shape != (n, 4) or X.shape != (n, 4, 3):
            raise ValueError("bad mesh arrays")
        self.n_tet, self.vid, self.X = n, vid, X
        J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)   # columns
        self.J = J
        self.detJ = np.linalg.det(J)
        if np.any(self.detJ <= 0):
            raise ValueError("tetrahedra must be positively oriented")
        self.vol = self.detJ / 6.0
        self.diam = np.max([np.linalg.norm(X[:, a] - X[:, b], axis=1) for a in range(4) for b in range(a + 1, 4)],
                           axis=0)
        scale = np.abs(X).max() + 1.0
        tol = 1e-9 * scale
        key_to_face = {}
        sides = []
        for t in range(n):
            for e in range(4):
                loc = [v for v in range(4) if v != e]
                ids = [int(vid[t, v]) for v in loc]
                if len(set(ids)) < 3:
                    raise ValueError("a face needs three distinct periodic vertex ids")
                order = sorted(range(3), key=lambda c: ids[c])
                perm = [loc[c] for c in order]            # local vertex of canonical vertex 0, 1, 2
                d1 = X[t, perm[1]] - X[t, perm[0]]
                d2 = X[t, perm[2]] - X[t, perm[0]]
                key = tuple(ids[c] for c in order) + tuple(int(round(v / tol)) for v in np.concatenate([d1, d2]))
                f = key_to_face.get(key)
                if f is None:
                    f = len(sides)
                    key_to_face[key] = f
                    sides.append([])
                sides[f].append((t, e, perm))
        for f, s in enumerate(sides):
            if len(s) != 2:
                raise ValueError("face %d has %d sides: closed meshes only" % (f, len(s)))
        self.n_face = len(sides)
        self.face_tet = np.array([[s[0][0], s[1][0]] for s in sides], dtype=np.int64)
        self.face_loc = np.array([[s[0][1], s[1][1]] for s in sides], dtype=np.int64)
        self.face_perm = np.array([[s[0][2], s[1][2]] for s in sides], dtype=np.int64)   # [F, 2, 3]
        self.tet_face = np.empty((n, 4), dtype=np.int64)
        for f in range(self.n_face):
            for s in range(2):
                self.tet_face[self.face_tet[f, s], self.face_loc[f, s]] = f
        # outward unit normal and area of every local face
        nrm = np.empty((n, 4, 3))
        area = np.empty((n, 4))
        for e in range(4):
            loc = [v for v in range(4) if v != e]
            c = np.cross(X[:, loc[1]] - X[:, loc[0]], X[:, loc[2]] - X[:, loc[0]])
            a = np.linalg.norm(c, axis=1)
            c = c / a[:, None]
            away = np.einsum("ti,ti->t", c, X[:, loc[0]] - X[:, e])
            nrm[:, e] = np.where((away > 0)[:, None], c, -c)
            area[:, e] = 0.5 * a
        self.normal, self.area = nrm, area
        self.face_area = area[self.face_tet[:, 0], self.face_loc[:, 0]]

    def face_points(self, f, side, st):
        """Physical points [m, q, 3] at canonical face coordinates st [q, 2], in side's own coordinates."""
        t = self.face_tet[f, side]
        p = self.face_perm[f, side]                              # [m, 3]
        P0 = self.X[t, p[:, 0]]
        P1 = self.X[t, p[:, 1]]
        P2 = self.X[t, p[:, 2]]
        return (P0[:, None, :] + st[None, :, 0, None] * (P1 - P0)[:, None, :]
                + st[None, :, 1, None] * (P2 - P0)[:, None, :])


# ------------------------------------------------------------ discretization
class Discretization3:
    """Spaces of Sec. 2.1 (d = 3) and the operators of Secs. 2.2-2.4 and 3 on a closed tetrahedral mesh.
    Coefficients U[t, c*ns + j]: component c of Bernstein polynomial j on tetrahedron t."""

    def __init__(self, tet_vertex_ids, tet_coords, k, nu, alpha=2.0):
        if k < 1:
            raise ValueError("k >= 1")
        self.topo = Topology3(tet_vertex_ids, tet_coords)
        self.k, self.nu, self.alpha = int(k), float(nu), float(alpha)
        self.exps = bernstein3(k)
        self.ns = len(self.exps)
        self.nd = 3 * self.ns
        self.wexps = bernstein3(k - 1)
        self.nw = len(self.wexps)
        self.lexps = bernstein2(k)
        self.nl = len(self.lexps)
        self.vol_xi, self.vol_w = tet_rule(3 * k + 2)
        self.fst, self.fw = face_rule(k)
        self.n_tet, self.n_face = self.topo.n_tet, self.topo.n_face
        self._ops = None

    # ---------------------------------------------------------------- basis
    def _basis(self, exps, tet, P):
        """Bernstein polynomials and their gradients at physical points P [m, q, 3] of tetrahedra tet."""
        T = self.topo
        Ji = np.linalg.inv(T.J[tet])                                    # d xi / d x
        xi = np.einsum("tij,tqj->tqi", Ji, P - T.X[tet, 0][:, None, :])
        lam = [1.0 - xi.sum(-1), xi[..., 0], xi[..., 1], xi[..., 2]]
        glam = [-(Ji[:, 0] + Ji[:, 1] + Ji[:, 2]), Ji[:, 0], Ji[:, 1], Ji[:, 2]]   # [m, 3]
        V, G = [], []
        for e in exps:
            c = _multinom(e)
            v = c * np.ones_like(lam[0])
            for a in range(4):
                v = v * lam[a] ** e[a]
            g = np.zeros(lam[0].shape + (3,))
            for a in range(4):
                if e[a] == 0:
                    continue
                ee = list(e)
                ee[a] -= 1
                term = c * e[a] * np.ones_like(lam[0])
                for b in range(4):
                    term = term * lam[b] ** ee[b]
                g += term[..., None] * glam[a][:, None, :]
            V.append(v)
            G.append(g)
        return np.stack(V, -1), np.stack(G, -2)

    def _face_basis(self, st):
        """Bernstein basis of P^k(F) in canonical face coordinates: [nl, q]."""
        lam = [1.0 - st[:, 0] - st[:, 1], st[:, 0], st[:, 1]]
        out = []
        for e in self.lexps:
            v = _multinom(e) * np.ones(len(st))
            for a in range(3):
                v = v * lam[a] ** e[a]
            out.append(v)
        return np.stack(out, 0)

    def _vol(self, tet):
        T = self.topo
        P = T.X[tet, 0][:, None, :] + np.einsum("tij,qj->tqi", T.J[tet], self.vol_xi)
        W = self.vol_w[None, :] * T.detJ[tet][:, None]
        return P, W

    def _side(self, f, s):
        P = self.topo.face_points(f, np.full(f.shape, s), self.fst)
        tet = self.topo.face_tet[f, s]
        V, G = self._basis(self.exps, tet, P)
        return tet, V, G

    def _penalty(self):
        T = self.topo
        return self.alpha * self.k ** 2 / np.maximum(T.diam[T.face_tet[:, 0]], T.diam[T.face_tet[:, 1]])

    # ------------------------------------------------------------- residual
    def residual(self, U, nu=None):
        """R[t, i] = L(u)(phi_i) = -C_h(u; u, phi_i) - B_h(u, phi_i) for every broken test phi_i
        (eq. (6)): the volume term (u x u - nu grad u) : grad phi, and per face the upwind flux
        (u.n) u^up with u.n the average of both traces, the SIPG consistency, symmetry and penalty
        terms, at the shared face points."""
        nu = self.nu if nu is None else float(nu)
        ns, T = self.ns, self.topo
        U = np.asarray(U, dtype=np.float64).reshape(self.n_tet, 3, ns)
        R = np.zeros((self.n_tet, 3, ns))
        tet = np.arange(self.n_tet)
        P, W = self._vol(tet)
        V, G = self._basis(self.exps, tet, P)
        u = np.einsum("tqj,tcj->tqc", V, U)
        du = np.einsum("tqjd,tcj->tqcd", G, U)
        Flx = u[..., :, None] * u[..., None, :] - nu * du
        R += np.einsum("tq,tqcd,tqjd->tcj", W, Flx, G, optimize=True)
        f = np.arange(self.n_face)
        t0, V0, G0 = self._side(f, 0)
        t1, V1, G1 = self._side(f, 1)
        n0 = T.normal[t0, T.face_loc[:, 0]]
        u0 = np.einsum("fqj,fcj->fqc", V0, U[t0])
        u1 = np.einsum("fqj,fcj->fqc", V1, U[t1])
        du0 = np.einsum("fqjd,fcj->fqcd", G0, U[t0])
        du1 = np.einsum("fqjd,fcj->fqcd", G1, U[t1])
        un = 0.5 * np.einsum("fqc,fc->fq", u0 + u1, n0)
        uup = np.where((un >= 0)[..., None], u0, u1)
        jump = u0 - u1
        dn_avg = 0.5 * np.einsum("fqcd,fd->fqc", du0 + du1, n0)
        sig = self._penalty()[:, None, None]
        wq = 2.0 * T.face_area[:, None] * self.fw[None, :]
        A0 = -un[..., None] * uup + nu * dn_avg - nu * sig * jump
        Bv = 0.5 * nu * jump
        dn0 = np.einsum("fqjd,fd->fqj", G0, n0)
        dn1 = np.einsum("fqjd,fd->fqj", G1, n0)
        c0 = np.einsum("fq,fqc,fqj->fcj", wq, A0, V0) + np.einsum("fq,fqc,fqj->fcj", wq, Bv, dn0)
        c1 = np.einsum("fq,fqc,fqj->fcj", wq, -A0, V1) + np.einsum("fq,fqc,fqj->fcj", wq, Bv, dn1)
        np.add.at(R, t0, c0)
        np.add.at(R, t1, c1)
        return R.reshape(self.n_tet, self.nd)

    # ------------------------------------------------------- local operators
    def _local_ops(self):
        """Per tetrahedron: M (mass of the broken velocity), D (w, div v), C ([mu, v.n] per local face)."""
        T, ns, nd, nw, nl = self.topo, self.ns, self.nd, self.nw, self.nl
        tet = np.arange(self.n_tet)
        P, W = self._vol(tet)
        V, G = self._basis(self.exps, tet, P)
        Ms = np.einsum("tq,tqi,tqj->tij", W, V, V)
        M = np.zeros((self.n_tet, nd, nd))
        for c in range(3):
            M[:, c * ns:(c + 1) * ns, c * ns:(c + 1) * ns] = Ms
        Z, _ = self._basis(self.wexps, tet, P) if nw else (None, None)
        D = np.zeros((self.n_tet, nw, nd))
        for c in range(3):
            D[:, :, c * ns:(c + 1) * ns] = np.einsum("tq,tqm,tqj->tmj", W, Z, G[..., c])
        C = np.zeros((self.n_tet, 4 * nl, nd))
        dof = np.empty((self.n_tet, 4 * nl), dtype=np.int64)
        mu = self._face_basis(self.fst)                                  # [nl, q]
        for e in range(4):
            f = T.tet_face[:, e]
            side = np.where((T.face_tet[f, 0] == tet) & (T.face_loc[f, 0] == e), 0, 1)
            Pf = T.face_points(f, side, self.fst)
            Vf, _ = self._basis(self.exps, tet, Pf)
            wq = 2.0 * T.area[:, e][:, None] * self.fw[None, :]
            n = T.normal[:, e]
            for c in range(3):
                C[:, e * nl:(e + 1) * nl, c * ns:(c + 1) * ns] = np.einsum(
                    "tq,mq,tqj->tmj", wq * n[:, c][:, None], mu, Vf)
            dof[:, e * nl:(e + 1) * nl] = f[:, None] * nl + np.arange(nl)[None, :]
        return M, D, C, dof

    def prepare(self):
        """Static condensation of eq. (12) per tetrahedron and the sparse LU of S, once (Sec. 4)."""
        if self._ops is not None:
            return self._ops
        n, nd, nw, nl = self.n_tet, self.nd, self.nw, self.nl
        M, D, C, dof = self._local_ops()
        A = np.zeros((n, nd + nw, nd + nw))
        A[:, :nd, :nd] = M
        A[:, :nd, nd:] = -np.transpose(D, (0, 2, 1))
        A[:, nd:, :nd] = -D
        Ai = np.linalg.inv(A)
        Pm, Wm = Ai[:, :nd, :nd], Ai[:, nd:, :nd]
        CP = np.einsum("tij,tjk->tik", C, Pm)
        Sloc = np.einsum("tik,tjk->tij", CP, C)
        nlam = self.n_face * nl
        rows = np.repeat(dof, 4 * nl, axis=1).ravel()
        cols = np.tile(dof, (1, 4 * nl)).ravel()
        S = sp.csc_matrix((Sloc.ravel(), (rows, cols)), shape=(nlam, nlam))
        act = np.arange(1, nlam)          # the constant multiplier is pinned through dof 0
        lu = spla.splu(S[act][:, act].tocsc())
        self._ops = dict(M=M, D=D, C=C, P=Pm, W=Wm, CP=CP, dof=dof, S=S, lu=lu, act=act)
        return self._ops

    def solve_condensed(self, F):
        """Hybrid-mixed solve of eq. (12) for the functional F (Theorem 2): (u, w, lam)."""
        o = self.prepare()
        F = np.asarray(F).reshape(self.n_tet, self.nd)
        g = np.bincount(o["dof"].ravel(), weights=np.einsum("tij,tj->ti", o["CP"], F).ravel(),
                        minlength=self.n_face * self.nl)
        lam = np.zeros_like(g)
        lam[o["act"]] = o["lu"].solve(g[o["act"]])
        r = F - np.einsum("tij,ti->tj", o["C"], lam[o["dof"]])
        return np.einsum("tij,tj->ti", o["P"], r), np.einsum("tij,tj->ti", o["W"], r), lam

    def solve_full(self, F):
        """The uncondensed saddle system of eq. (12) (an independent route, small meshes)."""
        o = self.prepare()
        n, nd, nw, nl = self.n_tet, self.nd, self.nw, self.nl
        nU, nW, nL = n * nd, n * nw, self.n_face * nl
        blocks = []
        for t in range(n):
            blocks.append(o["M"][t])
        Mg = sp.block_diag(blocks)
        Dg = sp.block_diag([o["D"][t] for t in range(n)]) if nw else sp.csr_matrix((0, nU))
        rows, cols, vals = [], [], []
        for t in range(n):
            for i in range(4 * nl):
                for j in range(nd):
                    rows.append(o["dof"][t, i])
                    cols.append(t * nd + j)
                    vals.append(o["C"][t, i, j])
        Cg = sp.csr_matrix((vals, (rows, cols)), shape=(nL, nU))
        K = sp.bmat([[Mg, -Dg.T, -Cg.T], [-Dg, None, None], [-Cg, None, None]]).tocsc()
        rhs = np.zeros(nU + nW + nL)
        rhs[:nU] = np.asarray(F).ravel()
        keep = np.ones(nU + nW + nL, dtype=bool)
        keep[nU + nW] = False          # pin the constant multiplier
        sol = np.zeros_like(rhs)
        sol[keep] = spla.spsolve(K[keep][:, keep].tocsc(), rhs[keep])
        return sol[:nU].reshape(n, nd)

    # --------------------------------------------------------------- steps
    def apply_mass(self, U):
        o = self.prepare()
        return np.einsum("tij,tj->ti", o["M"], np.asarray(U).reshape(self.n_tet, self.nd))

    def riesz(self, R):
        o = self.prepare()
        return np.linalg.solve(o["M"], np.asarray(R).reshape(self.n_tet, self.nd)[..., None])[..., 0]

    def project(self, U):
        """L2 projection onto V_h^{k,-1}: the solve with F = (u, .)."""
        return self.solve_condensed(self.apply_mass(U))[0]

    def stage(self, Un, Up, a, b, dt):
        """M u_new = a M u^n + b [M u' + dt L(u')] (eq. (8))."""
        F = a * self.apply_mass(Un) + b * (self.apply_mass(Up) + dt * self.residual(Up))
        return self.solve_condensed(F)[0]

    def rk3_step(self, U, dt, nsteps=1):
        for _ in range(int(nsteps)):
            U1 = self.stage(U, U, *RK3_STAGES[0], dt)
            U2 = self.stage(U, U1, *RK3_STAGES[1], dt)
            U = self.stage(U, U2, *RK3_STAGES[2], dt)
        return U

    def pressure(self, U):
        """(w, lam) of eq. (12) with the functional L(u) alone (Theorem 2, Remark 2): w ~ p in the
        elements and lam ~ p on the faces, both shifted by one constant so that the integral of w
        is zero (L^2_0, eq. (4e)). The Bernstein bases are partitions of unity, so the constant
        is the same shift of every coefficient."""
        _, w, lam = self.solve_condensed(self.residual(U))
        tet = np.arange(self.n_tet)
        P, W = self._vol(tet)
        Z, _ = self._basis(self.wexps, tet, P)
        c = np.einsum("tq,tqm,tm->", W, Z, w) / W.sum()
        return w - c, lam - c

    def pressure_lattice(self, w, lam):
        """Element pressure at the degree-(k-1) lattice points of each tetrahedron [n_tet, n_lat(k-1)]
        (the centroid for k = 1), face pressure at the degree-k lattice points of each face in
        canonical coordinates, (s, t) = (i/k, j/k), j = 0..k, i = 0..k-j (i fastest) [n_face, nl]."""
        T = self.topo
        xi = self._lattice_xi(self.k - 1)
        P = T.X[:, 0][:, None, :] + np.einsum("tij,qj->tqi", T.J, xi)
        Z, _ = self._basis(self.wexps, np.arange(self.n_tet), P)
        pe = np.einsum("tqm,tm->tq", Z, np.asarray(w).reshape(self.n_tet, self.nw))
        k = self.k
        st = np.array([(i / k, j / k) for j in range(k + 1) for i in range(k + 1 - j)])
        pf = np.asarray(lam).reshape(self.n_face, self.nl) @ self._face_basis(st)
        return pe, pf

    # ------------------------------------------------------------- lattice
    def _lattice_xi(self, m):
        if m == 0:
            return np.array([[0.25, 0.25, 0.25]])
        return np.array([(i / m, j / m, l / m) for l in range(m + 1) for j in range(m + 1 - l)
                         for i in range(m + 1 - l - j)])

    def _lattice_V(self, m):
        T = self.topo
        xi = self._lattice_xi(m)
        P = T.X[:, 0][:, None, :] + np.einsum("tij,qj->tqi", T.J, xi)
        V, _ = self._basis(self.exps, np.arange(self.n_tet), P)
        return V                                                          # [t, q, j]

    def from_lattice(self, vals):
        """Coefficients of the broken field interpolating lattice values [n_tet, n_lat(k), 3]."""
        V = self._lattice_V(self.k)
        vals = np.asarray(vals, dtype=np.float64)
        c = np.linalg.solve(V, vals)                                      # [t, j, 3]
        return np.transpose(c, (0, 2, 1)).reshape(self.n_tet, self.nd)

    def to_lattice(self, U):
        V = self._lattice_V(self.k)
        U = np.asarray(U).reshape(self.n_tet, 3, self.ns)
        return np.einsum("tqj,tcj->tqc", V, U)

    # ---------------------------------------------------------- diagnostics
    def energy(self, U):
        return float((np.asarray(U) * self.apply_mass(U)).sum())

    def diagnostics(self, U):
        """Energy ||u||^2, max |div u| at volume points, max |[u.n]| at the face points."""
        T, ns = self.topo, self.ns
        U = np.asarray(U).reshape(self.n_tet, 3, ns)
        tet = np.arange(self.n_tet)
        P, _ = self._vol(tet)
        _, G = self._basis(self.exps, tet, P)
        du = np.einsum("tqjd,tcj->tqcd", G, U)
        div = np.abs(du[..., 0, 0] + du[..., 1, 1] + du[..., 2, 2]).max()
        f = np.arange(self.n_face)
        t0, V0, _ = self._side(f, 0)
        t1, V1, _ = self._side(f, 1)
        n0 = T.normal[t0, T.face_loc[:, 0]]
        jmp = np.abs(np.einsum("fqc,fc->fq", np.einsum("fqj,fcj->fqc", V0, U[t0])
                               - np.einsum("fqj,fcj->fqc", V1, U[t1]), n0)).max()
        return dict(energy=self.energy(U.reshape(self.n_tet, -1)), max_div=float(div), max_jump=float(jmp))

    def upwind_dissipation(self, U):
        """(1/2) sum_F int_F |u.n| |u^+ - u^-|^2 at the face points (energy identity of Sec. 2.2)."""
        T = self.topo
        U = np.asarray(U).reshape(self.n_tet, 3, self.ns)
        f = np.arange(self.n_face)
        t0, V0, _ = self._side(f, 0)
        t1, V1, _ = self._side(f, 1)
        n0 = T.normal[t0, T.face_loc[:, 0]]
        u0 = np.einsum("fqj,fcj->fqc", V0, U[t0])
        u1 = np.einsum("fqj,fcj->fqc", V1, U[t1])
        un = 0.5 * np.einsum("fqc,fc->fq", u0 + u1, n0)
        wq = 2.0 * T.face_area[:, None] * self.fw[None, :]
        return float(0.5 * (wq * np.abs(un) * ((u0 - u1) ** 2).sum(-1)).sum())

    def l2_error(self, U, field):
        """||u_h - field|| with the oracle's volume rule."""
        tet = np.arange(self.n_tet)
        P, W = self._vol(tet)
        V, _ = self._basis(self.exps, tet, P)
        u = np.einsum("tqj,tcj->tqc", V, np.asarray(U).reshape(self.n_tet, 3, self.ns))
        ex = np.stack(field(P[..., 0], P[..., 1], P[..., 2]), -1)
        return float(np.sqrt((W[..., None] * (u - ex) ** 2).sum()))
