"""Plain FP64 oracle of the divergence-free DG method (test infrastructure only).

Every function states the passage of the paper it follows. Coefficients of a
broken vector field are stored as U[t, c*ns + j] for component c of the scalar
Bernstein polynomial j on triangle t. Bernstein polynomials in barycentric
coordinates are used because they are far better conditioned than monomials
(mass-matrix condition ~56 at k = 3) and unrelated to the CUDA path's basis.
"""
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import Topology, INFLOW, OUTFLOW
from .quadrature import triangle_rule, facet_rule

RK3_STAGES = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))  # Sec. 2.3, eq. (8)


def bernstein_indices(deg):
    """Barycentric exponents (i, j, l), i + j + l = deg, of the degree-deg Bernstein basis."""
    if deg < 0:
        return []
    return [(deg - j - l, j, l) for l in range(deg + 1) for j in range(deg + 1 - l)]


def _binom(n, m):
    return math.comb(n, m)


class Discretization:
    """Spaces of Sec. 2.1 (eq. (4)) and the operators of Secs. 2.2-2.4 and 3 on one mesh."""

    def __init__(self, tri_vertex_ids, tri_coords, k, nu, alpha=2.0, chunk=4096, boundary=None, inflow=None):
        """boundary: kind per triangle edge [n_tri, 3] (0 wall, 1 inflow, 2 outflow; used on boundary
        edges only), the boundary parts of Sec. 2.5, eq. (be); inflow: the inflow velocity u_in at the
        k+1 equispaced points of every edge in the triangle's counter-clockwise direction
        [n_tri, 3, k+1, 2] (read on inflow edges only)."""
        if k < 1:
            raise ValueError("k >= 1")
        self.topo = Topology(tri_vertex_ids, tri_coords, boundary)
        self.k = int(k)
        self.nu = float(nu)
        self.alpha = float(alpha)
        self.exps = bernstein_indices(k)
        self.ns = len(self.exps)
        self.nd = 2 * self.ns                       # broken [P^k]^2 per triangle
        self.wexps = bernstein_indices(k - 1)
        self.nw = len(self.wexps)                   # broken P^{k-1} per triangle
        self.nl = k + 1                             # P^k per facet
        self.vol_xi, self.vol_w = triangle_rule(3 * k + 2)
        self.ft, self.fw = facet_rule(k)
        self.chunk = int(chunk)
        self.n_tri = self.topo.n_tri
        self.n_facet = self.topo.n_facet
        self._ops = None
        self._set_inflow(inflow)

    # ------------------------------------------------------------------ basis
    def _basis(self, exps, tri, P):
        """Bernstein polynomials n!/(i!j!l!) l0^i l1^j l2^l and their x/y gradients at points P [m, q, 2]."""
        T = self.topo
        Jt = T.J[tri]
        det = T.detJ[tri]
        Ji = np.empty_like(Jt)                                   # inverse of [v1-v0, v2-v0]
        Ji[:, 0, 0] = Jt[:, 1, 1] / det
        Ji[:, 0, 1] = -Jt[:, 0, 1] / det
        Ji[:, 1, 0] = -Jt[:, 1, 0] / det
        Ji[:, 1, 1] = Jt[:, 0, 0] / det
        xi = np.einsum("tij,tqj->tqi", Ji, P - T.X[tri, 0][:, None, :])
        lam = [1.0 - xi[..., 0] - xi[..., 1], xi[..., 0], xi[..., 1]]
        glam = [-(Ji[:, 0, :] + Ji[:, 1, :]), Ji[:, 0, :], Ji[:, 1, :]]  # [m, 2] each
        V, G = [], []
        for (i, j, l) in exps:
            n = i + j + l
            c = math.factorial(n) / (math.factorial(i) * math.factorial(j) * math.factorial(l))
            pw = (i, j, l)
            V.append(c * lam[0] ** i * lam[1] ** j * lam[2] ** l)
            g = np.zeros(lam[0].shape + (2,))
            for a in range(3):
                if pw[a] == 0:
                    continue
                e = list(pw)
                e[a] -= 1
                term = c * pw[a] * lam[0] ** e[0] * lam[1] ** e[1] * lam[2] ** e[2]
                g += term[..., None] * glam[a][:, None, :]
            G.append(g)
        return np.stack(V, -1), np.stack(G, -2)

    def _vol(self, tri, rule=None):
        """Physical volume points [m, q, 2] and weights [m, q] on triangles tri."""
        T = self.topo
        xi, w = (self.vol_xi, self.vol_w) if rule is None else rule
        P = T.X[tri, 0][:, None, :] + np.einsum("tij,qj->tqi", T.J[tri], xi)
        W = w[None, :] * T.detJ[tri][:, None]
        return P, W

    def _chunks(self, n):
        for s in range(0, n, self.chunk):
            yield np.arange(s, min(n, s + self.chunk))

    def _interior_chunks(self):
        """Interior facets in chunks. A wall (boundary facet) adds no term to L(u): u.n = 0
        there for every u of the space, so the convective flux of eq. (7) vanishes, and the
        SIPG form eq. (18) sums over interior facets only (free slip, Sec. 3)."""
        ii = self.topo.interior
        for s in range(0, len(ii), self.chunk):
            yield ii[s:s + self.chunk]

    def _penalty(self):
        """alpha k^2 / h_F per facet, h_F the larger diameter of the facet's triangles (eq. (18))."""
        T = self.topo
        t1 = np.where(T.boundary, T.facet_tri[:, 0], T.facet_tri[:, 1])
        return self.alpha * self.k ** 2 / np.maximum(T.diam[T.facet_tri[:, 0]], T.diam[t1])

    def _facet_side(self, f, s):
        P = self.topo.facet_points(f, np.full(f.shape, s), self.ft)
        tri = self.topo.facet_tri[f, s]
        V, G = self._basis(self.exps, tri, P)
        return tri, V, G

    # ------------------------------------------------- inflow / outflow (Sec. 2.5)
    def _set_inflow(self, inflow):
        """u_in at the facet Gauss points of every inflow facet (canonical parameter) and the
        moments d_F[m] = <mu_m, u_in.n>_F of its normal component (n outward from the domain):
        the inhomogeneous constraint u.n = u_in.n on Gamma_in of eq. (be), tested against the
        multiplier space P^k(F) as the normal-continuity rows of eq. (12)."""
        T = self.topo
        nq = len(self.ft)
        self.inflow_q = np.zeros((self.n_facet, nq, 2))
        self.inflow_d = np.zeros(self.n_facet * self.nl)
        f = T.inflow
        if len(f) == 0:
            return
        if inflow is None:
            raise ValueError("inflow facets need inflow data")
        vals = np.asarray(inflow, dtype=np.float64).reshape(self.n_tri, 3, self.k + 1, 2)
        t0, e0, o0 = T.facet_tri[f, 0], T.facet_loc[f, 0], T.facet_orient[f, 0]
        v = vals[t0, e0]                                         # element direction
        v = np.where((o0 > 0)[:, None, None], v, v[:, ::-1, :])   # canonical direction
        nodes = np.arange(self.k + 1) / self.k
        Lq = np.stack([np.prod([(self.ft - nodes[j]) / (nodes[i] - nodes[j])
                                for j in range(self.k + 1) if j != i], axis=0) for i in range(self.k + 1)], 0)
        uq = np.einsum("iq,fic->fqc", Lq, v)
        self.inflow_q[f] = uq
        n0 = T.normal[t0, e0]
        wq = self.fw[None, :] * T.facet_len[f][:, None]
        mu = self._facet_basis(self.ft)
        d = np.einsum("fq,mq,fq->fm", wq, mu, np.einsum("fqc,fc->fq", uq, n0))
        self.inflow_d.reshape(self.n_facet, self.nl)[f] = d

    def _boundary_flux(self, U, R):
        """Convective terms of eq. (7) on inflow and outflow facets (Sec. 2.5): the flux
        (u.n) u^up with u.n the average of the interior trace and the exterior state, and the
        upwind value taken from the side u.n leaves. The exterior state is u_in on an inflow
        facet and the interior trace on an outflow facet. Walls add nothing (u.n = 0), and the
        viscous form has no boundary terms: natural conditions on every boundary facet."""
        T = self.topo
        f = np.concatenate([T.inflow, T.outflow])
        if len(f) == 0:
            return
        t0, V0, _ = self._facet_side(f, 0)
        e0 = T.facet_loc[f, 0]
        n0 = T.normal[t0, e0]
        u0 = np.einsum("fqj,fcj->fqc", V0, U[t0])
        uext = np.where((T.facet_kind[f] == INFLOW)[:, None, None], self.inflow_q[f], u0)
        un = 0.5 * np.einsum("fqc,fc->fq", u0 + uext, n0)
        uup = np.where((un >= 0)[..., None], u0, uext)
        wq = self.fw[None, :] * T.facet_len[f][:, None]
        c0 = np.einsum("fq,fqc,fqj->fcj", wq, -un[..., None] * uup, V0)
        np.add.at(R, t0, c0)

    # --------------------------------------------------------------- residual
    def residual(self, U, nu=None):
        """R[t, i] = L(u)(phi_i) = -C_h(u; u, phi_i) - B_h(u, phi_i) for every broken test phi_i.

        C_h: upwind convection form, Sec. 2.2 eq. (7); B_h: SIPG viscous form,
        Sec. 3 eq. (18) with penalty alpha k^2 / h_F, h_F = max diameter of the two
        triangles. On a facet u.n is the average of both traces and the upwind
        trace is the one on the side u.n points out of, pointwise at the facet
        Gauss points (a tie at u.n = 0 gives zero flux either way).
        """
        nu = self.nu if nu is None else float(nu)
        ns = self.ns
        U = np.asarray(U, dtype=np.float64).reshape(self.n_tri, 2, ns)
        R = np.zeros((self.n_tri, 2, ns))
        for tri in self._chunks(self.n_tri):
            P, W = self._vol(tri)
            V, G = self._basis(self.exps, tri, P)                 # [m,q,j], [m,q,j,d]
            u = np.einsum("tqj,tcj->tqc", V, U[tri])
            du = np.einsum("tqjd,tcj->tqcd", G, U[tri])            # du_c/dx_d
            Flx = u[..., :, None] * u[..., None, :] - nu * du      # (u x u) - nu grad u
            R[tri] += np.einsum("tq,tqcd,tqjd->tcj", W, Flx, G, optimize=True)
        T = self.topo
        Rf = np.zeros((self.n_tri, 3, 2, ns))
        sig_all = self._penalty()
        for f in self._interior_chunks():
            t0, V0, G0 = self._facet_side(f, 0)
            t1, V1, G1 = self._facet_side(f, 1)
            n0 = T.normal[t0, T.facet_loc[f, 0]]                   # outward from side 0
            u0 = np.einsum("fqj,fcj->fqc", V0, U[t0])
            u1 = np.einsum("fqj,fcj->fqc", V1, U[t1])
            du0 = np.einsum("fqjd,fcj->fqcd", G0, U[t0])
            du1 = np.einsum("fqjd,fcj->fqcd", G1, U[t1])
            un = 0.5 * np.einsum("fqc,fc->fq", u0 + u1, n0)
            uup = np.where((un >= 0)[..., None], u0, u1)
            flux = un[..., None] * uup
            jump = u0 - u1
            dn_avg = 0.5 * np.einsum("fqcd,fd->fqc", du0 + du1, n0)
            sig = sig_all[f][:, None, None]
            wq = self.fw[None, :] * T.facet_len[f][:, None]
            A0 = -flux + nu * dn_avg - nu * sig * jump
            Bv = 0.5 * nu * jump
            dn0 = np.einsum("fqjd,fd->fqj", G0, n0)
            dn1 = np.einsum("fqjd,fd->fqj", G1, n0)
            c0 = np.einsum("fq,fqc,fqj->fcj", wq, A0, V0) + np.einsum("fq,fqc,fqj->fcj", wq, Bv, dn0)
            c1 = np.einsum("fq,fqc,fqj->fcj", wq, -A0, V1) + np.einsum("fq,fqc,fqj->fcj", wq, Bv, dn1)
            Rf[t0, T.facet_loc[f, 0]] = c0                       # each (triangle, local facet) once
            Rf[t1, T.facet_loc[f, 1]] = c1
        R += Rf.sum(axis=1)
        self._boundary_flux(U, R)
        return R.reshape(self.n_tri, self.nd)

    # ---------------------------------------------------------------- tangent
    def residual_tangent(self, U, dU, dnu=0.0):
        """Directional derivative of R = L(u)(phi_i) at u along (du, dnu) (used to check the adjoint).

        Derivative of the volume term (u x u - nu grad u) : grad phi and of the facet
        terms of eq. (7) and eq. (18). The upwind flux (u.n) u^up is differentiated in
        its equivalent form 1/2 (u.n)(u0 + u1) + 1/2 |u.n| (u0 - u1) with d|s|/ds = sign(s),
        sign(0) = 0.
        """
        if len(self.topo.inflow) or len(self.topo.outflow):
            raise NotImplementedError("the tangent covers walls and periodic meshes only")
        nu = self.nu
        ns = self.ns
        U = np.asarray(U, dtype=np.float64).reshape(self.n_tri, 2, ns)
        dU = np.asarray(dU, dtype=np.float64).reshape(self.n_tri, 2, ns)
        R = np.zeros((self.n_tri, 2, ns))
        for tri in self._chunks(self.n_tri):
            P, W = self._vol(tri)
            V, G = self._basis(self.exps, tri, P)
            u = np.einsum("tqj,tcj->tqc", V, U[tri])
            du = np.einsum("tqj,tcj->tqc", V, dU[tri])
            gu = np.einsum("tqjd,tcj->tqcd", G, U[tri])
            gdu = np.einsum("tqjd,tcj->tqcd", G, dU[tri])
            Flx = du[..., :, None] * u[..., None, :] + u[..., :, None] * du[..., None, :] - nu * gdu - dnu * gu
            R[tri] += np.einsum("tq,tqcd,tqjd->tcj", W, Flx, G, optimize=True)
        T = self.topo
        Rf = np.zeros((self.n_tri, 3, 2, ns))
        sig_all = self._penalty()
        for f in self._interior_chunks():
            t0, V0, G0 = self._facet_side(f, 0)
            t1, V1, G1 = self._facet_side(f, 1)
            n0 = T.normal[t0, T.facet_loc[f, 0]]
            u0 = np.einsum("fqj,fcj->fqc", V0, U[t0])
            u1 = np.einsum("fqj,fcj->fqc", V1, U[t1])
            d0 = np.einsum("fqj,fcj->fqc", V0, dU[t0])
            d1 = np.einsum("fqj,fcj->fqc", V1, dU[t1])
            gu0 = np.einsum("fqjd,fcj->fqcd", G0, U[t0])
            gu1 = np.einsum("fqjd,fcj->fqcd", G1, U[t1])
            gd0 = np.einsum("fqjd,fcj->fqcd", G0, dU[t0])
            gd1 = np.einsum("fqjd,fcj->fqcd", G1, dU[t1])
            un = 0.5 * np.einsum("fqc,fc->fq", u0 + u1, n0)
            dun = 0.5 * np.einsum("fqc,fc->fq", d0 + d1, n0)
            sg = np.sign(un)
            dflux = (0.5 * dun[..., None] * (u0 + u1) + 0.5 * un[..., None] * (d0 + d1)
                     + 0.5 * (sg * dun)[..., None] * (u0 - u1) + 0.5 * np.abs(un)[..., None] * (d0 - d1))
            jump, djump = u0 - u1, d0 - d1
            dn_avg = 0.5 * np.einsum("fqcd,fd->fqc", gu0 + gu1, n0)
            ddn_avg = 0.5 * np.einsum("fqcd,fd->fqc", gd0 + gd1, n0)
            sig = sig_all[f][:, None, None]
            wq = self.fw[None, :] * T.facet_len[f][:, None]
            A0 = -dflux + nu * ddn_avg - nu * sig * djump + dnu * (dn_avg - sig * jump)
            Bv = 0.5 * (nu * djump + dnu * jump)
            dn0 = np.einsum("fqjd,fd->fqj", G0, n0)
            dn1 = np.einsum("fqjd,fd->fqj", G1, n0)
            c0 = np.einsum("fq,fqc,fqj->fcj", wq, A0, V0) + np.einsum("fq,fqc,fqj->fcj", wq, Bv, dn0)
            c1 = np.einsum("fq,fqc,fqj->fcj", wq, -A0, V1) + np.einsum("fq,fqc,fqj->fcj", wq, Bv, dn1)
            Rf[t0, T.facet_loc[f, 0]] = c0
            Rf[t1, T.facet_loc[f, 1]] = c1
        R += Rf.sum(axis=1)
        return R.reshape(self.n_tri, self.nd)

    def rk3_tangent(self, U, dU, dt, nsteps=1, dnu=0.0):
        """Tangent-linear model of SSP-RK3 (eq. (8)): returns (u_K, du_K) for the perturbation (du_0, dnu).

        Each stage is linear in its functional, so du_s = Q(a M du^n + b [M du' + dt dL(u')[du', dnu]])
        with Q the same hybrid-mixed solve as the forward stage.
        """
        for _ in range(int(nsteps)):
            Us, dUs = [U], [dU]
            for s, (a, b) in enumerate(RK3_STAGES):
                Up, dUp = Us[-1], dUs[-1]
                F = a * self.apply_mass(U) + b * (self.apply_mass(Up) + dt * self.residual(Up))
                dF = a * self.apply_mass(dU) + b * (self.apply_mass(dUp) + dt * self.residual_tangent(Up, dUp, dnu))
                Us.append(self.solve_condensed(F)[0])
                dUs.append(self.solve_condensed(dF)[0])
            U, dU = Us[-1], dUs[-1]
        return U, dU

    # ------------------------------------------------------------------- mass
    def scalar_mass(self, tri):
        P, W = self._vol(tri)
        V, _ = self._basis(self.exps, tri, P)
        return np.einsum("tq,tqi,tqj->tij", W, V, V)

    def apply_mass(self, U):
        """(u, phi_i) for every broken test phi_i (L2 inner product of Sec. 2.2)."""
        U = np.asarray(U).reshape(self.n_tri, 2, self.ns)
        out = np.empty_like(U)
        for tri in self._chunks(self.n_tri):
            out[tri] = np.einsum("tij,tcj->tci", self.scalar_mass(tri), U[tri])
        return out.reshape(self.n_tri, self.nd)

    def riesz(self, R):
        """Broken field r with (r, phi_i) = R[t, i] for every broken test phi_i (element mass solves)."""
        R = np.asarray(R).reshape(self.n_tri, 2, self.ns)
        out = np.empty_like(R)
        for tri in self._chunks(self.n_tri):
            out[tri] = np.transpose(np.linalg.solve(self.scalar_mass(tri), np.transpose(R[tri], (0, 2, 1))), (0, 2, 1))
        return out.reshape(self.n_tri, self.nd)

    # ------------------------------------------------------- local operators
    def _local_ops(self, tri):
        """M_T, D_T = (z_m, div phi_j)_T, C_T = <mu_m, phi_j.n>_{F_e} of eq. (12) on triangles tri."""
        T = self.topo
        ns, nd, nw, nl = self.ns, self.nd, self.nw, self.nl
        P, W = self._vol(tri)
        V, G = self._basis(self.exps, tri, P)
        Ms = np.einsum("tq,tqi,tqj->tij", W, V, V)
        M = np.zeros((len(tri), nd, nd))
        M[:, :ns, :ns] = Ms
        M[:, ns:, ns:] = Ms
        Z, _ = self._basis(self.wexps, tri, P) if nw else (np.zeros(V.shape[:2] + (0,)), None)
        D = np.einsum("tq,tqm,tqjc->tmcj", W, Z, G).reshape(len(tri), nw, nd)
        C = np.zeros((len(tri), 3 * nl, nd))
        dof = np.zeros((len(tri), 3 * nl), dtype=np.int64)
        mu = self._facet_basis(self.ft)                                # [m, q], canonical t
        for e in range(3):
            f = T.tri_facet[tri, e]
            side = np.where((T.facet_tri[f, 0] == tri) & (T.facet_loc[f, 0] == e), 0, 1)
            Pf = T.facet_points(f, side, self.ft)
            Vf, _ = self._basis(self.exps, tri, Pf)
            n = T.normal[tri, e]
            wq = self.fw[None, :] * T.edge_len[tri, e][:, None]
            blk = np.einsum("fq,mq,fqj,fc->fmcj", wq, mu, Vf, n).reshape(len(tri), nl, nd)
            C[:, e * nl:(e + 1) * nl, :] = blk
            dof[:, e * nl:(e + 1) * nl] = f[:, None] * nl + np.arange(nl)[None, :]
        return M, D, C, dof

    def prepare(self):
        """Static condensation of eq. (12) and the sparse factorisation, computed once (Sec. 4).

        Per triangle the saddle block A_T = [[M_T, -D_T^T], [-D_T, 0]] is inverted,
        P_T = (A_T^-1)_uu and W_T = (A_T^-1)_wu. The facet system S = sum C_T P_T C_T^T
        is singular only by the constant multiplier (paired with a constant w), so
        the first coefficient of facet 0 is pinned to zero before factorising.
        """
        if self._ops is not None:
            return self._ops
        n, nd, nw, nl = self.n_tri, self.nd, self.nw, self.nl
        Pm = np.empty((n, nd, nd))
        Wm = np.empty((n, nw, nd))
        Cm = np.empty((n, 3 * nl, nd))
        Mm = np.empty((n, nd, nd))
        Dm = np.empty((n, nw, nd))
        dof = np.empty((n, 3 * nl), dtype=np.int64)
        for tri in self._chunks(n):
            M, D, C, dm = self._local_ops(tri)
            A = np.zeros((len(tri), nd + nw, nd + nw))
            A[:, :nd, :nd] = M
            A[:, :nd, nd:] = -np.transpose(D, (0, 2, 1))
            A[:, nd:, :nd] = -D
            Ai = np.linalg.inv(A)
            Pm[tri] = Ai[:, :nd, :nd]
            Wm[tri] = Ai[:, nd:, :nd]
            Cm[tri], Mm[tri], Dm[tri], dof[tri] = C, M, D, dm
        CP = np.einsum("tij,tjk->tik", Cm, Pm)
        Sloc = np.einsum("tik,tjk->tij", CP, Cm)
        nlam = self.n_facet * nl
        rows = np.repeat(dof, 3 * nl, axis=1).ravel()
        cols = np.tile(dof, (1, 3 * nl)).ravel()
        S = sp.csc_matrix((Sloc.ravel(), (rows, cols)), shape=(nlam, nlam))
        # p = 0 on Gamma_out (eq. (be)): the multipliers of outflow facets are zero, and the rest
        # of S is nonsingular; without outflow facets the constant multiplier is pinned instead
        act = np.ones(nlam, dtype=bool)
        out = self.topo.outflow
        if len(out):
            act[(out[:, None] * nl + np.arange(nl)[None, :]).ravel()] = False
        else:
            act[0] = False
        act = np.flatnonzero(act)
        lu = spla.splu(S[act][:, act].tocsc())
        Zint = None
        if nw:
            Pp, Wq = self._vol(np.arange(n))
            Zv, _ = self._basis(self.wexps, np.arange(n), Pp)
            Zint = np.einsum("tq,tqm->tm", Wq, Zv)
        self._ops = dict(P=Pm, W=Wm, C=Cm, M=Mm, D=Dm, CP=CP, dof=dof, S=S, lu=lu, Zint=Zint, act=act)
        return self._ops

    # ------------------------------------------------------------------ solve
    def solve_condensed(self, F, homogeneous=False):
        """Hybrid-mixed solve of eq. (12) for the functional F[t, i] (Theorem 2).

        Returns (u, w, lam): u in the globally divergence-free space, w and lam
        before the constant shift (see normalize_pressure). With inflow facets u.n = u_in.n
        holds there (Sec. 2.5): the facet system is S lam = g - d with the data moments d;
        homogeneous = True solves with u.n = 0 instead (the time derivative of a state that
        keeps the inflow data, as for the pressure functional L(u)).
        """
        o = self.prepare()
        F = np.asarray(F).reshape(self.n_tri, self.nd)
        gloc = np.einsum("tij,tj->ti", o["CP"], F)
        g = np.bincount(o["dof"].ravel(), weights=gloc.ravel(), minlength=self.n_facet * self.nl)
        if not homogeneous:
            g = g - self.inflow_d
        lam = np.zeros_like(g)
        lam[o["act"]] = o["lu"].solve(g[o["act"]])
        r = F - np.einsum("tij,ti->tj", o["C"], lam[o["dof"]])
        u = np.einsum("tij,tj->ti", o["P"], r)
        w = np.einsum("tij,tj->ti", o["W"], r)
        return u, w, lam

    def normalize_pressure(self, w, lam):
        """Shift w and lam by one constant so that the integral of w over the domain is zero (L^2_0, eq. (4e)).
        With outflow facets p = 0 there fixes the constant (eq. (be)): no shift."""
        if len(self.topo.outflow):
            return w, lam
        o = self.prepare()
        c = (o["Zint"] * w).sum() / self.topo.area.sum()
        w = w.copy()
        lam = lam.copy()
        w -= c          # Bernstein bases are partitions of unity: the constant is all ones
        lam -= c
        return w, lam

    def solve_full(self, F):
        """Same system eq. (12) solved uncondensed: one sparse saddle-point factorisation."""
        o = self.prepare()
        n, nd, nw, nl = self.n_tri, self.nd, self.nw, self.nl
        nu_, nwt, nlam = n * nd, n * nw, self.n_facet * nl
        blocks_r, blocks_c, blocks_v = [], [], []

        def add(r, c, v):
            blocks_r.append(r.ravel())
            blocks_c.append(c.ravel())
            blocks_v.append(v.ravel())
        ui = np.arange(nu_).reshape(n, nd)
        wi = nu_ + np.arange(nwt).reshape(n, nw)
        li = nu_ + nwt + o["dof"]
        add(np.repeat(ui, nd, 1), np.tile(ui, (1, nd)), o["M"])
        if nw:
            add(np.repeat(ui, nw, 1), np.tile(wi, (1, nd)), -np.transpose(o["D"], (0, 2, 1)))
            add(np.repeat(wi, nd, 1), np.tile(ui, (1, nw)), -o["D"])
        add(np.repeat(ui, 3 * nl, 1), np.tile(li, (1, nd)), np.transpose(o["C"], (0, 2, 1)))
        add(np.repeat(li, nd, 1), np.tile(ui, (1, 3 * nl)), o["C"])
        N = nu_ + nwt + nlam
        K = sp.csr_matrix((np.concatenate(blocks_v), (np.concatenate(blocks_r), np.concatenate(blocks_c))),
                          shape=(N, N))
        keep = np.ones(N, dtype=bool)
        keep[nu_ + nwt + np.setdiff1d(np.arange(nlam), o["act"])] = False   # outflow (or the pinned dof)
        rhs = np.zeros(N)
        rhs[:nu_] = np.asarray(F).ravel()
        rhs[nu_ + nwt:] = self.inflow_d       # C u = d on inflow facets, 0 elsewhere
        x = np.zeros(N)
        x[keep] = spla.spsolve(K[keep][:, keep].tocsc(), rhs[keep])
        return x[:nu_].reshape(n, nd), x[nu_:nu_ + nwt].reshape(n, nw), x[nu_ + nwt:]

    def constraint_matrix(self):
        """Rows: element divergence moments against P^{k-1} and facet normal-jump moments against P^k.

        Its null space in the broken space is the globally divergence-free space
        V_h^{k,-1} of eq. (4d) (div V_h^k = Q^{k-1}, Theorem 1).
        """
        o = self.prepare()
        n, nd, nw = self.n_tri, self.nd, self.nw
        Dg = sp.block_diag([o["D"][t] for t in range(n)]) if nw else sp.csr_matrix((0, n * nd))
        rows = np.repeat(o["dof"], nd, axis=1).ravel()
        cols = (np.arange(n)[:, None, None] * nd + np.arange(nd)[None, None, :]).repeat(3 * self.nl, 1).ravel()
        Cg = sp.csr_matrix((o["C"].ravel(), (rows, cols)), shape=(self.n_facet * self.nl, n * nd))
        return sp.vstack([Dg, Cg]).tocsr()

    def _active_constraints(self):
        """Constraint rows and right-hand side: the outflow facets' normal-trace rows are
        dropped (u.n is free there), inflow rows carry the data moments (Sec. 2.5)."""
        B = self.constraint_matrix()
        nw_all = self.n_tri * self.nw
        keep = np.ones(B.shape[0], dtype=bool)
        out = self.topo.outflow
        if len(out):
            keep[nw_all + (out[:, None] * self.nl + np.arange(self.nl)[None, :]).ravel()] = False
        c = np.concatenate([np.zeros(nw_all), self.inflow_d])
        return B[keep], c[keep]

    def divfree_basis(self):
        """Explicit orthonormal basis Z of V_h^{k,-1} (with the boundary conditions: the space
        with u.n = 0 on inflow facets) by SVD (tiny meshes only)."""
        B, _ = self._active_constraints()
        return sla.null_space(B.toarray(), rcond=1e-11)

    def project_nullspace(self, F):
        """L2 projection through the explicit basis onto the affine space {B u = c}:
        u = u_p + Z (Z^T M Z)^-1 Z^T (F - M u_p), u_p any solution of B u = c."""
        o = self.prepare()
        Z = self.divfree_basis()
        B, c = self._active_constraints()
        up = np.linalg.lstsq(B.toarray(), c, rcond=None)[0]
        Mg = sp.block_diag([o["M"][t] for t in range(self.n_tri)]).toarray()
        a = np.linalg.solve(Z.T @ Mg @ Z, Z.T @ (np.asarray(F).ravel() - Mg @ up))
        return (up + Z @ a).reshape(self.n_tri, self.nd)

    def solve_fe4(self, F):
        """Locally divergence-free hybrid variant eq. (13): broken div-free velocity and lam only.

        The multiplier enters with the opposite sign, so lam_FE4 = -lam_FE3; the
        velocity is the same (Remark 3).
        """
        o = self.prepare()
        n, nl = self.n_tri, self.nl
        F = np.asarray(F).reshape(n, self.nd)
        Y = [sla.null_space(o["D"][t]) if self.nw else np.eye(self.nd) for t in range(n)]
        rows, cols, vals = [], [], []
        g = np.zeros(self.n_facet * nl)
        loc = []
        for t in range(n):
            Yt = Y[t]
            Mz = Yt.T @ o["M"][t] @ Yt
            Cz = o["C"][t] @ Yt
            Mi = np.linalg.inv(Mz)
            Sl = Cz @ Mi @ Cz.T
            d = o["dof"][t]
            rows.append(np.repeat(d, len(d)))
            cols.append(np.tile(d, len(d)))
            vals.append(Sl.ravel())
            np.add.at(g, d, -Cz @ Mi @ (Yt.T @ F[t]))
            loc.append((Yt, Mi, Cz))
        S = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n_facet * nl,) * 2)
        lam = np.zeros_like(g)
        lam[1:] = spla.spsolve(S[1:, 1:].tocsc(), g[1:])
        u = np.empty((n, self.nd))
        for t in range(n):
            Yt, Mi, Cz = loc[t]
            u[t] = Yt @ (Mi @ (Yt.T @ F[t] + Cz.T @ lam[o["dof"][t]]))
        return u, lam

    # ------------------------------------------------------------ time steps
    def project(self, U):
        """L2 projection of a broken field onto V_h^{k,-1} (the solve with F = (u, .))."""
        u, _, _ = self.solve_condensed(self.apply_mass(U))
        return u

    def stage(self, Un, Up, a, b, dt):
        """One SSP-RK3 stage in the paper's form: M u_new = a M u^n + b [M u' + dt L(u')] (eq. (8))."""
        F = a * self.apply_mass(Un) + b * (self.apply_mass(Up) + dt * self.residual(Up))
        u, _, _ = self.solve_condensed(F)
        return u

    def rk3_step(self, U, dt, nsteps=1):
        for _ in range(int(nsteps)):
            U1 = self.stage(U, U, *RK3_STAGES[0], dt)
            U2 = self.stage(U, U1, *RK3_STAGES[1], dt)
            U = self.stage(U, U2, *RK3_STAGES[2], dt)
        return U

    def slope(self, U):
        """Time derivative of the semi-discrete system eq. (6) on V_h^{k,-1}: the hybrid-mixed
        solve of eq. (12) with the functional L(u) alone (the mass inversion of Sec. 3.1)."""
        du, _, _ = self.solve_condensed(self.residual(U), homogeneous=True)
        return du

    def euler_step(self, U, dt, nsteps=1):
        """Forward Euler, eq. (FE) of Sec. 3.1, with the full L of eq. (6) (viscous terms
        included): M u^(n+1) = M u^n + dt L(u^n), one hybrid-mixed solve per step."""
        for _ in range(int(nsteps)):
            U, _, _ = self.solve_condensed(self.apply_mass(U) + dt * self.residual(U))
        return U

    def rk4_step(self, U, dt, nsteps=1):
        """The classical four-stage, fourth-order Runge-Kutta scheme used for the temporal
        accuracy test (Example 1b, Table 2), applied to du/dt = slope(u)."""
        for _ in range(int(nsteps)):
            k1 = self.slope(U)
            k2 = self.slope(U + 0.5 * dt * k1)
            k3 = self.slope(U + 0.5 * dt * k2)
            k4 = self.slope(U + dt * k3)
            U = U + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        return U

    def pressure(self, U):
        """(w, lam) of eq. (12) with the functional L(u) alone: w ~ p, lam ~ p on the skeleton (Theorem 2, Remark 2)."""
        _, w, lam = self.solve_condensed(self.residual(U), homogeneous=True)
        return self.normalize_pressure(w, lam)

    # --------------------------------------------------------------- lattice
    def _facet_basis(self, t):
        """Bernstein basis of P^k on a facet in its canonical parameter t: C(k,m) t^m (1-t)^(k-m)."""
        k = self.k
        return np.stack([_binom(k, m) * t ** m * (1.0 - t) ** (k - m) for m in range(k + 1)], 0)

    def _lattice_xi(self, m):
        if m == 0:
            return np.array([[1.0 / 3.0, 1.0 / 3.0]])
        return np.array([(i / m, j / m) for j in range(m + 1) for i in range(m + 1 - j)])

    def _lattice_V(self, exps, m):
        T = self.topo
        xi = self._lattice_xi(m)
        P = T.X[:, 0][:, None, :] + np.einsum("tij,qj->tqi", T.J, xi)
        V, _ = self._basis(exps, np.arange(self.n_tri), P)
        return V

    def from_lattice(self, vals):
        """Coefficients of the broken P^k field with the given values at the degree-k lattice."""
        vals = np.asarray(vals, dtype=np.float64).reshape(self.n_tri, self.ns, 2)
        V = self._lattice_V(self.exps, self.k)
        c = np.linalg.solve(V, vals)                   # [t, j, comp]
        return np.transpose(c, (0, 2, 1)).reshape(self.n_tri, self.nd)

    def to_lattice(self, U):
        V = self._lattice_V(self.exps, self.k)
        U = np.asarray(U).reshape(self.n_tri, 2, self.ns)
        return np.einsum("tpj,tcj->tpc", V, U)

    def pressure_lattice(self, w, lam):
        """w at the degree-(k-1) lattice [n_tri, n_lat(k-1)] and lam at t = i/k on each facet [n_facet, k+1]."""
        V = self._lattice_V(self.wexps, self.k - 1)
        pe = np.einsum("tpm,tm->tp", V, w)
        ti = np.arange(self.k + 1) / self.k
        pf = lam.reshape(self.n_facet, self.nl) @ self._facet_basis(ti)
        return pe, pf

    # ------------------------------------------------------------ diagnostics
    def energy(self, U):
        return float((np.asarray(U) * self.apply_mass(U)).sum())

    def diagnostics(self, U):
        """Energy ||u||^2, enstrophy ||curl_h u||^2 (Example 2), max |div u| and max |[u.n]| at quadrature points."""
        ns = self.ns
        U = np.asarray(U).reshape(self.n_tri, 2, ns)
        ens = 0.0
        divmax = 0.0
        for tri in self._chunks(self.n_tri):
            P, W = self._vol(tri)
            V, G = self._basis(self.exps, tri, P)
            du = np.einsum("tqjd,tcj->tqcd", G, U[tri])
            om = du[..., 1, 0] - du[..., 0, 1]
            ens += float((W * om * om).sum())
            divmax = max(divmax, float(np.abs(du[..., 0, 0] + du[..., 1, 1]).max()))
        T = self.topo
        f = np.arange(self.n_facet)
        t0, V0, _ = self._facet_side(f, 0)
        n0 = T.normal[t0, T.facet_loc[:, 0]]
        u0 = np.einsum("fqj,fcj->fqc", V0, U[t0])
        u1 = np.zeros_like(u0)                      # walls: the jump is u.n itself
        fi = T.interior
        _, V1, _ = self._facet_side(fi, 1)
        u1[fi] = np.einsum("fqj,fcj->fqc", V1, U[T.facet_tri[fi, 1]])
        u1[T.inflow] = self.inflow_q[T.inflow]      # inflow: against the data; outflow: u.n is free
        jmp = np.abs(np.einsum("fqc,fc->fq", u0 - u1, n0))
        jmp[T.outflow] = 0.0
        jmax = float(jmp.max())
        return dict(energy=self.energy(U.reshape(self.n_tri, -1)), enstrophy=ens, max_div=divmax, max_jump=jmax)

    def upwind_dissipation(self, U):
        """(1/2) sum_F int_F |u.n| |u^+ - u^-|^2 at the facet Gauss points (energy identity of Sec. 2.2)."""
        T = self.topo
        U = np.asarray(U).reshape(self.n_tri, 2, self.ns)
        f = T.interior                              # walls carry no flux (u.n = 0)
        t0, V0, _ = self._facet_side(f, 0)
        t1, V1, _ = self._facet_side(f, 1)
        n0 = T.normal[t0, T.facet_loc[f, 0]]
        u0 = np.einsum("fqj,fcj->fqc", V0, U[t0])
        u1 = np.einsum("fqj,fcj->fqc", V1, U[t1])
        un = 0.5 * np.einsum("fqc,fc->fq", u0 + u1, n0)
        wq = self.fw[None, :] * T.facet_len[f][:, None]
        return 0.5 * float((wq * np.abs(un) * ((u0 - u1) ** 2).sum(-1)).sum())

    def l2_error(self, U, field, rule_degree=None):
        """||u_h - u||_{L2} against an analytic field (x, y) -> (u1, u2)."""
        rule = triangle_rule(rule_degree or (2 * self.k + 12))
        U = np.asarray(U).reshape(self.n_tri, 2, self.ns)
        err = 0.0
        for tri in self._chunks(self.n_tri):
            P, W = self._vol(tri, rule)
            V, _ = self._basis(self.exps, tri, P)
            u = np.einsum("tqj,tcj->tqc", V, U[tri])
            e1, e2 = field(P[..., 0], P[..., 1])
            err += float((W * ((u[..., 0] - e1) ** 2 + (u[..., 1] - e2) ** 2)).sum())
        return np.sqrt(err)

    def pressure_l2_error(self, w, pfield, rule_degree=None):
        """||w - p||_{L2} for a mean-free analytic pressure (x, y) -> p."""
        rule = triangle_rule(rule_degree or (2 * self.k + 12))
        err = 0.0
        for tri in self._chunks(self.n_tri):
            P, W = self._vol(tri, rule)
            Z, _ = self._basis(self.wexps, tri, P)
            wv = np.einsum("tqm,tm->tq", Z, w[tri])
            err += float((W * (wv - pfield(P[..., 0], P[..., 1])) ** 2).sum())
        return np.sqrt(err)
