"""Pins of the three-dimensional oracle (oracle/dg3.py) against what the paper and mathematics fix.

Each test would fail for a plausible mistake in the oracle: wrong quadrature, wrong face
matching or normal, a dropped or mis-signed flux or SIPG term, a wrong condensation.
"""
import math

import numpy as np
import pytest

from oracle.dg3 import Discretization3, face_rule, tet_rule
from synth.mesh3 import abc_flow, kuhn_cube_mesh, sample_lattice3


def disc(N, k, nu=0.0):
    vid, X = kuhn_cube_mesh(N)
    return Discretization3(vid, X, k, nu), X


@pytest.mark.parametrize("degree", [2, 5, 8])
def test_tet_rule_integrates_monomials_exactly(degree):
    # int over the reference tetrahedron of x^a y^b z^c = a! b! c! / (a + b + c + 3)!
    xi, w = tet_rule(degree)
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            for c in range(degree + 1 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                assert abs((w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c).sum() - exact) < 1e-15


@pytest.mark.parametrize("k", [1, 2, 3])
def test_face_rule_integrates_degree_3k_exactly(k):
    # int over the reference triangle of s^a t^b = a! b! / (a + b + 2)!, to degree 3k
    st, w = face_rule(k)
    for a in range(3 * k + 1):
        for b in range(3 * k + 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs((w * st[:, 0] ** a * st[:, 1] ** b).sum() - exact) < 1e-15


@pytest.mark.parametrize("N", [2, 3])
def test_periodic_kuhn_topology(N):
    d, X = disc(N, 1)
    T = d.topo
    assert d.n_tet == 6 * N ** 3 and d.n_face == 12 * N ** 3
    assert abs(T.vol.sum() - (2 * np.pi) ** 3) < 1e-9
    f = np.arange(d.n_face)
    # both sides of every face: opposite normals, equal areas, the same canonical points up to a period
    n0 = T.normal[T.face_tet[:, 0], T.face_loc[:, 0]]
    n1 = T.normal[T.face_tet[:, 1], T.face_loc[:, 1]]
    assert np.abs(n0 + n1).max() < 1e-14
    assert np.abs(T.area[T.face_tet[:, 0], T.face_loc[:, 0]] - T.area[T.face_tet[:, 1], T.face_loc[:, 1]]).max() < 1e-12
    P0 = T.face_points(f, np.zeros_like(f), d.fst)
    P1 = T.face_points(f, np.ones_like(f), d.fst)
    off = (P0 - P1) / (2 * np.pi)
    assert np.abs(off - np.round(off)).max() < 1e-12
    # the divergence theorem per tetrahedron: sum of area-weighted outward normals is zero
    assert np.abs(np.einsum("te,tei->ti", T.area, T.normal)).max() < 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_divergence_free_space_dimension(k):
    # v -> (div v, [v.n]) from broken [P^k]^3 onto broken P^{k-1} x face P^k has a one-dimensional
    # cokernel (w constant, mu = w on the faces), so
    # dim V_h^{k,-1} = N_T n_u - N_T n_w - N_F n_lambda + 1
    d, X = disc(2, k)
    o = d.prepare()
    n, nd, nw, nl = d.n_tet, d.nd, d.nw, d.nl
    rows = np.zeros((n * nw + d.n_face * nl, n * nd))
    for t in range(n):
        rows[t * nw:(t + 1) * nw, t * nd:(t + 1) * nd] = o["D"][t]
        for i in range(4 * nl):
            rows[n * nw + o["dof"][t, i], t * nd:(t + 1) * nd] += o["C"][t, i]
    rank = np.linalg.matrix_rank(rows)
    assert n * nd - rank == n * nd - n * nw - d.n_face * nl + 1


@pytest.mark.parametrize("k", [1, 2])
def test_condensed_and_saddle_solves_agree_and_project(k):
    d, X = disc(2, k)
    F = np.random.default_rng(k).standard_normal((d.n_tet, d.nd))
    u1 = d.solve_condensed(F)[0]
    u2 = d.solve_full(F)
    assert np.abs(u1 - u2).max() < 1e-11 * np.abs(u1).max()
    dg = d.diagnostics(u1)
    assert dg["max_div"] < 1e-11 and dg["max_jump"] < 1e-11
    # L2 projection: idempotent, and the removed part is orthogonal to the divergence-free space
    U = d.project(F)
    assert np.abs(d.project(U) - U).max() < 1e-11
    V = d.project(np.random.default_rng(9).standard_normal((d.n_tet, d.nd)))
    assert abs(((F - U) * d.apply_mass(V)).sum()) < 1e-10 * np.abs(F).max() * np.abs(V).max() * d.n_tet


@pytest.mark.parametrize("k", [1, 2])
def test_energy_identity_of_upwind_form(k):
    # Sec. 2.2: for divergence-free u, C_h(u; u, u) = 1/2 sum_F int_F |u.n| |u+ - u-|^2; with nu = 0,
    # L(u)(u) = -C_h(u; u, u)
    d, X = disc(2, k)
    U = d.project(np.random.default_rng(3).standard_normal((d.n_tet, d.nd)))
    diss = d.upwind_dissipation(U)
    assert diss > 1.0
    assert abs((d.residual(U, nu=0.0) * U).sum() + diss) < 1e-11 * diss


def test_sipg_form_is_symmetric_and_nonnegative():
    # eq. (18) is symmetric: B_h(u, v) = B_h(v, u), read off the viscous part of L; and B_h(u, u) >= 0
    # on the divergence-free space at alpha = 2, k = 2
    d, X = disc(2, 2, nu=1.0)
    rng = np.random.default_rng(5)
    u = d.project(rng.standard_normal((d.n_tet, d.nd)))
    v = d.project(rng.standard_normal((d.n_tet, d.nd)))

    def B(a):
        return -(d.residual(a, nu=1.0) - d.residual(a, nu=0.0))
    buv, bvu = (B(u) * v).sum(), (B(v) * u).sum()
    assert abs(buv - bvu) < 1e-10 * abs(buv)
    assert (B(u) * u).sum() > 0


def test_constant_velocity_is_steady():
    # a constant field lies in the divergence-free space, and its residual vanishes for every test
    # function (the face fluxes cancel the integration by parts of the volume term)
    d, X = disc(2, 2, nu=0.05)
    vals = sample_lattice3(lambda x, y, z: (0.3 + 0 * x, -0.7 + 0 * y, 0.2 + 0 * z), X, 2)
    U = d.from_lattice(vals)
    assert np.abs(d.project(U) - U).max() < 1e-12
    assert np.abs(d.residual(U)).max() < 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_abc_flow_projection_converges_at_order_k_plus_1(k):
    # the Arnold-Beltrami-Childress field (divergence free, smooth, periodic): the L2 projection onto
    # V_h^{k,-1} converges at order k + 1 (Sec. 2.1, the approximation of BDM_k)
    errs = []
    for N in (3, 4):
        d, X = disc(N, k)
        U = d.project(d.from_lattice(sample_lattice3(abc_flow(), X, k)))
        errs.append(d.l2_error(U, abc_flow()))
    eoc = math.log(errs[0] / errs[1]) / math.log(4 / 3)
    assert eoc > k + 1 - 0.25, eoc


def test_abc_flow_decays_as_exp_minus_nu_t():
    # curl u = u for the ABC field, so u exp(-nu t) solves Navier-Stokes; SSP-RK3 steps of its
    # projection follow that decay to the spatial error, which falls with N at about the order k+1
    k, nu, t_end = 2, 0.1, 0.4
    errs = []
    for N in (2, 3):
        d, X = disc(N, k, nu=nu)
        U = d.project(d.from_lattice(sample_lattice3(abc_flow(), X, k)))
        steps = 8
        U = d.rk3_step(U, t_end / steps, steps)
        f = abc_flow()

        def ex(x, y, z):
            return tuple(c * math.exp(-nu * t_end) for c in f(x, y, z))
        errs.append(d.l2_error(U, ex))
    assert errs[1] < 0.45 * errs[0], errs


def _abc_pressure(P, A=1.0, B=0.7, C=0.4):
    # the ABC flow is a Beltrami field (curl u = u), so (u.grad) u = grad |u|^2 / 2 and the steady
    # Euler pressure is p = -|u|^2 / 2 + const; its mean over the periodic cube is -(A^2+B^2+C^2)/2
    u = np.stack(abc_flow(A, B, C)(P[..., 0], P[..., 1], P[..., 2]), -1)
    return -0.5 * (u ** 2).sum(-1) + 0.5 * (A * A + B * B + C * C)


@pytest.mark.parametrize("k,Ns", [(1, (4, 6)), (2, (3, 4))])
def test_abc_pressure_converges_at_order_k(k, Ns):
    # w ~ p (Theorem 2, Remark 2) in broken P^(k-1): L2 error of order k (measured 1.09 and 1.87);
    # the face multiplier approximates the same pressure on the skeleton. A sign error in the
    # pressure, the condensation or the constant shift leaves an O(1) error that does not fall.
    e_el, e_fa = [], []
    for N in Ns:
        d, X = disc(N, k)
        U = d.project(d.from_lattice(sample_lattice3(abc_flow(), X, k)))
        w, lam = d.pressure(U)
        tet = np.arange(d.n_tet)
        P, W = d._vol(tet)
        Z, _ = d._basis(d.wexps, tet, P)
        assert abs(np.einsum("tq,tqm,tm->", W, Z, w)) < 1e-10 * W.sum()
        e_el.append(math.sqrt((W * (np.einsum("tqm,tm->tq", Z, w) - _abc_pressure(P)) ** 2).sum()))
        _, pf = d.pressure_lattice(w, lam)
        T = d.topo
        st = np.array([(i / k, j / k) for j in range(k + 1) for i in range(k + 1 - j)])
        f = np.arange(d.n_face)
        pts = T.face_points(f, np.zeros_like(f), st)
        e_fa.append(np.abs(pf - _abc_pressure(pts)).max())
    rate = math.log(e_el[0] / e_el[1]) / math.log(Ns[1] / Ns[0])
    assert abs(rate - k) < 0.4, (k, rate, e_el)
    assert e_fa[1] < e_fa[0], e_fa
