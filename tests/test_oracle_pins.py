"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test is chosen so that a plausible mistake in one part of the oracle
(a dropped term, a wrong sign, a transposed operand, a wrong stage
coefficient) fails it. None of them compares the oracle with itself.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import Discretization
from oracle.quadrature import triangle_rule, facet_rule

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def disc(N, k, nu=0.0, L=2 * np.pi, alpha=2.0):
    vid, X = synth.split_square_mesh(N, L=L)
    return Discretization(vid, X, k, nu, alpha=alpha), X


def projected(d, X, field):
    return d.project(d.from_lattice(synth.sample_lattice(field, X, d.k)))


def load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return rows


# ------------------------------------------------------------------ quadrature
@pytest.mark.parametrize("deg", [2, 5, 8, 11])
def test_triangle_rule_exact_for_monomials(deg):
    # closed form: int over the unit right triangle of x^a y^b = a! b! / (a + b + 2)!
    xi, w = triangle_rule(deg)
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs((w * xi[:, 0] ** a * xi[:, 1] ** b).sum() - exact) < 1e-15


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_facet_rule_exact_to_degree_3k(k):
    t, w = facet_rule(k)
    assert len(t) == math.ceil((3 * k + 1) / 2)
    for p in range(3 * k + 1):
        assert abs((w * t ** p).sum() - 1.0 / (p + 1)) < 1e-15


# ------------------------------------------------------------------------ mesh
@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_periodic_split_square_topology(N):
    d, _ = disc(N, 1)
    T = d.topo
    assert d.n_tri == 2 * N * N and d.n_facet == 3 * N * N
    # every facet is shared by two triangles traversing it in opposite directions
    assert np.all(T.facet_orient[:, 0] == -T.facet_orient[:, 1])
    # both sides see the same edge length and opposite outward normals
    l0 = T.edge_len[T.facet_tri[:, 0], T.facet_loc[:, 0]]
    l1 = T.edge_len[T.facet_tri[:, 1], T.facet_loc[:, 1]]
    n0 = T.normal[T.facet_tri[:, 0], T.facet_loc[:, 0]]
    n1 = T.normal[T.facet_tri[:, 1], T.facet_loc[:, 1]]
    assert np.allclose(l0, l1) and np.allclose(n0, -n1)
    # the two copies of a facet point differ by a period (or coincide)
    t = np.array([0.3])
    f = np.arange(d.n_facet)
    p0 = T.facet_points(f, np.zeros_like(f), t)[:, 0]
    p1 = T.facet_points(f, np.ones_like(f), t)[:, 0]
    shift = (p0 - p1) / (2 * np.pi)
    assert np.allclose(shift, np.round(shift), atol=1e-12)


def test_nonmanifold_mesh_rejected():
    # a repeated triangle puts three triangles on its edges
    vid, X = synth.split_square_mesh(3)
    with pytest.raises(ValueError):
        Discretization(np.concatenate([vid, vid[:1]]), np.concatenate([X, X[:1]]), 1, 0.0)


def test_box_topology_has_walls():
    # N x N split squares of the unit square: 3N^2 + 2N facets, 4N of them on the walls
    for N in (1, 3):
        vid, X = synth.split_square_mesh(N, L=1.0, periodic=False)
        T = Discretization(vid, X, 1, 0.0).topo
        assert T.n_facet == 3 * N * N + 2 * N and T.boundary.sum() == 4 * N
        # every wall facet lies on the square's boundary and its normal points outward
        f = np.flatnonzero(T.boundary)
        mid = T.facet_points(f, np.zeros_like(f), np.array([0.5]))[:, 0]
        on = np.minimum(np.minimum(mid[:, 0], 1 - mid[:, 0]), np.minimum(mid[:, 1], 1 - mid[:, 1]))
        assert np.abs(on).max() < 1e-14
        n = T.normal[T.facet_tri[f, 0], T.facet_loc[f, 0]]
        assert np.all(((mid - 0.5) * n).sum(-1) > 0)


# ------------------------------------------------------------ walls (free slip)
@pytest.mark.parametrize("N,k", [(1, 1), (2, 1), (2, 2), (2, 3), (3, 2)])
def test_divfree_dimension_in_box_with_walls(N, k):
    # V_h with u.n = 0 on the walls is curl of the continuous P^{k+1} stream functions that
    # vanish on the boundary (exact sequence on a simply connected domain): one per interior
    # Lagrange node of degree k+1, ((k+1) N - 1)^2 on the split-square mesh
    vid, X = synth.split_square_mesh(N, L=1.0, periodic=False)
    d = Discretization(vid, X, k, 0.0)
    assert d.divfree_basis().shape[1] == ((k + 1) * N - 1) ** 2


@pytest.mark.parametrize("k", [1, 2, 3])
def test_wall_projection_routes_agree(k):
    # condensed solve = uncondensed saddle solve = projection through the explicit basis, and
    # the result has no normal velocity on the walls
    vid, X = synth.split_square_mesh(2, L=1.0, periodic=False)
    d = Discretization(vid, X, k, 0.0)
    rng = np.random.default_rng(k)
    F = d.apply_mass(rng.standard_normal((d.n_tri, d.nd)))
    u1, _, _ = d.solve_condensed(F)
    u2, _, _ = d.solve_full(F)
    u3 = d.project_nullspace(F)
    assert np.abs(u1 - u2).max() < 1e-12 and np.abs(u1 - u3).max() < 1e-12
    dg = d.diagnostics(u1)
    assert dg["max_jump"] < 1e-12 and dg["max_div"] < 1e-11


def test_taylor_green_cell_with_free_slip_walls():
    # u = (sin pi x cos pi y, -cos pi x sin pi y) on the unit square has u.n = 0 and zero
    # vorticity (hence zero tangential stress) on the walls and solves Navier-Stokes with
    # u(t) = u0 exp(-2 nu pi^2 t): velocity error of order k+1 (Table 1 shape)
    nu, k, T = 1e-2, 2, 0.1
    tg = synth.taylor_green(L=2.0)
    errs = []
    for N in (4, 8):
        vid, X = synth.split_square_mesh(N, L=1.0, periodic=False)
        d = Discretization(vid, X, k, nu)
        U = d.project(d.from_lattice(synth.sample_lattice(tg, X, k)))
        n = 2 * N
        U = d.rk3_step(U, T / n, n)
        dec = math.exp(-2.0 * nu * math.pi ** 2 * T)
        errs.append(d.l2_error(U, lambda x, y: tuple(v * dec for v in tg(x, y))))
        assert d.diagnostics(U)["max_jump"] < 1e-12
    assert abs(math.log2(errs[0] / errs[1]) - (k + 1)) < 0.35, errs


def test_wall_energy_non_increasing_and_identity():
    # nu = 0, walls: the wall facets carry no flux, so the energy identity of Sec. 2.2 keeps
    # only the interior upwind dissipation and the energy does not grow
    vid, X = synth.split_square_mesh(5, L=1.0, periodic=False)
    d = Discretization(vid, X, 2, 0.0)
    U = d.project(d.from_lattice(synth.sample_lattice(synth.random_spectrum_velocity(5, kmax=4, L=1.0), X, 2)))
    dt = synth.cfl_dt(X, 2, np.abs(d.to_lattice(U)).max(), 0.0)
    E = [d.energy(U)]
    for _ in range(6):
        U = d.rk3_step(U, dt, 1)
        E.append(d.energy(U))
    assert np.all(np.diff(E) <= 1e-14 * E[0]) and E[-1] < E[0]
    rate = -2.0 * d.upwind_dissipation(U)
    for h in (1e-3, 5e-4):
        est = (d.energy(d.rk3_step(U, h, 1)) - d.energy(U)) / h
        assert abs(est - rate) < 50 * h * abs(rate) + 1e-12


# ------------------------------------------------------------ space dimensions
@pytest.mark.parametrize("N,k", [(1, 1), (2, 1), (2, 2), (3, 2), (2, 3), (3, 3)])
def test_divfree_dimension_on_torus(N, k):
    # V_h^{k,-1} = curl of continuous P^{k+1} (Remark 1): N^2 (k+1)^2 - 1 curls plus 2 constant fields
    d, _ = disc(N, k)
    assert d.divfree_basis().shape[1] == N * N * (k + 1) ** 2 + 1
    # the BDM space (normal continuity only) has N^2 (k+1)(2k+1) dimensions on the torus
    B = d.constraint_matrix().toarray()
    nf = d.n_facet * d.nl
    jump_rows = B[d.n_tri * d.nw:]
    assert jump_rows.shape[0] == nf
    bdm = d.n_tri * d.nd - np.linalg.matrix_rank(jump_rows)
    assert bdm == N * N * (k + 1) * (2 * k + 1)


def test_table3_dof_counts():
    # NGSolve variant of Remark 3: velocity with div in P^0 plus a constant pressure per element,
    # multipliers P^k per facet; Table 3 totals over 488 triangles and 772 facets
    import scipy.linalg as sla
    for k, local, glob in load_golden("table3_dofs.txt"):
        k = int(k)
        d, _ = disc(2, k)
        D = d.prepare()["D"][0]                               # (z_m, div phi_j) on triangle 0
        P, W = d._vol(np.array([0]))
        Z, _ = d._basis(d.wexps, np.array([0]), P)
        mean = np.einsum("tq,tqm->m", W, Z)                   # (z_m, 1)
        Q = sla.null_space(mean[None, :])                     # mean-free pressures
        dim_vel = d.nd - np.linalg.matrix_rank(Q.T @ D)
        assert 488 * (dim_vel + 1) == int(local)
        assert 772 * d.nl == int(glob)


# ------------------------------------------------------------------ the solve
@pytest.mark.parametrize("N,k", [(2, 1), (2, 2), (3, 3)])
def test_four_solve_routes_agree(N, k):
    d, X = disc(N, k)
    rng = np.random.default_rng(7)
    F = rng.standard_normal((d.n_tri, d.nd))
    u1, w1, l1 = d.solve_condensed(F)
    u2 = d.project_nullspace(F)
    u3, w3, l3 = d.solve_full(F)
    u4, l4 = d.solve_fe4(F)
    s = np.linalg.norm(u1)
    assert np.linalg.norm(u1 - u2) / s < 1e-12
    assert np.linalg.norm(u1 - u3) / s < 1e-12
    assert np.linalg.norm(u1 - u4) / s < 1e-12
    w1n, l1n = d.normalize_pressure(w1, l1)
    w3n, l3n = d.normalize_pressure(w3, l3)
    assert np.abs(w1n - w3n).max() < 1e-10 * max(1, np.abs(w1n).max())
    # eq. (13) carries the multiplier with the opposite sign (defined up to the same constant)
    _, l4n = d.normalize_pressure(w1, -l4)
    assert np.abs(l4n - l1n).max() < 1e-10 * max(1, np.abs(l1n).max())


def test_projection_is_divfree_idempotent_and_symmetric():
    d, X = disc(3, 2)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((d.n_tri, d.nd))
    P1 = d.project(U)
    dg = d.diagnostics(P1)
    assert dg["max_div"] < 1e-12 and dg["max_jump"] < 1e-12
    P2 = d.project(P1)
    assert np.abs(P2 - P1).max() < 1e-12 * np.abs(P1).max()
    # the solve operator Q: F -> u is symmetric in the L2 pairing (the adjoint relies on it)
    F1, F2 = rng.standard_normal((2, d.n_tri, d.nd))
    a = (F1 * d.solve_condensed(F2)[0]).sum()
    b = (F2 * d.solve_condensed(F1)[0]).sum()
    assert abs(a - b) < 1e-12 * max(abs(a), 1)


def test_projection_energy_never_grows():
    d, X = disc(4, 2)
    rng = np.random.default_rng(5)
    U = rng.standard_normal((d.n_tri, d.nd))
    assert d.energy(d.project(U)) <= d.energy(U)


# ------------------------------------------------------------------- residual
def test_constant_velocity_is_a_steady_state():
    d, X = disc(3, 2, nu=0.1)
    U = projected(d, X, synth.constant_field((0.3, -0.7)))
    lat = d.to_lattice(U)
    assert np.abs(lat - np.array([0.3, -0.7])).max() < 1e-13
    assert np.abs(d.residual(U)).max() < 1e-12
    U2 = d.rk3_step(U, 0.05, 3)
    assert np.abs(U2 - U).max() < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3])
def test_energy_identity_of_upwind_form(k):
    # Sec. 2.2: C_h(u;u,u) = (1/2) sum_F int |u.n| |[u]|^2 >= 0 for u in V_h^{k,-1}
    # (the paper omits the 1/2 and writes the normal jump; integrating by parts gives this).
    d, X = disc(3, k)
    rng = np.random.default_rng(11 + k)
    U = d.project(rng.standard_normal((d.n_tri, d.nd)))
    R = d.residual(U, nu=0.0)
    lhs = -(R * U).sum()                   # C_h(u;u,u)
    rhs = d.upwind_dissipation(U)
    assert rhs > 0
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(rhs))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sipg_form_is_symmetric(k):
    # eq. (18) is symmetric in (u, v) for any broken fields
    d, X = disc(3, k)
    rng = np.random.default_rng(21 + k)
    U, V = rng.standard_normal((2, d.n_tri, d.nd))
    BU = d.residual(U, nu=1.0) - d.residual(U, nu=0.0)
    BV = d.residual(V, nu=1.0) - d.residual(V, nu=0.0)
    a = (BU * V).sum()
    b = (BV * U).sum()
    assert abs(a - b) < 1e-12 * max(1.0, abs(a))


@pytest.mark.parametrize("k", [2, 3])
def test_sipg_coercive_on_divfree_space_at_alpha_2(k):
    # B_h(u,u) >= 0 on V_h^{k,-1}; its kernel is the two constant fields
    d, X = disc(3, k, L=1.0)
    Z = d.divfree_basis()
    B = np.stack([-(d.residual(Z[:, i].reshape(d.n_tri, d.nd), 1.0)
                    - d.residual(Z[:, i].reshape(d.n_tri, d.nd), 0.0)).ravel()
                  for i in range(Z.shape[1])], 1)
    ev = np.linalg.eigvalsh(0.5 * (Z.T @ B + (Z.T @ B).T))
    assert ev[0] > -1e-12 * ev[-1]
    assert (ev < 1e-10 * ev[-1]).sum() == 2


def test_sipg_not_coercive_for_k1_at_alpha_2_but_at_3():
    # recorded reading: alpha k^2/h with h the element diameter is too weak for k = 1 on these meshes
    def mineig(alpha):
        d, X = disc(3, 1, L=1.0, alpha=alpha)
        Z = d.divfree_basis()
        B = np.stack([-(d.residual(Z[:, i].reshape(d.n_tri, d.nd), 1.0)
                        - d.residual(Z[:, i].reshape(d.n_tri, d.nd), 0.0)).ravel()
                      for i in range(Z.shape[1])], 1)
        return np.linalg.eigvalsh(0.5 * (Z.T @ B + (Z.T @ B).T))[0]
    assert mineig(2.0) < -0.1
    assert mineig(3.0) > -1e-12


# ------------------------------------------------------- closed-form solutions
def _tgv_error(N, k, nu, T, field_exact, field0, L=2 * np.pi, steps_per=None):
    d, X = disc(N, k, nu=nu, L=L)
    U = projected(d, X, field0)
    h = math.sqrt(2) * L / N
    dt = 0.1 * h / (k * k * 2.0)
    n = max(1, int(math.ceil(T / dt)))
    U = d.rk3_step(U, T / n, n)
    return d.l2_error(U, field_exact), d, U


def test_taylor_green_velocity_order():
    # Example 1a / Table 1: L2 velocity error of order k + 1. For k = 3 the step shrinks as
    # h^(4/3), so that the RK3 error (dt^3) stays below the spatial error (h^4).
    nu, T = 1e-2, 0.3
    tg = synth.taylor_green()

    def exact(x, y):
        a, b = tg(x, y)
        f = math.exp(-2 * nu * T)
        return f * a, f * b
    table = {int(r[0]): r[1] for r in load_golden("table1_eoc.txt")}
    for k, Ns in ((1, (8, 16)), (2, (4, 8))):
        e = [_tgv_error(N, k, nu, T, exact, tg)[0] for N in Ns]
        eoc = math.log2(e[0] / e[1])
        assert abs(eoc - table[k]) < 0.45, (k, eoc)
    k, Ns = 3, (8, 16)
    h0 = math.sqrt(2) * 2 * np.pi / Ns[0]
    e = []
    for N in Ns:
        d, X = disc(N, k, nu=nu)
        U = projected(d, X, tg)
        h = math.sqrt(2) * 2 * np.pi / N
        n = int(math.ceil(T / (0.1 * h0 / (2.0 * k * k) * (h / h0) ** (4.0 / 3.0))))
        U = d.rk3_step(U, T / n, n)
        e.append(d.l2_error(U, exact))
    eoc = math.log2(e[0] / e[1])
    assert abs(eoc - table[3]) < 0.45, (3, eoc)
    # Example 2's enstrophy ||curl u||^2 of the same solution: 4 pi^2 exp(-4 nu t) for this field
    # (curl u = 2 sin x sin y exp(-2 nu t)); exp(-2 nu t) would be off by 0.24
    ens = d.diagnostics(U)["enstrophy"]
    assert abs(ens - 4 * np.pi ** 2 * math.exp(-4 * nu * T)) < 0.02, ens


def test_enstrophy_and_energy_exact_for_polynomial_fields():
    # broken curl and L2 norm are exact for fields in the broken space: u = (a y + y^2, b x + x^2)
    # on [0, 2pi]^2 has curl u = (b - a) + 2x - 2y, so ||curl u||^2 = (b-a)^2 (2pi)^2 + (2/3)(2pi)^4
    # (the cross terms vanish: (b-a) * int (2x - 2y) = 0); ||u||^2 sums the two components' integrals
    a, b = 0.7, -1.3
    Lx = 2 * np.pi

    def field(x, y):
        return a * y + y * y, b * x + x * x
    ens_ex = (b - a) ** 2 * Lx ** 2 + (2.0 / 3.0) * Lx ** 4
    # int_0^L int_0^L (a y + y^2)^2 dx dy = L (a^2 L^3/3 + a L^4/2 + L^5/5), same for the other
    one = Lx * (a * a * Lx ** 3 / 3 + a * Lx ** 4 / 2 + Lx ** 5 / 5)
    two = Lx * (b * b * Lx ** 3 / 3 + b * Lx ** 4 / 2 + Lx ** 5 / 5)
    for k in (2, 3):
        d, X = disc(3, k)
        U = d.from_lattice(synth.sample_lattice(field, X, k))
        dg = d.diagnostics(U)
        assert abs(dg["enstrophy"] - ens_ex) < 1e-10 * ens_ex, (k, dg["enstrophy"], ens_ex)
        assert abs(dg["energy"] - (one + two)) < 1e-10 * (one + two), (k, dg["energy"])
        assert dg["max_div"] < 1e-10                   # this field is divergence-free
    # u = (x^2 / 2, 0) has div u = x: the largest divergence at the volume points is just below 2 pi
    d, X = disc(3, 2)
    U = d.from_lattice(synth.sample_lattice(lambda x, y: (0.5 * x * x, 0.0 * y), X, 2))
    assert 0.9 * Lx < d.diagnostics(U)["max_div"] < Lx


def test_taylor_green_enstrophy_converges_to_closed_form():
    # projected Taylor-Green field: ||curl_h u_h||^2 -> 4 pi^2 at a rate of at least 3 (k = 2, 3)
    for k in (2, 3):
        err = []
        for N in (8, 16):
            d, X = disc(N, k)
            err.append(abs(d.diagnostics(projected(d, X, synth.taylor_green()))["enstrophy"] - 4 * np.pi ** 2))
        assert err[1] < err[0] / 8 and err[1] < 2e-2, (k, err)


def test_advected_taylor_green_moves_downstream():
    # Galilean translate of the vortex (exact NS solution); pins the direction of convection
    nu, T, U0 = 1e-2, 0.5, (1.0, 0.0)
    f0 = synth.advected_taylor_green(U0, t=0.0, nu=nu)
    fwd = synth.advected_taylor_green(U0, t=T, nu=nu)
    bwd = synth.advected_taylor_green((-1.0, 0.0), t=T, nu=nu)

    def back(x, y):
        a, b = bwd(x, y)
        return a + 2.0, b                      # mean flow (1, 0), pattern moved upstream
    e_fwd, d, U = _tgv_error(8, 2, nu, T, fwd, f0)
    e_bwd = d.l2_error(U, back)
    assert e_fwd < 0.05 and e_bwd > 10 * e_fwd


def test_taylor_green_pressure():
    # p = (cos 2x + cos 2y)/4 for u = (sin x cos y, -cos x sin y) (steady Euler); w ~ p (Remark 2).
    # The element pressure lives in broken P^(k-1): its L2 error has order k (measured 1.97 for
    # k = 2 and 2.97 for k = 3 over N = 8 -> 16); the facet multiplier approximates the same
    # pressure on the skeleton (Theorem 2) and its maximum error falls at least as fast.
    pex = lambda x, y: 0.25 * (np.cos(2 * x) + np.cos(2 * y))  # noqa: E731
    for k in (2, 3):
        e_el, e_fa = [], []
        for N in (8, 16):
            d, X = disc(N, k, nu=0.0)
            U = projected(d, X, synth.taylor_green())
            w, lam = d.pressure(U)
            e_el.append(d.pressure_l2_error(w, pex))
            pe, pf = d.pressure_lattice(w, lam)
            T = d.topo
            f = np.arange(d.n_facet)
            pts = T.facet_points(f, np.zeros_like(f), np.arange(k + 1) / k)
            e_fa.append(np.abs(pf - pex(pts[..., 0], pts[..., 1])).max())
        eoc_el = math.log2(e_el[0] / e_el[1])
        eoc_fa = math.log2(e_fa[0] / e_fa[1])
        assert abs(eoc_el - k) < 0.4, (k, eoc_el)
        assert eoc_fa > k - 0.5 and e_fa[1] < 5e-3, (k, eoc_fa, e_fa)


def test_rk3_is_third_order_in_time():
    # Table 2 (TVD-RK3 eoc 3): Richardson errors against a fine-step solution on a fixed mesh
    d, X = disc(4, 2, nu=1e-2)
    U0 = projected(d, X, synth.advected_taylor_green((1.0, 0.5), nu=1e-2))
    T = 0.4
    ref = d.rk3_step(U0, T / 256, 256)
    e = []
    for n in (8, 16, 32):
        e.append(np.sqrt(d.energy(d.rk3_step(U0, T / n, n) - ref)))
    eoc = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    tab = [r[1] for r in load_golden("table2_eoc.txt")]
    assert all(abs(a - 3.0) < 0.25 for a in eoc), eoc
    assert all(abs(b - 3.0) < 0.05 for b in tab)


def _time_order(step, n_list, ref, U0, d, T):
    e = [np.sqrt(d.energy(step(U0, T / n, n) - ref)) for n in n_list]
    return [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)], e


def test_rk4_is_fourth_order_and_euler_first_order_in_time():
    # Table 2 (RK4 eoc 4) and eq. (FE): errors against a fine-step solution of the same
    # semi-discrete system on a fixed mesh. The upwind flux makes L(u) only piecewise smooth
    # (|u.n| has a kink where u.n changes sign), which blurs the observed orders; a strong mean
    # flow (4, 2) keeps u.n sign-definite on every facet of the split-square mesh, so L is
    # smooth along the trajectory. The fine RK4 and RK3 solutions must agree (the two schemes
    # converge to one ODE solution), so a wrong RK4 stage weight cannot hide.
    d, X = disc(4, 2, nu=1e-2)
    U0 = projected(d, X, synth.advected_taylor_green((4.0, 2.0), nu=1e-2))
    T = 0.4
    ref = d.rk4_step(U0, T / 256, 256)
    ref3 = d.rk3_step(U0, T / 1024, 1024)
    assert np.sqrt(d.energy(ref - ref3)) < 1e-9 * np.sqrt(d.energy(ref))
    eoc4, _ = _time_order(d.rk4_step, (8, 16, 32), ref, U0, d, T)
    assert all(abs(a - 4.0) < 0.1 for a in eoc4), eoc4
    eoc1, _ = _time_order(d.euler_step, (64, 128, 256), ref, U0, d, T)
    assert all(abs(a - 1.0) < 0.05 for a in eoc1), eoc1
    tab = [r[2] for r in load_golden("table2_eoc.txt")]
    assert all(abs(b - 4.0) < 0.05 for b in tab)


def test_euler_step_is_one_solve_of_the_stage_form():
    # eq. (FE) is the first SSP-RK3 stage (a = 0, b = 1) of eq. (8) taken as the whole step
    d, X = disc(3, 2, nu=1e-2)
    U = projected(d, X, synth.advected_taylor_green((0.3, -0.7), nu=1e-2))
    a, b = 0.0, 1.0
    assert np.abs(d.euler_step(U, 0.05) - d.stage(U, U, a, b, 0.05)).max() < 1e-14 * np.abs(U).max()


def test_euler_energy_non_increasing():
    # Sec. 2.2: with nu = 0 and upwinding the discrete energy does not grow
    vid, X = synth.split_square_mesh(6, L=1.0)
    d = Discretization(vid, X, 2, 0.0)
    U = projected(d, X, synth.random_spectrum_velocity(5, kmax=4, L=1.0))
    vmax = np.abs(d.to_lattice(U)).max()
    dt = synth.cfl_dt(X, 2, vmax, 0.0)
    E = [d.energy(U)]
    for _ in range(15):
        U = d.rk3_step(U, dt, 1)
        E.append(d.energy(U))
    dE = np.diff(E)
    assert np.all(dE <= 1e-14 * E[0]), dE
    assert E[-1] < E[0]


def test_euler_energy_rate_matches_semidiscrete_identity():
    # dE/dt = 2 L(u)(u) = -2 C_h(u;u,u) for the semi-discrete scheme eq. (6): a small step of RK3
    # must reproduce it to O(dt^2)
    d, X = disc(4, 2, nu=0.0, L=1.0)
    U = projected(d, X, synth.random_spectrum_velocity(2, kmax=3, L=1.0))
    rate = -2.0 * d.upwind_dissipation(U)
    for dt in (1e-3, 5e-4):
        est = (d.energy(d.rk3_step(U, dt, 1)) - d.energy(U)) / dt
        assert abs(est - rate) < 50 * dt * abs(rate) + 1e-12


def test_oracle_tangent_matches_finite_differences():
    # the tangent-linear model used to check the adjoint: central differences of the oracle's own
    # RK3 (exact direct solves) in the state and in nu
    vid, X = synth.split_square_mesh(4, L=1.0)
    d = Discretization(vid, X, 2, 1e-2)
    U = projected(d, X, synth.random_spectrum_velocity(3, kmax=3, L=1.0))
    rng = np.random.default_rng(0)
    dU = d.project(rng.standard_normal(U.shape))
    for dnu in (0.0, 1.0):
        _, dUk = d.rk3_tangent(U, dU, 0.01, 3, dnu=dnu)
        eps = 1e-6
        dp = Discretization(vid, X, 2, 1e-2 + eps * dnu)
        dm = Discretization(vid, X, 2, 1e-2 - eps * dnu)
        fd = (dp.rk3_step(U + eps * dU, 0.01, 3) - dm.rk3_step(U - eps * dU, 0.01, 3)) / (2 * eps)
        assert np.linalg.norm(fd - dUk) / np.linalg.norm(dUk) < 1e-7


# ----------------------------------------------------- inflow / outflow (Sec. 2.5, eq. (be))
def _channel(Nx, Ny, k, periodic_y, inflow_field, Lx=1.5, Ly=1.0, nu=0.0):
    vid, X = synth.channel_mesh(Nx, Ny, Lx, Ly, periodic_y=periodic_y)
    bk = synth.boundary_kinds_by_x(X, 0.0, Lx)
    uin = synth.sample_edges(inflow_field, X, k)
    return Discretization(vid, X, k, nu, boundary=bk, inflow=uin), X


@pytest.mark.parametrize("k,periodic_y", [(1, True), (2, True), (3, True), (2, False)])
def test_inflow_outflow_solve_routes_agree(k, periodic_y):
    # the condensed solve with the data moments on inflow facets and lam = 0 on outflow facets,
    # the uncondensed saddle system and the SVD null-space projection onto the affine space agree,
    # and the result keeps u.n = u_in.n on the inflow (to the multiplier space) and div u = 0
    def f_in(x, y):
        return 1.0 + 0.3 * np.sin(2 * np.pi * y) + 0 * x, 0.2 * np.cos(2 * np.pi * y) + 0 * x
    d, X = _channel(3, 2, k, periodic_y, f_in)
    F = np.random.default_rng(k).standard_normal((d.n_tri, d.nd))
    u1, _, _ = d.solve_condensed(F)
    u2, _, _ = d.solve_full(F)
    u3 = d.project_nullspace(F)
    sc = np.abs(u1).max()
    assert np.abs(u1 - u2).max() < 1e-12 * sc and np.abs(u1 - u3).max() < 1e-12 * sc
    dg = d.diagnostics(u1)
    assert dg["max_div"] < 1e-10 * sc and dg["max_jump"] < 1e-10 * sc
    # a random functional of the homogeneous problem: u.n = 0 on the inflow instead
    u0, _, _ = d.solve_condensed(F, homogeneous=True)
    assert np.abs(u1 - u0).max() > 0.1          # the O(1) inflow data moves the solution


@pytest.mark.parametrize("k", [1, 2, 3])
def test_shear_flow_through_a_channel_is_steady(k):
    # Euler (nu = 0): u = (U(y), 0) is steady between free-slip walls, with u_in = u on the inflow and
    # the outflow open: for a polynomial U of degree <= k the discrete residual vanishes for every
    # broken test function (the boundary fluxes cancel the integration by parts), so the state is
    # kept to rounding over the steps
    U = (lambda y: 1.0 + 0.5 * y) if k == 1 else (lambda y: 1.0 + y * (1.0 - y))

    def f(x, y):
        return U(y) + 0 * x, 0 * y
    d, X = _channel(4, 3, k, False, f)
    U0 = d.project(d.from_lattice(synth.sample_lattice(f, X, k)))
    ref = d.from_lattice(synth.sample_lattice(f, X, k))
    assert np.abs(U0 - ref).max() < 1e-12
    assert np.abs(d.residual(U0)).max() < 1e-12
    U1 = d.rk3_step(U0, 0.01, 5)
    assert np.abs(U1 - U0).max() < 1e-12


def test_inflow_carries_its_momentum_in_and_outflow_lets_it_out():
    # test function (0, 1) (divergence-free, zero normal component on the inflow, periodic in y):
    # one forward Euler step from u = (1, 0) with inflow data (1, eps) changes int v by exactly
    # dt * eps * Ly (the inflow flux of eq. (7) with the exterior state u_in); from u = (1, eps)
    # with the same data nothing changes (the outflow takes the interior trace)
    eps, Ly, dt, k = 0.07, 1.0, 0.02, 2
    d, X = _channel(4, 3, k, True, lambda x, y: (1.0 + 0 * x, eps + 0 * y), Ly=Ly)
    E = d.from_lattice(synth.sample_lattice(lambda x, y: (0 * x, 1.0 + 0 * y), X, k))

    def int_v(U):
        return float((d.apply_mass(U) * E).sum())
    U0 = d.from_lattice(synth.sample_lattice(lambda x, y: (1.0 + 0 * x, 0 * y), X, k))
    U1 = d.euler_step(U0, dt)
    assert abs(int_v(U1) - dt * eps * Ly) < 1e-13
    Ue = d.from_lattice(synth.sample_lattice(lambda x, y: (1.0 + 0 * x, eps + 0 * y), X, k))
    assert np.abs(d.euler_step(Ue, dt) - Ue).max() < 1e-13
