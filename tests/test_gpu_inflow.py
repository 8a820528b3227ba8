"""Inflow and outflow boundaries (Sec. 2.5, eq. (be)) on channel meshes: the CUDA path through the
C ABI (dg_mesh_create_ex, dg_set_inflow) against the FP64 oracle on the same seeded inputs.

Channels are split-square triangulations of [0, Lx] x [0, Ly] with the inflow on x = 0 and the
outflow on x = Lx, either periodic in y or with free-slip walls at y = 0 and y = Ly. Tolerances
(relative L2 over lattice values): 1e-12 for the FP64 form, 1e-9 for the mixed form.
"""
import numpy as np
import pytest

import synth
from oracle import Discretization

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 1e-9


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1808_04669_gb300 import build
    build.build()
    import paper_1808_04669_gb300 as pkg
    return pkg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def f_in(x, y):
    """Inflow profile: periodic in y with period 1, mostly entering (u_x > 0)."""
    return 1.0 + 0.3 * np.sin(2 * np.pi * y) + 0 * x, 0.2 * np.cos(2 * np.pi * y) + 0 * x


def channel(Nx, Ny, k, periodic_y, field=f_in, Lx=1.5, Ly=1.0):
    vid, X = synth.channel_mesh(Nx, Ny, Lx, Ly, periodic_y=periodic_y)
    bk = synth.boundary_kinds_by_x(X, 0.0, Lx)
    uin = synth.sample_edges(field, X, k)
    return vid, X, bk, uin


def start_field(X, k, seed, Lx=1.5):
    """Smooth channel flow plus a seeded random perturbation (lattice values)."""
    base = synth.sample_lattice(lambda x, y: (1.0 + 0.2 * np.sin(2 * np.pi * y) + 0 * x,
                                              0.1 * np.sin(np.pi * x / Lx) + 0 * y), X, k)
    rng = np.random.default_rng(seed)
    return base + 0.2 * rng.standard_normal(base.shape)


@pytest.mark.parametrize("k,periodic_y,precond", [(1, True, 0), (2, True, 0), (3, True, 0), (2, False, 0),
                                                  (2, True, 1), (3, False, 1), (3, False, 2)])
def test_projection_parity_channel(g, k, periodic_y, precond):
    # the L2 projection onto the affine space u.n = u_in.n on the inflow, lam = 0 on the outflow
    vid, X, bk, uin = channel(5, 4, k, periodic_y)
    d = Discretization(vid, X, k, 0.0, boundary=bk, inflow=uin)
    v = start_field(X, k, 11 + k)
    ref = d.to_lattice(d.project(d.from_lattice(v)))
    for prec, tol in ((0, TOL64), (1, TOLMIX)):
        mesh = g.DGMesh(vid, X, k, 0.0, precision=prec, precond=precond, boundary=bk, inflow=uin)
        mesh.set_velocity(v)
        mesh.project_divfree()
        assert rel(mesh.get_velocity(), ref) < tol, prec
        dg = mesh.diagnostics()
        # inflow facets: the jump against the data is (u - u_in).n, zero up to the multiplier space
        # (u_in is a polynomial of degree k on every edge, so exactly); outflow facets are free
        assert dg["max_jump"] < 1e-10 and dg["max_div"] < 1e-10, prec


@pytest.mark.parametrize("k,periodic_y,nu", [(1, True, 0.0), (2, False, 1e-2), (3, True, 1e-3)])
def test_residual_parity_channel(g, k, periodic_y, nu):
    # L(u) with the boundary convective fluxes: exterior state u_in on inflow facets, the interior
    # trace on outflow facets, no viscous boundary terms
    vid, X, bk, uin = channel(4, 3, k, periodic_y)
    d = Discretization(vid, X, k, nu, boundary=bk, inflow=uin)
    v = start_field(X, k, 3 + k)
    mesh = g.DGMesh(vid, X, k, nu, boundary=bk, inflow=uin)
    mesh.set_velocity(v)
    ref = d.to_lattice(d.riesz(d.residual(d.from_lattice(v))))
    assert rel(mesh.eval_residual(), ref) < TOL64


@pytest.mark.parametrize("k,periodic_y,precond", [(1, True, 0), (2, True, 0), (3, True, 0), (2, False, 0),
                                                  (3, False, 1)])
def test_rk3_parity_channel(g, k, periodic_y, precond):
    # SSP-RK3 steps through a channel, FP64 and mixed forms, multilevel (AUTO) and block-Jacobi
    # preconditioners, against the oracle's exact solves
    nu = 1e-3
    vid, X, bk, uin = channel(6, 4, k, periodic_y)
    v = start_field(X, k, 21 + k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((v ** 2).sum(-1)).max()), nu)
    d = Discretization(vid, X, k, nu, boundary=bk, inflow=uin)
    U = d.rk3_step(d.project(d.from_lattice(v)), dt, 4)
    ref = d.to_lattice(U)
    od = d.diagnostics(U)
    for prec, tol in ((0, TOL64), (1, TOLMIX)):
        mesh = g.DGMesh(vid, X, k, nu, precision=prec, precond=precond, boundary=bk, inflow=uin)
        mesh.set_velocity(v)
        mesh.project_divfree()
        mesh.rk3_step(dt, 4)
        assert rel(mesh.get_velocity(), ref) < tol, prec
        dg = mesh.diagnostics()
        assert abs(dg["energy"] - od["energy"]) < 1e-9 * od["energy"], prec
        assert dg["max_jump"] < 1e-10, prec
        st = mesh.solver_stats()
        assert st["lattice"] == 0.0


@pytest.mark.parametrize("precision", [0, 1])
def test_rk3_parity_channel_multilevel_larger(g, precision):
    # 48 x 16 channel with walls, BDM_3: several aggregation levels, isolated outflow rows left out
    # of the aggregates; 3 steps
    k, nu = 3, 1e-3
    vid, X, bk, uin = channel(48, 16, k, False, Lx=3.0)
    v = start_field(X, k, 5, Lx=3.0)
    dt = synth.cfl_dt(X, k, float(np.sqrt((v ** 2).sum(-1)).max()), nu)
    d = Discretization(vid, X, k, nu, boundary=bk, inflow=uin)
    ref = d.to_lattice(d.rk3_step(d.project(d.from_lattice(v)), dt, 3))
    mesh = g.DGMesh(vid, X, k, nu, precision=precision, boundary=bk, inflow=uin)
    assert mesh.solver_stats()["precond_kind"] == 2.0
    mesh.set_velocity(v)
    mesh.project_divfree()
    mesh.rk3_step(dt, 3)
    assert rel(mesh.get_velocity(), ref) < (TOL64 if precision == 0 else TOLMIX)
    st = mesh.solver_stats()
    assert st["total_iters"] / st["solves"] < 60


@pytest.mark.parametrize("k", [1, 2, 3])
def test_shear_flow_through_a_channel_is_steady(g, k):
    # Euler: u = (U(y), 0) between free-slip walls with u_in = u and an open outflow is a discrete
    # steady state for polynomial U of degree <= k (the oracle pins the same)
    U = (lambda y: 1.0 + 0.5 * y) if k == 1 else (lambda y: 1.0 + y * (1.0 - y))

    def f(x, y):
        return U(y) + 0 * x, 0 * y
    vid, X, bk, uin = channel(4, 3, k, False, field=f)
    vals = synth.sample_lattice(f, X, k)
    for prec, tol in ((0, 1e-12), (1, 1e-10)):
        mesh = g.DGMesh(vid, X, k, 0.0, precision=prec, boundary=bk, inflow=uin)
        mesh.set_velocity(vals)
        mesh.project_divfree()
        assert np.abs(mesh.get_velocity() - vals).max() < tol, prec
        mesh.rk3_step(0.01, 5)
        assert np.abs(mesh.get_velocity() - vals).max() < tol, prec


def test_pressure_parity_channel(g):
    # pressure of L(u) alone: u.n = 0 on the inflow, and no mean shift (p = 0 on the outflow)
    k, nu = 2, 1e-2
    vid, X, bk, uin = channel(5, 4, k, True)
    d = Discretization(vid, X, k, nu, boundary=bk, inflow=uin)
    v = start_field(X, k, 8)
    U = d.project(d.from_lattice(v))
    w, lam = d.pressure(U)
    pe_ref, pf_ref = d.pressure_lattice(w, lam)
    mesh = g.DGMesh(vid, X, k, nu, boundary=bk, inflow=uin)
    mesh.set_velocity(v)
    mesh.project_divfree()
    pe, pf = mesh.get_pressure()
    assert rel(pe, pe_ref) < 1e-11 and rel(pf, pf_ref) < 1e-11


def test_inflow_data_can_change_between_steps(g):
    # dg_set_inflow replaces the data of a live mesh: the next steps follow the oracle built with
    # the new data from the same state
    k, nu = 2, 1e-3
    vid, X, bk, uin = channel(5, 4, k, True)
    uin2 = synth.sample_edges(lambda x, y: (0.7 + 0.1 * np.cos(2 * np.pi * y) + 0 * x, 0 * x + 0.05), X, k)
    v = start_field(X, k, 9)
    dt = synth.cfl_dt(X, k, float(np.sqrt((v ** 2).sum(-1)).max()), nu)
    d1 = Discretization(vid, X, k, nu, boundary=bk, inflow=uin)
    d2 = Discretization(vid, X, k, nu, boundary=bk, inflow=uin2)
    U = d2.rk3_step(d1.rk3_step(d1.project(d1.from_lattice(v)), dt, 2), dt, 2)
    mesh = g.DGMesh(vid, X, k, nu, boundary=bk, inflow=uin)
    mesh.set_velocity(v)
    mesh.project_divfree()
    mesh.rk3_step(dt, 2)
    mesh.set_inflow(uin2)
    mesh.rk3_step(dt, 2)
    assert rel(mesh.get_velocity(), d2.to_lattice(U)) < TOL64


def test_boundary_argument_errors(g):
    k = 2
    vid, X, bk, uin = channel(3, 2, k, True)
    bad = bk.copy()
    bad[bk == 1] = 3
    with pytest.raises(g.DGError) as e:
        g.DGMesh(vid, X, k, 0.0, boundary=bad)
    assert e.value.code == -1
    # no inflow facets: dg_set_inflow is refused
    walls = np.where(bk == 1, 0, bk).astype(np.int8)
    mesh = g.DGMesh(vid, X, k, 0.0, boundary=walls)
    with pytest.raises(g.DGError) as e:
        mesh.set_inflow(uin)
    assert e.value.code == -1
    # non-finite data
    mesh = g.DGMesh(vid, X, k, 0.0, boundary=bk)
    u_bad = uin.copy()
    u_bad[0, 0, 0, 0] = np.nan
    with pytest.raises(g.DGError):
        mesh.set_inflow(u_bad)
    # the adjoint does not cover inflow / outflow boundaries
    mesh.set_inflow(uin)
    with pytest.raises(g.DGError) as e:
        mesh.rk3_vjp(0.01, 1, np.zeros((mesh.n_tri, 2 * mesh.n_lat)))
    assert e.value.code == -3


@pytest.mark.parametrize("scheme", ["EULER", "RK4"])
def test_euler_and_rk4_parity_channel(g, scheme):
    # forward Euler and classical RK4 through dg_step: every stage solve imposes the full inflow
    # data (the stage's state coefficients sum to one), as the oracle's forms do
    k, nu = 2, 1e-3
    vid, X, bk, uin = channel(5, 4, k, False)
    v = start_field(X, k, 17)
    dt = synth.cfl_dt(X, k, float(np.sqrt((v ** 2).sum(-1)).max()), nu)
    d = Discretization(vid, X, k, nu, boundary=bk, inflow=uin)
    U0 = d.project(d.from_lattice(v))
    ref = d.to_lattice((d.euler_step if scheme == "EULER" else d.rk4_step)(U0, dt, 3))
    for prec, tol in ((0, TOL64), (1, TOLMIX)):
        mesh = g.DGMesh(vid, X, k, nu, precision=prec, boundary=bk, inflow=uin)
        mesh.set_velocity(v)
        mesh.project_divfree()
        mesh.step(dt, 3, scheme=getattr(g, scheme))
        assert rel(mesh.get_velocity(), ref) < tol, prec
