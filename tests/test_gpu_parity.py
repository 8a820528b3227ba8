"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on the same seeded inputs.

Tolerances (relative L2 over all lattice values): 1e-12 for the FP64 form,
1e-9 for the mixed-precision form.
"""
import math

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


def pair(g, N, k, nu, L=2 * np.pi, precision=0, perturb=0.0, seed=0, **kw):
    vid, X = synth.split_square_mesh(N, L=L)
    if perturb:
        rng = np.random.default_rng(seed)
        X = X + (perturb * L / N * rng.uniform(-1, 1, size=(N * N, 2)))[vid]
    mesh = g.DGMesh(vid, X, k, nu, precision=precision, **kw)
    d = Discretization(vid, X, k, nu)
    return mesh, d, X


def random_lattice(n_tri, k, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_tri, (k + 1) * (k + 2) // 2, 2))


# ------------------------------------------------------------------- basics
@pytest.mark.parametrize("k", [1, 2, 3])
def test_lattice_roundtrip(g, k):
    mesh, d, X = pair(g, 3, k, 0.0)
    v = random_lattice(mesh.n_tri, k, 1)
    mesh.set_velocity(v)
    assert np.abs(mesh.get_velocity() - v).max() < 1e-13


def test_mesh_info_uniform_classes(g):
    mesh, d, X = pair(g, 8, 2, 0.0)
    assert mesh.n_tri == 128 and mesh.n_facet == 192
    assert mesh.n_class == 2 and mesh.n_stencil == 3


# ----------------------------------------------------------------- residual
@pytest.mark.parametrize("N,k,nu,perturb", [(1, 1, 0.0, 0.0), (2, 2, 0.05, 0.0), (3, 3, 0.01, 0.0),
                                            (5, 2, 0.02, 0.0), (4, 3, 0.0, 0.12), (3, 1, 0.3, 0.1)])
def test_residual_parity(g, N, k, nu, perturb):
    mesh, d, X = pair(g, N, k, nu, perturb=perturb, seed=N)
    v = random_lattice(mesh.n_tri, k, 10 + N)
    mesh.set_velocity(v)
    gpu = mesh.eval_residual()
    U = d.from_lattice(v)
    ref = d.to_lattice(d.riesz(d.residual(U)))
    assert rel(gpu, ref) < TOL64


@pytest.mark.parametrize("k", [2, 3])
def test_residual_parity_projected_field(g, k):
    # divergence-free field: u.n is continuous, so the upwind side is decided by the traces' average
    mesh, d, X = pair(g, 6, k, 1e-3)
    v = random_lattice(mesh.n_tri, k, 33)
    mesh.set_velocity(v)
    mesh.project_divfree()
    U = d.project(d.from_lattice(v))
    gpu = mesh.eval_residual()
    ref = d.to_lattice(d.riesz(d.residual(U)))
    assert rel(gpu, ref) < TOL64


# --------------------------------------------------------------- projection
@pytest.mark.parametrize("N,k,perturb,precond", [(1, 1, 0.0, 0), (2, 3, 0.0, 0), (4, 2, 0.0, 0), (4, 2, 0.0, 1),
                                                  (5, 3, 0.0, 0), (5, 3, 0.0, 1), (4, 2, 0.1, 0), (8, 3, 0.0, 0)])
def test_projection_parity(g, N, k, perturb, precond):
    mesh, d, X = pair(g, N, k, 0.0, perturb=perturb, seed=3, precond=precond)
    v = random_lattice(mesh.n_tri, k, 20 + N)
    mesh.set_velocity(v)
    mesh.project_divfree()
    gpu = mesh.get_velocity()
    ref = d.to_lattice(d.project(d.from_lattice(v)))
    assert rel(gpu, ref) < TOL64
    dg = mesh.diagnostics()
    assert dg["max_div"] < 1e-11 * max(1.0, np.abs(ref).max()) * N
    assert dg["max_jump"] < 1e-10


def test_projection_idempotent_and_orthogonal(g):
    mesh, d, X = pair(g, 8, 3, 0.0)
    v = random_lattice(mesh.n_tri, 3, 5)
    mesh.set_velocity(v)
    e0 = mesh.diagnostics()["energy"]
    mesh.project_divfree()
    u1 = mesh.get_velocity()
    e1 = mesh.diagnostics()["energy"]
    mesh.project_divfree()
    u2 = mesh.get_velocity()
    assert rel(u2, u1) < 1e-12
    assert e1 <= e0


# ------------------------------------------------------------------- RK3
@pytest.mark.parametrize("precond", [0, 1])
def test_rk3_parity_taylor_green_n8_k2(g, precond):
    # Taylor-Green, 8x8 split squares, BDM_2, nu = 1e-2, 100 SSP-RK3 steps, FP64; lattice (Fourier)
    # preconditioner and block Jacobi
    vid, X, vals, dt = synth.make_workload("tgv_n8_k2")
    mesh = g.DGMesh(vid, X, 2, 1e-2, precond=precond)
    assert mesh.solver_stats()["lattice"] == (1.0 if precond == 0 else 0.0)
    d = Discretization(vid, X, 2, 1e-2)
    mesh.set_velocity(vals)
    mesh.project_divfree()
    mesh.rk3_step(dt, 100)
    gpu = mesh.get_velocity()
    U = d.rk3_step(d.project(d.from_lattice(vals)), dt, 100)
    ref = d.to_lattice(U)
    assert rel(gpu, ref) < TOL64
    # closed form u(t) = u0 exp(-2 nu t): the GPU error equals the oracle's
    T = 100 * dt
    ex = synth.sample_lattice(synth.taylor_green(), X, 2) * math.exp(-2e-2 * T)
    assert abs(rel(gpu, ex) - rel(ref, ex)) < 1e-9
    dg = mesh.diagnostics()
    assert dg["max_jump"] < 1e-11 and dg["max_div"] < 1e-11


@pytest.mark.parametrize("N,k,precond", [(12, 1, 0), (12, 3, 0), (12, 3, 1), (16, 3, 0), (8, 2, 0)])
def test_rk3_parity_shear_layer(g, N, k, precond):
    # lattice preconditioner: radix-2 FFT (N = 8, 16) or direct DFT (N = 12); block Jacobi (precond = 1)
    nu = 1e-4
    vid, X = synth.split_square_mesh(N)
    vals = synth.sample_lattice(synth.double_shear_layer(), X, k)
    vmax = float(np.sqrt((vals ** 2).sum(-1)).max())
    dt = synth.cfl_dt(X, k, vmax, nu)
    d = Discretization(vid, X, k, nu)
    U = d.rk3_step(d.project(d.from_lattice(vals)), dt, 5)
    ref = d.to_lattice(U)
    for prec, tol in ((0, TOL64), (1, TOLMIX)):
        mesh = g.DGMesh(vid, X, k, nu, precision=prec, precond=precond)
        mesh.set_velocity(vals)
        mesh.project_divfree()
        mesh.rk3_step(dt, 5)
        assert rel(mesh.get_velocity(), ref) < tol, prec
        st = mesh.solver_stats()
        assert st["lattice"] == (1.0 if precond == 0 else 0.0)
        if st["lattice"]:
            assert st["total_iters"] / st["solves"] <= 6


# ------------------------------------------------------- other explicit schemes
@pytest.mark.parametrize("scheme", ["EULER", "RK4"])
@pytest.mark.parametrize("N,k,precond", [(8, 2, 0), (12, 3, 0), (6, 3, 1)])
def test_scheme_parity_shear_layer(g, scheme, N, k, precond):
    # forward Euler (eq. (FE)) and classical RK4 (Example 1b) through dg_step, against the
    # oracle's own forms (one solve per Euler step; RK4 from the four projected slopes)
    nu = 1e-3
    vid, X = synth.split_square_mesh(N)
    vals = synth.sample_lattice(synth.double_shear_layer(), X, k)
    vmax = float(np.sqrt((vals ** 2).sum(-1)).max())
    dt = synth.cfl_dt(X, k, vmax, nu)
    d = Discretization(vid, X, k, nu)
    U0 = d.project(d.from_lattice(vals))
    ref = d.to_lattice((d.euler_step if scheme == "EULER" else d.rk4_step)(U0, dt, 4))
    for prec, tol in ((0, TOL64), (1, TOLMIX)):
        mesh = g.DGMesh(vid, X, k, nu, precision=prec, precond=precond)
        mesh.set_velocity(vals)
        mesh.project_divfree()
        mesh.step(dt, 4, scheme=getattr(g, scheme))
        assert rel(mesh.get_velocity(), ref) < tol, prec
        dg = mesh.diagnostics()
        assert dg["max_jump"] < 1e-10 and dg["max_div"] < 1e-10


def test_scheme_switching_parity(g):
    # RK3, RK4, Euler and RK3 again on one mesh: each switch drops the multiplier history of
    # the previous scheme's stages (warm starts only), the results follow the oracle
    N, k, nu = 8, 3, 1e-3
    vid, X = synth.split_square_mesh(N)
    vals = synth.sample_lattice(synth.double_shear_layer(), X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((vals ** 2).sum(-1)).max()), nu)
    d = Discretization(vid, X, k, nu)
    U = d.project(d.from_lattice(vals))
    U = d.rk3_step(U, dt, 2)
    U = d.rk4_step(U, dt, 2)
    U = d.euler_step(U, 0.5 * dt, 1)
    U = d.rk3_step(U, dt, 2)
    ref = d.to_lattice(U)
    for prec, tol in ((0, TOL64), (1, TOLMIX)):
        mesh = g.DGMesh(vid, X, k, nu, precision=prec)
        mesh.set_velocity(vals)
        mesh.project_divfree()
        mesh.rk3_step(dt, 2)
        mesh.step(dt, 2, scheme=g.RK4)
        mesh.step(0.5 * dt, 1, scheme=g.EULER)
        mesh.step(dt, 2, scheme=g.SSPRK3)
        assert rel(mesh.get_velocity(), ref) < tol, prec


def test_step_rejects_unknown_scheme(g):
    from paper_1808_04669_gb300 import DGError
    mesh, d, X = pair(g, 2, 1, 0.0)
    with pytest.raises(DGError) as e:
        mesh.step(0.01, 1, scheme=7)
    assert e.value.code == -1


# ------------------------------------------------------- walls (free slip)
def box(g, N, k, nu, precision=0):
    vid, X = synth.split_square_mesh(N, L=1.0, periodic=False)
    return g.DGMesh(vid, X, k, nu, precision=precision), Discretization(vid, X, k, nu), X


@pytest.mark.parametrize("k", [1, 2, 3])
def test_wall_projection_parity(g, k):
    # a random field in a box: the projection has no normal velocity on the walls
    for prec, tol in ((0, TOL64), (1, TOLMIX)):
        mesh, d, X = box(g, 3, k, 0.0, prec)
        v = random_lattice(mesh.n_tri, k, 11 + k)
        mesh.set_velocity(v)
        mesh.project_divfree()
        ref = d.to_lattice(d.project(d.from_lattice(v)))
        assert rel(mesh.get_velocity(), ref) < tol, prec
        assert mesh.solver_stats()["lattice"] == 0.0
        dg = mesh.diagnostics()
        assert dg["max_jump"] < 1e-11 and dg["max_div"] < 1e-10


@pytest.mark.parametrize("k", [2, 3])
def test_wall_taylor_green_cell_rk3_parity(g, k):
    # Taylor-Green cell on the unit square with free-slip walls, 12 SSP-RK3 steps
    nu = 1e-2
    vid, X = synth.split_square_mesh(6, L=1.0, periodic=False)
    vals = synth.sample_lattice(synth.taylor_green(L=2.0), X, k)
    dt = synth.cfl_dt(X, k, float(np.abs(vals).max()), nu)
    d = Discretization(vid, X, k, nu)
    U = d.rk3_step(d.project(d.from_lattice(vals)), dt, 12)
    ref = d.to_lattice(U)
    od = d.diagnostics(U)
    for prec, tol in ((0, TOL64), (1, TOLMIX)):
        mesh = g.DGMesh(vid, X, k, nu, precision=prec)
        mesh.set_velocity(vals)
        mesh.project_divfree()
        mesh.rk3_step(dt, 12)
        assert rel(mesh.get_velocity(), ref) < tol, prec
        dg = mesh.diagnostics()
        assert abs(dg["energy"] - od["energy"]) < 1e-9 * od["energy"]
        assert dg["max_jump"] < 1e-11


def test_wall_rk4_and_pressure_parity(g):
    # RK4 through dg_step and the pressure of the final state, with walls
    k, nu = 2, 1e-3
    vid, X = synth.split_square_mesh(5, L=1.0, periodic=False)
    vals = synth.sample_lattice(synth.random_spectrum_velocity(3, kmax=3, L=1.0), X, k)
    dt = synth.cfl_dt(X, k, float(np.abs(vals).max()), nu)
    d = Discretization(vid, X, k, nu)
    U = d.rk4_step(d.project(d.from_lattice(vals)), dt, 3)
    w, lam = d.pressure(U)
    pe_ref, pf_ref = d.pressure_lattice(w, lam)
    mesh = g.DGMesh(vid, X, k, nu)
    mesh.set_velocity(vals)
    mesh.project_divfree()
    mesh.step(dt, 3, scheme=g.RK4)
    assert rel(mesh.get_velocity(), d.to_lattice(U)) < TOL64
    pe, pf = mesh.get_pressure()
    assert rel(pe, pe_ref) < 1e-11 and rel(pf, pf_ref) < 1e-11


# --------------------------------------------------------- tensor-core (tcgen05) recovery
@pytest.mark.parametrize("N,k,walls", [(8, 1, False), (12, 2, False), (16, 3, False), (6, 3, True), (130, 3, False)])
def test_tensor_core_recovery_matches_double_float_recovery(g, N, k, walls):
    # the mixed form on a mesh with two geometry classes recovers u = [P, -G^T] [f; lam] on the
    # tensor cores (8-bit digit splits, exact FP32 accumulation); the same steps with the
    # double-float recovery on the FP32 units agree to the splits' 4e-15 (N = 130: 33800
    # triangles, tiles with a ragged tail)
    vid, X = synth.split_square_mesh(N, L=1.0, periodic=not walls)
    vals = synth.sample_lattice(synth.random_spectrum_velocity(2, kmax=3, L=1.0), X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((vals ** 2).sum(-1)).max()), 1e-3)
    out = []
    for tc in (1, 0):
        mesh = g.DGMesh(vid, X, k, 1e-3, precision=1)
        mesh.set_tensor_cores(tc)
        mesh.set_velocity(vals)
        mesh.project_divfree()
        mesh.rk3_step(dt, 3)
        out.append(mesh.get_velocity())
        dg = mesh.diagnostics()
        assert dg["max_jump"] < 1e-11 and dg["max_div"] < 1e-10
    assert rel(out[0], out[1]) < 1e-12


def test_tensor_core_recovery_against_oracle(g):
    # shear layer, N = 16, BDM_3, five steps: the mixed form with the tensor-core recovery
    # against the FP64 oracle at the mixed tolerance
    k, nu, N = 3, 1e-4, 16
    vid, X = synth.split_square_mesh(N)
    vals = synth.sample_lattice(synth.double_shear_layer(), X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((vals ** 2).sum(-1)).max()), nu)
    d = Discretization(vid, X, k, nu)
    ref = d.to_lattice(d.rk3_step(d.project(d.from_lattice(vals)), dt, 5))
    mesh = g.DGMesh(vid, X, k, nu, precision=1)
    mesh.set_tensor_cores(1)
    mesh.set_velocity(vals)
    mesh.project_divfree()
    mesh.rk3_step(dt, 5)
    assert rel(mesh.get_velocity(), ref) < TOLMIX


def test_tensor_core_switch_rejected_where_not_set_up(g):
    from paper_1808_04669_gb300 import DGError
    vid, X = synth.split_square_mesh(4)
    mesh = g.DGMesh(vid, X, 2, 0.0, precision=0)      # FP64 form: no tensor-core recovery
    with pytest.raises(DGError) as e:
        mesh.set_tensor_cores(1)
    assert e.value.code == -3
    mesh.set_tensor_cores(0)


# ------------------------------------------------- multilevel preconditioner (non-lattice meshes)
@pytest.mark.parametrize("N,k,walls,perturb", [(12, 2, True, 0.0), (12, 3, True, 0.0), (20, 1, True, 0.0),
                                               (10, 3, False, 0.12), (17, 2, False, 0.1)])
def test_multilevel_rk3_parity(g, N, k, walls, perturb):
    # walls and perturbed tori take the multilevel PCG by default; three SSP-RK3 steps of a
    # random-spectrum field against the oracle's direct solves, both precision forms (N = 17, 20:
    # more than 256 facets, so the facet-constant level is coarsened by aggregation)
    nu = 1e-3
    vid, X = synth.split_square_mesh(N, L=1.0, periodic=not walls)
    if perturb:
        rng = np.random.default_rng(N)
        X = X + (perturb / N * rng.uniform(-1, 1, size=(N * N, 2)))[vid]
    vals = synth.sample_lattice(synth.random_spectrum_velocity(5, kmax=3, L=1.0), X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((vals ** 2).sum(-1)).max()), nu)
    d = Discretization(vid, X, k, nu)
    ref = d.to_lattice(d.rk3_step(d.project(d.from_lattice(vals)), dt, 3))
    for prec, tol in ((0, TOL64), (1, TOLMIX)):
        mesh = g.DGMesh(vid, X, k, nu, precision=prec)
        st = mesh.solver_stats()
        assert st["preconditioner"] == "multilevel", st
        mesh.set_velocity(vals)
        mesh.project_divfree()
        mesh.rk3_step(dt, 3)
        assert rel(mesh.get_velocity(), ref) < tol, prec
        st = mesh.solver_stats()
        assert st["total_iters"] / st["solves"] <= 45, st
        dg = mesh.diagnostics()
        assert dg["max_jump"] < 1e-11 and dg["max_div"] < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_multilevel_warm_start_history_across_step_sizes_and_schemes(g, prec):
    # the multilevel solves start from the same stage's multipliers in the last steps (quadratic
    # extrapolation once three steps had the same dt, linear with two, the last one rescaled after
    # a change of dt, none after a change of scheme); whatever the start, every solve meets
    # cg_rtol, so the states follow the oracle's direct solves through the whole sequence, and
    # with a full history the solves take fewer iterations than without one
    k, nu = 2, 1e-3
    vid, X = synth.split_square_mesh(12, L=1.0, periodic=False)
    vals = synth.sample_lattice(synth.random_spectrum_velocity(7, kmax=3, L=1.0), X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((vals ** 2).sum(-1)).max()), nu)
    d = Discretization(vid, X, k, nu)
    U = d.project(d.from_lattice(vals))
    mesh = g.DGMesh(vid, X, k, nu, precision=prec)
    assert mesh.solver_stats()["preconditioner"] == "multilevel"
    mesh.set_velocity(vals)
    mesh.project_divfree()
    tol = TOL64 if prec == 0 else TOLMIX
    its = []
    for n, h, scheme in ((1, dt, g.SSPRK3), (5, dt, g.SSPRK3), (2, 0.5 * dt, g.SSPRK3), (4, dt, g.SSPRK3),
                         (2, dt, g.RK4), (3, dt, g.SSPRK3)):
        st0 = mesh.solver_stats()
        mesh.step(h, n, scheme=scheme)
        st1 = mesh.solver_stats()
        its.append((st1["total_iters"] - st0["total_iters"]) / (st1["solves"] - st0["solves"]))
        if scheme == g.RK4:
            U = d.rk4_step(U, h, n)
        else:
            U = d.rk3_step(U, h, n)
        assert rel(mesh.get_velocity(), d.to_lattice(U)) < tol, (prec, n, h, scheme)
    # the first step starts cold (then from the previous stage rescaled); five more steps at the
    # same dt bring the full history
    assert its[1] < its[0], its


def test_multilevel_iterations_on_a_128_box_with_walls(g):
    # the case block Jacobi handles worst: 128 x 128 box, BDM_3 (1934 iterations per solve);
    # the multilevel PCG stays at a few dozen and gives the same projection
    k, nu = 3, 1e-4
    vid, X = synth.split_square_mesh(128, L=1.0, periodic=False)
    vals = synth.sample_lattice(synth.taylor_green(L=2.0), X, k)
    out = {}
    for pc in (g.PRECOND_MULTILEVEL, g.PRECOND_BLOCK_JACOBI):
        mesh = g.DGMesh(vid, X, k, nu, precond=pc)
        mesh.set_velocity(vals)
        mesh.project_divfree()
        out[pc] = (mesh.get_coefficients(), mesh.solver_stats())
    (a, sa), (b, sb) = out[g.PRECOND_MULTILEVEL], out[g.PRECOND_BLOCK_JACOBI]
    assert sa["preconditioner"] == "multilevel" and sb["preconditioner"] == "block Jacobi"
    assert sa["last_iters"] <= 50 and sb["last_iters"] > 20 * sa["last_iters"], (sa, sb)
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("precision", [0, 1])
def test_multilevel_steps_on_a_128_box_with_walls(g, precision):
    # SSP-RK3 steps on the 128 x 128 box: each stage's right-hand side is a small difference
    # (the divergence-free u^n cancels in it), so the solve runs down to the rounding level, where
    # the residual must be kept free of the constant multiplier that the V-cycle would amplify
    k, nu = 3, 1e-4
    vid, X = synth.split_square_mesh(128, L=1.0, periodic=False)
    vals = synth.sample_lattice(synth.random_spectrum_velocity(5, kmax=3, L=1.0), X, k)
    dt = synth.cfl_dt(X, k, float(np.abs(vals).max()), nu)
    mesh = g.DGMesh(vid, X, k, nu, precision=precision)
    mesh.set_velocity(vals)
    mesh.project_divfree()
    s0 = mesh.solver_stats()
    mesh.rk3_step(dt, 2)
    s1 = mesh.solver_stats()
    assert s1["preconditioner"] == "multilevel"
    assert (s1["total_iters"] - s0["total_iters"]) / (s1["solves"] - s0["solves"]) <= 40, s1
    assert s1["last_relres"] <= 1e-13
    dg = mesh.diagnostics()
    assert dg["max_jump"] < 1e-11 and dg["max_div"] < 1e-10


@pytest.mark.parametrize("N,k,walls", [(8, 3, True), (64, 3, True), (64, 2, False)])
def test_multilevel_device_v_cycle_matches_host_reference(g, N, k, walls):
    # one V-cycle of the device kernel against the host set-up's reference V-cycle
    vid, X = synth.split_square_mesh(N, L=1.0, periodic=not walls)
    if not walls:
        rng = np.random.default_rng(1)
        X = X + (0.1 / N * rng.uniform(-1, 1, size=(N * N, 2)))[vid]
    mesh = g.DGMesh(vid, X, k, 1e-4, precond=g.PRECOND_MULTILEVEL)
    r = np.random.default_rng(2).standard_normal((2, mesh.n_facet * (k + 1)))
    host = g.host_multilevel(vid, X, k, r=r)["z"]
    for i in range(2):
        assert rel(mesh.test_multilevel_apply(r[i]), host[i]) < 1e-13


@pytest.mark.parametrize("N,k,walls", [(8, 3, True), (64, 3, True), (64, 2, False)])
def test_multilevel_fp32_v_cycle_matches_host_reference(g, N, k, walls):
    # the mixed form runs the V-cycle in FP32 (the PCG vectors and S stay FP64): one V-cycle
    # against the host's FP64 reference, for inputs in the range of S (the constant multiplier,
    # the kernel of S on closed meshes, removed), to FP32 rounding amplified by the cycle
    vid, X = synth.split_square_mesh(N, L=1.0, periodic=not walls)
    if not walls:
        rng = np.random.default_rng(1)
        X = X + (0.1 / N * rng.uniform(-1, 1, size=(N * N, 2)))[vid]
    mesh = g.DGMesh(vid, X, k, 1e-4, precision=1, precond=g.PRECOND_MULTILEVEL)
    r = np.random.default_rng(2).standard_normal((2, mesh.n_facet, k + 1))
    r[:, :, 0] -= r[:, :, 0].mean(axis=1, keepdims=True)
    r = r.reshape(2, -1)
    host = g.host_multilevel(vid, X, k, r=r)["z"]
    for i in range(2):
        assert rel(mesh.test_multilevel_apply(r[i]), host[i]) < 1e-5


@pytest.mark.parametrize("k", [1, 2])
def test_split_column_pass_parity_n64(g, k):
    # N = 64: the lattice solver splits each column into even and odd wavenumbers (N/2+1 <= SMs);
    # results follow the oracle and the warm-started solves keep their short iteration count
    nu = 1e-4
    vid, X = synth.split_square_mesh(64)
    vals = synth.sample_lattice(synth.double_shear_layer(), X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((vals ** 2).sum(-1)).max()), nu)
    d = Discretization(vid, X, k, nu)
    ref = d.to_lattice(d.rk3_step(d.project(d.from_lattice(vals)), dt, 3))
    for prec, tol in ((0, TOL64), (1, TOLMIX)):
        mesh = g.DGMesh(vid, X, k, nu, precision=prec)
        mesh.set_velocity(vals)
        mesh.project_divfree()
        mesh.rk3_step(dt, 3)
        assert rel(mesh.get_velocity(), ref) < tol, prec
        st = mesh.solver_stats()
        assert st["lattice"] == 1.0 and st["total_iters"] / st["solves"] <= 6


@pytest.mark.parametrize("precond", [0, 1])
def test_mixed_precision_taylor_green(g, precond):
    vid, X, vals, dt = synth.make_workload("tgv_n8_k2")
    mesh = g.DGMesh(vid, X, 2, 1e-2, precision=1, precond=precond)
    d = Discretization(vid, X, 2, 1e-2)
    mesh.set_velocity(vals)
    mesh.project_divfree()
    mesh.rk3_step(dt, 30)
    U = d.rk3_step(d.project(d.from_lattice(vals)), dt, 30)
    assert rel(mesh.get_velocity(), d.to_lattice(U)) < TOLMIX
    dg = mesh.diagnostics()
    assert dg["max_jump"] < 1e-10


def test_euler_energy_non_increasing(g):
    vid, X = synth.split_square_mesh(16, L=1.0)
    f = synth.random_spectrum_velocity(0, kmax=6, L=1.0)
    vals = synth.sample_lattice(f, X, 2)
    dt = synth.cfl_dt(X, 2, float(np.sqrt((vals ** 2).sum(-1)).max()), 0.0)
    mesh = g.DGMesh(vid, X, 2, 0.0)
    mesh.set_velocity(vals)
    mesh.project_divfree()
    E = [mesh.diagnostics()["energy"]]
    for _ in range(10):
        mesh.rk3_step(dt, 1)
        E.append(mesh.diagnostics()["energy"])
    assert np.all(np.diff(E) <= 1e-14 * E[0])


# ---------------------------------------------------------------- pressure
@pytest.mark.parametrize("N,k", [(4, 2), (3, 3), (2, 1)])
def test_pressure_parity(g, N, k):
    mesh, d, X = pair(g, N, k, 1e-2)
    v = synth.sample_lattice(synth.taylor_green(), X, k) + 0.3 * random_lattice(mesh.n_tri, k, 7)
    mesh.set_velocity(v)
    mesh.project_divfree()
    pe, pf = mesh.get_pressure()
    U = d.project(d.from_lattice(v))
    w, lam = d.pressure(U)
    pe_ref, pf_ref = d.pressure_lattice(w, lam)
    assert rel(pe, pe_ref) < 1e-11
    assert rel(pf, pf_ref) < 1e-11


def test_diagnostics_parity(g):
    # integrals match; the normal jump is taken at the same facet Gauss points on both sides
    # (the max of the divergence is over different volume point sets, so it is only bounded)
    mesh, d, X = pair(g, 5, 3, 0.0)
    v = random_lattice(mesh.n_tri, 3, 9)
    mesh.set_velocity(v)
    dg = mesh.diagnostics()
    ref = d.diagnostics(d.from_lattice(v))
    for key in ("energy", "enstrophy", "max_jump"):
        assert abs(dg[key] - ref[key]) < 1e-12 * max(1.0, abs(ref[key])), key
    assert 0.5 * ref["max_div"] < dg["max_div"] < 2.0 * ref["max_div"]


# --------------------------------------------------------------- edge cases
def test_zero_state_and_zero_steps(g):
    mesh, d, X = pair(g, 2, 2, 0.1)
    mesh.project_divfree()
    mesh.rk3_step(0.01, 0)
    mesh.rk3_step(0.01, 3)
    assert np.abs(mesh.get_velocity()).max() == 0.0


def test_constant_velocity_preserved(g):
    mesh, d, X = pair(g, 3, 3, 0.05)
    v = synth.sample_lattice(synth.constant_field((0.4, -0.2)), X, 3)
    mesh.set_velocity(v)
    mesh.project_divfree()
    mesh.rk3_step(0.02, 5)
    assert np.abs(mesh.get_velocity() - v).max() < 1e-12


def test_invalid_inputs_raise(g):
    from paper_1808_04669_gb300 import DGError
    mesh, d, X = pair(g, 2, 1, 0.0)
    with pytest.raises(DGError):
        mesh.rk3_step(-1.0, 1)
    v = random_lattice(mesh.n_tri, 1, 0)
    v[0, 0, 0] = np.nan
    with pytest.raises(DGError) as e:
        mesh.set_velocity(v)
    assert e.value.code == -6
    vid, X = synth.split_square_mesh(2)
    with pytest.raises(DGError) as e:
        g.DGMesh(vid, X, 4, 0.0)
    assert e.value.code == -3


def test_iteration_cap_reports_not_converged(g):
    from paper_1808_04669_gb300 import DGError
    vid, X = synth.split_square_mesh(8)
    mesh = g.DGMesh(vid, X, 2, 0.0, cg_maxit=1, precond=1)   # block Jacobi (the Fourier path converges in 1)
    mesh.set_velocity(random_lattice(mesh.n_tri, 2, 4))
    with pytest.raises(DGError) as e:
        mesh.project_divfree()
    assert e.value.code == -5
