"""The three-dimensional path (include/dgdf3.h: closed tetrahedral meshes, FP64) against the 3-D
oracle (oracle/dg3.py) on the same seeded inputs: periodic Kuhn cube meshes, the ABC flow plus
seeded noise. Tolerance: 1e-12 relative L2 over lattice values."""
import numpy as np
import pytest

from oracle.dg3 import Discretization3
from synth.mesh3 import abc_flow, kuhn_cube_mesh, sample_lattice3

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def field(X, k, seed, noise=0.3):
    v = sample_lattice3(abc_flow(), X, k)
    return v + noise * np.random.default_rng(seed).standard_normal(v.shape)


@pytest.mark.parametrize("k", [1, 2])
def test_lattice_roundtrip_and_info(g, k):
    vid, X = kuhn_cube_mesh(2)
    m = g.DGMesh3(vid, X, k, 0.0)
    assert m.n_tet == 48 and m.n_face == 96
    v = field(X, k, 1)
    m.set_velocity(v)
    assert np.abs(m.get_velocity() - v).max() < 1e-13


@pytest.mark.parametrize("N,k,nu", [(2, 1, 0.0), (2, 2, 0.05), (3, 1, 0.02), (3, 2, 0.0)])
def test_residual_parity(g, N, k, nu):
    vid, X = kuhn_cube_mesh(N)
    d = Discretization3(vid, X, k, nu)
    v = field(X, k, 10 + N)
    m = g.DGMesh3(vid, X, k, nu)
    m.set_velocity(v)
    ref = d.to_lattice(d.riesz(d.residual(d.from_lattice(v))))
    assert rel(m.eval_residual(), ref) < TOL


@pytest.mark.parametrize("N,k,precond", [(2, 1, 0), (2, 2, 0), (3, 2, 0), (2, 1, 1), (3, 2, 1)])
def test_projection_parity(g, N, k, precond):
    # multilevel (default) and block-Jacobi PCG
    vid, X = kuhn_cube_mesh(N)
    d = Discretization3(vid, X, k, 0.0)
    v = field(X, k, 20 + N)
    m = g.DGMesh3(vid, X, k, 0.0, precond=precond)
    m.set_velocity(v)
    m.project_divfree()
    ref = d.to_lattice(d.project(d.from_lattice(v)))
    assert rel(m.get_velocity(), ref) < TOL
    dg = m.diagnostics()
    assert dg["max_div"] < 1e-11 and dg["max_jump"] < 1e-11


@pytest.mark.parametrize("N,k,nu,precond", [(2, 1, 0.01, 0), (2, 2, 0.01, 0), (3, 2, 1e-3, 0), (3, 2, 1e-3, 1)])
def test_rk3_parity(g, N, k, nu, precond):
    vid, X = kuhn_cube_mesh(N)
    d = Discretization3(vid, X, k, nu)
    v = field(X, k, 30 + N, noise=0.1)
    dt = 0.3 * (2 * np.pi / N) / (k * k * np.abs(v).max())
    U = d.rk3_step(d.project(d.from_lattice(v)), dt, 3)
    m = g.DGMesh3(vid, X, k, nu, precond=precond)
    m.set_velocity(v)
    m.project_divfree()
    m.rk3_step(dt, 3)
    assert rel(m.get_velocity(), d.to_lattice(U)) < TOL
    dg = m.diagnostics()
    od = d.diagnostics(U)
    assert abs(dg["energy"] - od["energy"]) < 1e-11 * od["energy"]
    assert dg["max_jump"] < 1e-11


def test_abc_flow_decays_as_exp_minus_nu_t(g):
    # the ABC field decays as exp(-nu t); the discrete energy of its projection follows on 4^3 cells
    k, nu, N = 2, 0.05, 4
    vid, X = kuhn_cube_mesh(N)
    m = g.DGMesh3(vid, X, k, nu)
    m.set_velocity(sample_lattice3(abc_flow(), X, k))
    m.project_divfree()
    e0 = m.diagnostics()["energy"]
    T, steps = 0.5, 20
    m.rk3_step(T / steps, steps)
    e1 = m.diagnostics()["energy"]
    assert abs(e1 / e0 - np.exp(-2 * nu * T)) < 0.02


def test_arguments_rejected(g):
    vid, X = kuhn_cube_mesh(2)
    with pytest.raises(g.DGError) as e:
        g.DGMesh3(vid, X, 3, 0.0)
    assert e.value.code == -3
    # an open mesh (one cube's six tetrahedra without periodic identification): faces with one side
    vid1, X1 = kuhn_cube_mesh(2)
    sel = np.arange(6)
    ids = np.arange(24).reshape(6, 4)
    with pytest.raises(g.DGError) as e:
        g.DGMesh3(ids, X1[sel], 1, 0.0)
    assert e.value.code in (-2, -3)


def test_multilevel_iterations_stay_flat_on_16_cubes(g):
    # 16^3 Kuhn cubes, BDM_2: the multilevel PCG needs a few dozen iterations per projection, block
    # Jacobi several hundred, and both give the same projection
    k = 2
    vid, X = kuhn_cube_mesh(16)
    v = field(X, k, 3)
    out = {}
    for pc in (g.PRECOND_AUTO, g.PRECOND_BLOCK_JACOBI):
        m = g.DGMesh3(vid, X, k, 0.0, precond=pc)
        m.set_velocity(v)
        m.project_divfree()
        out[pc] = (m.get_velocity(), m.diagnostics())
    (a, da), (b, db) = out[g.PRECOND_AUTO], out[g.PRECOND_BLOCK_JACOBI]
    assert da["last_iters"] <= 60 and db["last_iters"] > 4 * da["last_iters"], (da, db)
    assert rel(a, b) < 1e-11
    assert da["max_div"] < 1e-10 and da["max_jump"] < 1e-10


@pytest.mark.parametrize("precond", [0, 1])
def test_errors_and_edge_cases(g, precond):
    vid, X = kuhn_cube_mesh(2)
    k = 2
    v = field(X, k, 7)
    # an iteration cap that cannot be met is reported, not hidden
    m = g.DGMesh3(vid, X, k, 0.0, cg_maxit=1, precond=precond)
    m.set_velocity(v)
    with pytest.raises(g.DGError) as e:
        m.project_divfree()
    assert e.value.code == -5
    # non-finite input is refused before it reaches the device state
    m = g.DGMesh3(vid, X, k, 0.0, precond=precond)
    bad = v.copy()
    bad[3, 1, 2] = np.inf
    with pytest.raises(g.DGError) as e:
        m.set_velocity(bad)
    assert e.value.code == -6
    # zero steps leave the state; the projection is idempotent
    m.set_velocity(v)
    m.project_divfree()
    u1 = m.get_velocity()
    m.rk3_step(0.01, 0)
    assert np.array_equal(m.get_velocity(), u1)
    m.project_divfree()
    assert rel(m.get_velocity(), u1) < 1e-12


def test_rk3_parity_k1_multilevel_n3(g):
    vid, X = kuhn_cube_mesh(3)
    k, nu = 1, 0.02
    d = Discretization3(vid, X, k, nu)
    v = field(X, k, 41, noise=0.2)
    dt = 0.2 * (2 * np.pi / 3) / np.abs(v).max()
    U = d.rk3_step(d.project(d.from_lattice(v)), dt, 4)
    m = g.DGMesh3(vid, X, k, nu)
    m.set_velocity(v)
    m.project_divfree()
    m.rk3_step(dt, 4)
    assert rel(m.get_velocity(), d.to_lattice(U)) < TOL


@pytest.mark.parametrize("N,k,nu,precond", [(2, 1, 0.01, 0), (2, 2, 0.0, 0), (3, 2, 0.01, 0), (3, 1, 0.0, 1)])
def test_pressure_parity(g, N, k, nu, precond):
    # the pressure of L(u) (eq. (12) with that functional alone), mean-free, at the element's
    # degree-(k-1) lattice points and the face's degree-k lattice points
    vid, X = kuhn_cube_mesh(N)
    d = Discretization3(vid, X, k, nu)
    v = field(X, k, 40 + N, noise=0.2)
    m = g.DGMesh3(vid, X, k, nu, precond=precond)
    m.set_velocity(v)
    m.project_divfree()
    m.rk3_step(0.01, 1)                    # a solve history, which the pressure solve must not use
    pe, pf = m.get_pressure()
    U = d.from_lattice(m.get_velocity())
    w, lam = d.pressure(U)
    pe_ref, pf_ref = d.pressure_lattice(w, lam)
    assert pe.shape == pe_ref.shape and pf.shape == pf_ref.shape
    assert rel(pe, pe_ref) < 1e-11
    assert rel(pf, pf_ref) < 1e-11
    # element pressure alone; the state is unchanged and steps still match
    pe2, none = m.get_pressure(with_face=False)
    assert none is None and rel(pe2, pe) < 1e-13
    u0 = m.get_velocity()
    m.rk3_step(0.01, 1)
    ref = d.to_lattice(d.rk3_step(d.from_lattice(u0), 0.01, 1))
    assert rel(m.get_velocity(), ref) < TOL



@pytest.mark.parametrize("precond", [0, 1])
def test_rk3_warm_start_history_across_step_sizes(g, precond):
    # each stage's face solve starts from the same stage's multipliers in the last steps:
    # quadratic extrapolation once three steps had the same dt, linear with two, the last one
    # rescaled after a change of dt; every solve meets cg_rtol whatever the start
    N, k, nu = 2, 2, 1e-2
    vid, X = kuhn_cube_mesh(N)
    d = Discretization3(vid, X, k, nu)
    v = field(X, k, 60, noise=0.1)
    dt = 0.2 * (2 * np.pi / N) / (k * k * np.abs(v).max())
    m = g.DGMesh3(vid, X, k, nu, precond=precond)
    m.set_velocity(v)
    m.project_divfree()
    U = d.project(d.from_lattice(v))
    its = []
    for n, h in ((1, dt), (5, dt), (2, 0.5 * dt), (3, dt)):
        before = m.diagnostics()
        m.rk3_step(h, n)
        after = m.diagnostics()
        its.append((after["total_iters"] - before["total_iters"]) / (after["solves"] - before["solves"]))
        U = d.rk3_step(U, h, n)
        assert rel(m.get_velocity(), d.to_lattice(U)) < TOL, (n, h)
    assert its[1] < its[0], its
