"""Hand-written adjoint of the SSP-RK3 rollout (dg_rk3_vjp) and its torch.autograd binding.

Checked against the FP64 oracle's tangent-linear model by the dot-product identity
<ubar, du_K> = <J^T ubar, du_0> (and the same for nu), against central finite
differences of the GPU forward map, and for independence of the checkpoint spacing.
"""
import numpy as np
import pytest

import synth
from oracle import Discretization

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1808_04669_gb300 import build
    build.build()
    import paper_1808_04669_gb300 as pkg
    return pkg


def setup_case(g, N=4, k=2, nu=1e-2, steps=4, seed=3):
    vid, X = synth.split_square_mesh(N, L=1.0)
    v0 = synth.sample_lattice(synth.random_spectrum_velocity(seed, kmax=3, L=1.0), X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((v0 ** 2).sum(-1)).max()), nu)
    mesh = g.DGMesh(vid, X, k, nu)
    mesh.set_velocity(v0)
    mesh.project_divfree()
    scratch = g.DGMesh(vid, X, k, nu)

    def coef(lat):
        scratch.set_velocity(lat)
        return scratch.get_coefficients()
    return vid, X, v0, dt, mesh, coef, steps


@pytest.mark.parametrize("k", [2, 3])
def test_adjoint_matches_oracle_tangent(g, k):
    vid, X, v0, dt, mesh, coef, K = setup_case(g, k=k)
    nu = 1e-2
    rng = np.random.default_rng(7)
    dv = rng.standard_normal(v0.shape)            # broken perturbation of u_0 (lattice values)
    gv = rng.standard_normal(v0.shape)            # output cotangent as a field (lattice values)
    d = Discretization(vid, X, k, nu)
    U0 = d.project(d.from_lattice(v0))
    G = d.from_lattice(gv)
    _, dUk = d.rk3_tangent(U0, d.from_lattice(dv), dt, K)
    _, dUn = d.rk3_tangent(U0, np.zeros_like(U0), dt, K, dnu=1.0)
    lhs_u = float((d.apply_mass(G) * dUk).sum())
    lhs_nu = float((d.apply_mass(G) * dUn).sum())
    u0bar, nubar = mesh.rk3_vjp(dt, K, coef(gv), checkpoint_every=2)
    rhs_u = float((u0bar * coef(dv)).sum())
    assert abs(lhs_u - rhs_u) < 1e-9 * abs(lhs_u)
    assert abs(lhs_nu - nubar) < 1e-9 * abs(lhs_nu)


def test_adjoint_independent_of_checkpoint_spacing(g):
    vid, X, v0, dt, mesh, coef, K = setup_case(g, N=8, k=2, steps=6)
    u0 = mesh.get_coefficients()
    ubar = np.random.default_rng(1).standard_normal(u0.shape)
    res = []
    for ck in (1, 2, 6):
        mesh.set_coefficients(u0)
        res.append(mesh.rk3_vjp(dt, K, ubar, checkpoint_every=ck))
    for r in res[1:]:
        assert np.abs(r[0] - res[0][0]).max() < 1e-11 * np.abs(res[0][0]).max()
        assert abs(r[1] - res[0][1]) < 1e-11 * abs(res[0][1])
    # the call leaves the forward result as the state
    mesh.set_coefficients(u0)
    mesh.rk3_step(dt, K)
    uk = mesh.get_coefficients()
    mesh.set_coefficients(u0)
    mesh.rk3_vjp(dt, K, ubar)
    assert np.abs(mesh.get_coefficients() - uk).max() < 1e-13


def test_autograd_gradients_match_finite_differences(g):
    import torch
    from paper_1808_04669_gb300.autograd import rk3_rollout
    vid, X, v0, dt, mesh, coef, K = setup_case(g, N=8, k=2, nu=1e-3, steps=5)
    dev = torch.device("cuda")
    u0 = torch.from_numpy(mesh.get_coefficients()).to(dev)
    target = torch.from_numpy(coef(synth.sample_lattice(synth.random_spectrum_velocity(4, kmax=3, L=1.0), X, 2))).to(dev)
    nu = torch.tensor(1e-3, dtype=torch.float64, device=dev, requires_grad=True)
    x = u0.clone().requires_grad_(True)

    def loss(u, n):
        uk = rk3_rollout(mesh, u, n, dt, K, checkpoint_every=2)
        return 0.5 * ((uk - target) ** 2).sum()
    J = loss(x, nu)
    J.backward()
    # divergence-free direction: the projection of a random field
    rng = np.random.default_rng(2)
    mesh.set_coefficients(rng.standard_normal(u0.shape))
    mesh.project_divfree()
    du = torch.from_numpy(mesh.get_coefficients()).to(dev)
    eps = 1e-4
    with torch.no_grad():
        fd_u = (loss(u0 + eps * du, nu) - loss(u0 - eps * du, nu)) / (2 * eps)
        epsn = 1e-7
        fd_nu = (loss(u0, nu + epsn) - loss(u0, nu - epsn)) / (2 * epsn)
    ad_u = float((x.grad * du).sum())
    assert abs(ad_u - float(fd_u)) < 1e-6 * abs(ad_u)
    assert abs(float(nu.grad) - float(fd_nu)) < 1e-6 * abs(float(nu.grad))


def test_adjoint_gradient_at_the_gradient_workload_scale(g):
    # The gradient workload: 128 x 128 unit square, BDM_2, nu = 1e-3, random-spectrum u0 (seed 3)
    # and target (seed 4), J = 1/2 ||u_K - u*||^2 after K = 200 SSP-RK3 steps, checkpoints every 20.
    # dg_rk3_vjp against central finite differences along a divergence-free direction and in nu.
    w = synth.WORKLOADS["adjoint_n128_k2"]
    vid, X, vals, dt = synth.make_workload(w)
    mesh = g.DGMesh(vid, X, w.k, w.nu)
    mesh.set_velocity(synth.sample_lattice(synth.random_spectrum_velocity(4, L=1.0), X, w.k, grid=(w.k * w.N, 1.0)))
    target = mesh.get_coefficients()
    mesh.set_velocity(vals)
    mesh.project_divfree()
    u0 = mesh.get_coefficients()
    K = w.steps

    def J(u, nu):
        mesh.set_viscosity(nu)
        mesh.set_coefficients(u)
        mesh.rk3_step(dt, K)
        return 0.5 * float(((mesh.get_coefficients() - target) ** 2).sum())
    mesh.set_coefficients(u0)
    mesh.rk3_step(dt, K)
    ubar = mesh.get_coefficients() - target
    mesh.set_coefficients(u0)
    u0bar, nubar = mesh.rk3_vjp(dt, K, ubar, checkpoint_every=20)
    # divergence-free direction with the norm of u0
    mesh.set_coefficients(np.random.default_rng(9).standard_normal(u0.shape))
    mesh.project_divfree()
    du = mesh.get_coefficients()
    du *= np.linalg.norm(u0) / np.linalg.norm(du)
    eps = 1e-5
    fd_u = (J(u0 + eps * du, w.nu) - J(u0 - eps * du, w.nu)) / (2 * eps)
    epsn = 1e-6
    fd_nu = (J(u0, w.nu + epsn) - J(u0, w.nu - epsn)) / (2 * epsn)
    ad_u = float((u0bar * du).sum())
    assert abs(ad_u - fd_u) < 1e-6 * abs(ad_u), (ad_u, fd_u)
    assert abs(nubar - fd_nu) < 1e-6 * abs(nubar), (nubar, fd_nu)


def test_adjoint_of_the_mixed_form_matches_the_fp64_form(g):
    # the mixed form runs the forward and the projections Q in double-float; the transposed
    # residual Jacobian is FP64 in both forms: the two gradients agree to the mixed tolerance
    vid, X = synth.split_square_mesh(16, L=1.0)
    k, nu = 2, 1e-3
    v0 = synth.sample_lattice(synth.random_spectrum_velocity(3, kmax=4, L=1.0), X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((v0 ** 2).sum(-1)).max()), nu)
    out = []
    for prec in (0, 1):
        mesh = g.DGMesh(vid, X, k, nu, precision=prec)
        mesh.set_velocity(v0)
        mesh.project_divfree()
        ubar = np.random.default_rng(4).standard_normal(mesh.get_coefficients().shape)
        out.append(mesh.rk3_vjp(dt, 10, ubar, checkpoint_every=5))
    (a, na), (b, nb) = out
    assert np.linalg.norm(b - a) < 1e-9 * np.linalg.norm(a)
    assert abs(nb - na) < 1e-9 * abs(na)
