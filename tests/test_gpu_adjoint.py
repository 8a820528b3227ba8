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
