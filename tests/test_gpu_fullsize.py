"""Checks at the benchmark's full sizes, in the configuration bench.py times.

The oracle cannot factorise these systems in test time, so the solve is checked
through properties that hold at any size (divergence, normal continuity,
idempotence and orthogonality of the projection, mixed vs FP64 agreement), while
the residual kernels are compared with the oracle element by element on the
full mesh (the residual needs no solve).
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_full_size_256_bdm3_residual_matches_oracle(g):
    # A random field: for a smooth one the residual is a small difference of O(1/h) terms and
    # rounding alone moves it by ~1e-11 (N/32)^2 relative (measured by changing only the
    # oracle's quadrature rule), so element-by-element parity is checked where it is defined.
    # Both precision forms against one oracle evaluation: FP64 kernel k_stage<3,double> at 1e-12,
    # the double-float kernel the bench times (k_stage_df2<3>) at 1e-11.
    vid, X, _, dt = synth.make_workload("shear_n256_k3")
    vals = np.random.default_rng(2024).standard_normal((vid.shape[0], 10, 2))
    d = Discretization(vid, X, 3, 1e-4, chunk=16384)
    ref = d.to_lattice(d.riesz(d.residual(d.from_lattice(vals))))
    for prec, tol in ((g.FP64, 1e-12), (g.MIXED, 1e-11)):
        mesh = g.DGMesh(vid, X, 3, 1e-4, precision=prec)
        mesh.set_velocity(vals)
        gpu = mesh.eval_residual()
        assert rel(gpu, ref) < tol, prec
        mesh.close()


@pytest.mark.parametrize("name", ["shear_n256_k3", "spectrum_n1024_k2"])
def test_full_size_projection_and_step_properties(g, name):
    vid, X, vals, dt = synth.make_workload(name)
    w = synth.WORKLOADS[name]
    fp64 = g.DGMesh(vid, X, w.k, w.nu, precision=g.FP64)
    mixed = g.DGMesh(vid, X, w.k, w.nu, precision=g.MIXED)
    assert fp64.solver_stats()["lattice"] == 1.0 and mixed.solver_stats()["lattice"] == 1.0
    fp64.set_velocity(vals)
    u = fp64.get_coefficients()
    fp64.project_divfree()
    pu = fp64.get_coefficients()
    # L2-orthogonal projection: <u - Pu, Pu> = 0, and idempotent
    assert abs(float(((u - pu) * pu).sum())) < 1e-11 * float((pu * pu).sum())
    # u - Pu is orthogonal to the whole divergence-free space, not only to Pu: to P r for random r
    # (with div = 0 and [u.n] = 0 below, this identifies the L2 projection, Theorem 2). The
    # coefficients are in an orthonormal basis, so the Euclidean product is the L2 product.
    rng = np.random.default_rng(7)
    for _ in range(3):
        fp64.set_velocity(rng.standard_normal(vals.shape))
        fp64.project_divfree()
        pr = fp64.get_coefficients()
        scale = np.linalg.norm(u) * np.linalg.norm(pr)
        assert abs(float(((u - pu) * pr).sum())) < 1e-11 * scale
    fp64.set_coefficients(pu)
    fp64.project_divfree()
    assert np.abs(fp64.get_coefficients() - pu).max() < 1e-11 * np.abs(pu).max()
    dg = fp64.diagnostics()
    assert dg["max_div"] < 1e-10 and dg["max_jump"] < 1e-11
    mixed.set_coefficients(pu)
    fp64.rk3_step(dt, 2)
    mixed.rk3_step(dt, 2)
    a, b = mixed.get_velocity(), fp64.get_velocity()
    assert rel(a, b) < 1e-9
    for m in (fp64, mixed):
        dgm = m.diagnostics()
        assert dgm["max_div"] < 1e-10 and dgm["max_jump"] < 1e-10
    # energy: non-increasing (Euler: upwind dissipation only; NS: plus viscosity)
    e0 = float((pu * pu).sum())
    assert fp64.diagnostics()["energy"] <= e0 * (1 + 1e-14)


def test_rk3_parity_n128_bdm3_both_forms(g):
    # The bench workload at N = 128: the lattice solver takes the paths it takes at N = 256 (a
    # four-step FFT with a radix-16 factor, the column pass split into even and odd wavenumbers).
    # Two SSP-RK3 steps from the projected field, so that the second step's solves start from the
    # multiplier history, against the oracle's sparse direct solves (about 100 s on one host core).
    vid, X, vals, dt = synth.make_workload("shear_n256_k3", N=128)
    d = Discretization(vid, X, 3, 1e-4, chunk=16384)
    U = d.rk3_step(d.project(d.from_lattice(vals)), dt, 2)
    ref = d.to_lattice(U)
    for prec, tol in ((g.FP64, 1e-12), (g.MIXED, 1e-9)):
        mesh = g.DGMesh(vid, X, 3, 1e-4, precision=prec)
        assert mesh.solver_stats()["lattice"] == 1.0
        mesh.set_velocity(vals)
        mesh.project_divfree()
        mesh.rk3_step(dt, 2)
        assert rel(mesh.get_velocity(), ref) < tol, prec
        mesh.close()
