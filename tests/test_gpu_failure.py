"""Failure detection on the CUDA path, without faulting the GPU.

- Bounded grid-barrier waits: one block of the persistent solver kernel is made to leave
  at its first barrier without arriving (dg_test_barrier_fault), so the other blocks' wait
  runs out. The call must return DG_ERR_CUDA ("timed out") instead of hanging, and the
  device context must stay usable: after the hook is turned off the same mesh gives the
  result of a fresh one.
- Energy watchdog (dg_set_energy_watchdog): the kinetic energy of the scheme does not grow
  at nu = 0 under the CFL step (Sec. 2.2), so the watchdog stays quiet there; a step size far
  above the stability limit makes ||u||^2 grow and the call returns DG_ERR_UNSTABLE.
"""
import numpy as np
import pytest

import synth

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


def random_lattice(n_tri, k, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_tri, (k + 1) * (k + 2) // 2, 2))


@pytest.mark.parametrize("precision,precond", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_barrier_timeout_is_reported_and_context_stays_usable(g, precision, precond):
    from paper_1808_04669_gb300 import DGError
    N, k = 32, 2
    vid, X = synth.split_square_mesh(N)
    v = random_lattice(2 * N * N, k, 5)
    mesh = g.DGMesh(vid, X, k, 1e-3, precision=precision, precond=precond)
    assert mesh.solver_stats()["blocks"] >= 2
    mesh.set_velocity(v)
    mesh.test_barrier_fault(spin_limit=1 << 14, skip_block=1)
    with pytest.raises(DGError) as e:
        mesh.project_divfree()
    assert e.value.code == -4 and "timed out" in str(e.value)
    # hook off: the same mesh works again and agrees with a fresh mesh
    mesh.test_barrier_fault(0, -1)
    mesh.set_velocity(v)
    mesh.project_divfree()
    mesh.rk3_step(0.01, 2)
    fresh = g.DGMesh(vid, X, k, 1e-3, precision=precision, precond=precond)
    fresh.set_velocity(v)
    fresh.project_divfree()
    fresh.rk3_step(0.01, 2)
    a, b = mesh.get_velocity(), fresh.get_velocity()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


def test_barrier_fault_hook_rejects_bad_arguments(g):
    from paper_1808_04669_gb300 import DGError
    vid, X = synth.split_square_mesh(2)
    mesh = g.DGMesh(vid, X, 1, 0.0)
    with pytest.raises(DGError):
        mesh.test_barrier_fault(-1, -1)
    with pytest.raises(DGError):
        mesh.test_barrier_fault(0, -2)


@pytest.mark.parametrize("precision", [0, 1])
def test_energy_watchdog_quiet_under_cfl_and_fires_above_it(g, precision):
    from paper_1808_04669_gb300 import DGError
    N, k = 16, 2
    vid, X = synth.split_square_mesh(N, L=1.0)
    v = random_lattice(2 * N * N, k, 11)
    dt = synth.cfl_dt(X, k, float(np.sqrt((v ** 2).sum(-1)).max()), 0.0)
    mesh = g.DGMesh(vid, X, k, 0.0, precision=precision)
    mesh.set_energy_watchdog(1e-10)
    mesh.set_velocity(v)
    mesh.project_divfree()
    E0 = mesh.diagnostics()["energy"]
    mesh.rk3_step(dt, 10)                    # stable: energy does not grow, no error
    assert mesh.diagnostics()["energy"] <= E0 * (1 + 1e-12)
    code = None
    for _ in range(30):                      # 40 x the CFL step: the unstable modes grow
        try:
            mesh.rk3_step(40 * dt, 1)
        except DGError as e:
            code = e.code
            assert "energy watchdog" in str(e)
            break
    assert code == -8
    # off again: the same oversized step no longer reports
    mesh.set_energy_watchdog(0.0)
    mesh.set_velocity(v)
    mesh.project_divfree()
    mesh.rk3_step(40 * dt, 1)
