"""Ensembles (dg_batch_*): uneven meshes, degrees, viscosities and precision forms advanced together
through one captured CUDA graph per step must give exactly what each member gives on its own."""
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


MEMBERS = [  # (N, k, nu, precision, perturb, L, periodic)
    (4, 1, 1e-2, 0, 0.0, 2 * np.pi, True),     # lattice, FP64
    (6, 2, 1e-3, 0, 0.0, 2 * np.pi, True),     # lattice, direct DFT (N not a power of two)
    (8, 3, 0.0, 1, 0.0, 1.0, True),            # lattice, mixed
    (5, 2, 1e-2, 1, 0.1, 1.0, True),           # perturbed (not translation invariant), mixed
    (4, 3, 1e-3, 1, 0.0, 1.0, False),          # box with walls, mixed
]


def make(g, spec, seed):
    N, k, nu, prec, perturb, L, periodic = spec
    vid, X = synth.split_square_mesh(N, L=L, periodic=periodic)
    if perturb:
        rng = np.random.default_rng(seed)
        X = X + (perturb * L / N * rng.uniform(-1, 1, size=(N * N, 2)))[vid]
    f = synth.random_spectrum_velocity(seed, kmax=3, L=L)
    vals = synth.sample_lattice(f, X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((vals ** 2).sum(-1)).max()), nu)
    meshes = []
    for _ in range(2):
        m = g.DGMesh(vid, X, k, nu, precision=prec)
        m.set_velocity(vals)
        m.project_divfree()
        meshes.append(m)
    return meshes, dt


def test_batch_equals_members_stepped_alone(g):
    pairs = [make(g, spec, 40 + i) for i, spec in enumerate(MEMBERS)]
    batch_members = [p[0][0] for p in pairs]
    solo = [p[0][1] for p in pairs]
    dts = np.array([p[1] for p in pairs])
    batch = g.DGBatch(batch_members)
    batch.set_lanes(1)
    batch.rk3_step(dts, 4)          # eager first step, graph capture, 3 replays
    batch.rk3_step(dts, 2)          # replays of the cached graph
    for m, dt in zip(solo, dts):
        m.rk3_step(dt, 6)
    for mb, ms in zip(batch_members, solo):
        a, b = mb.get_velocity(), ms.get_velocity()
        assert np.abs(a - b).max() <= 1e-14 * max(1.0, np.abs(b).max())
    # new step sizes: one eager step, then a re-captured graph
    batch.rk3_step(0.5 * dts, 3)
    for m, dt in zip(solo, dts):
        m.rk3_step(0.5 * dt, 3)
    for mb, ms in zip(batch_members, solo):
        a, b = mb.get_velocity(), ms.get_velocity()
        assert np.abs(a - b).max() <= 1e-14 * max(1.0, np.abs(b).max())
        dg = mb.diagnostics()
        assert dg["max_jump"] < 1e-10
    batch.close()


def test_batch_sees_a_viscosity_changed_between_calls(g):
    # the graph holds each member's kernel arguments by value: after dg_set_viscosity on a member the
    # next batch call must not replay the old viscosity
    specs = [MEMBERS[0], MEMBERS[2]]
    pairs = [make(g, spec, 60 + i) for i, spec in enumerate(specs)]
    batch_members = [p[0][0] for p in pairs]
    solo = [p[0][1] for p in pairs]
    dts = np.array([p[1] for p in pairs])
    batch = g.DGBatch(batch_members)
    batch.set_lanes(1)
    batch.rk3_step(dts, 4)          # eager step, capture, replays
    for m, dt in zip(solo, dts):
        m.rk3_step(dt, 4)
    for m in (batch_members[0], solo[0]):
        m.set_viscosity(0.3)        # a large change, so a stale graph would show
    batch.rk3_step(dts, 3)          # same step sizes: only the viscosity changed
    for m, dt in zip(solo, dts):
        m.rk3_step(dt, 3)
    for mb, ms in zip(batch_members, solo):
        a, b = mb.get_velocity(), ms.get_velocity()
        assert np.abs(a - b).max() <= 1e-14 * max(1.0, np.abs(b).max())
    batch.close()


@pytest.mark.parametrize("lanes", [4, 0])
def test_batch_on_parallel_lanes_equals_members_stepped_alone(g, lanes):
    # members dealt out to parallel branches of the graph, solver grids divided by the lanes
    # (fixed 4 lanes, or chosen by the tuner); results equal the solo runs up to the rounding of
    # the solvers' block-wise reductions
    pairs = [make(g, spec, 70 + i) for i, spec in enumerate(MEMBERS)]
    batch_members = [p[0][0] for p in pairs]
    solo = [p[0][1] for p in pairs]
    dts = np.array([p[1] for p in pairs])
    batch = g.DGBatch(batch_members)
    batch.set_lanes(lanes)
    batch.rk3_step(dts, 14)         # eager step, tuning replays (lanes = 0), captured replays
    chosen, times = batch.tuning()
    assert chosen in (1, 2, 4, 8, 16)
    if lanes == 0:
        assert 1 in times and len(times) >= 2, times
    else:
        assert chosen == lanes
    for m, dt in zip(solo, dts):
        m.rk3_step(dt, 14)
    for mb, ms in zip(batch_members, solo):
        a, b = mb.get_velocity(), ms.get_velocity()
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())
        assert mb.diagnostics()["max_jump"] < 1e-10
    batch.close()


def test_batch_rejects_bad_arguments(g):
    from paper_1808_04669_gb300 import DGError
    (m, _), dt = make(g, MEMBERS[0], 1)
    with pytest.raises(DGError):
        g.DGBatch([m, m])
    b = g.DGBatch([m])
    with pytest.raises(DGError):
        b.rk3_step([-1.0], 1)
    with pytest.raises(DGError):
        b.set_lanes(3)
    b.close()
