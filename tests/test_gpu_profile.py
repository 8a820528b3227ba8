"""Per-kernel profiling (dg_profile): CUDA-event times per kernel class during SSP-RK3 steps.
Inside a step, consecutive launches share one event (the end of one launch is the start of the
next), so the per-class times of a step add up to no more than the step's own event time, and
every launch is counted once."""
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


@pytest.mark.parametrize("prec,solver", [(0, "facet_pcg_fft_fp64"), (1, "facet_pcg_fft_fp32")])
def test_profile_counts_each_launch_and_fits_in_the_step(g, prec, solver):
    import torch
    N, k, nu, steps = 32, 3, 1e-4, 6
    vid, X = synth.split_square_mesh(N)
    vals = synth.sample_lattice(synth.taylor_green(), X, k)
    dt = synth.cfl_dt(X, k, float(np.sqrt((vals ** 2).sum(-1)).max()), nu)
    stream = torch.cuda.current_stream()
    with g.DGMesh(vid, X, k, nu, precision=prec, stream=stream.cuda_stream) as m:
        m.set_velocity(vals)
        m.project_divfree()
        m.rk3_step(dt, 2)
        torch.cuda.synchronize()
        m.profile(2)
        m.profile(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.rk3_step(dt, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = m.profile(0)
        total = e0.elapsed_time(e1)
        # the profile is cleared by profile(2) and collected by profile(0)
        assert prof["stage_residual"][1] == 3 * steps
        assert prof[solver][1] == 3 * steps
        assert prof["recover"][1] == 3 * steps
        launched = {n: v for n, v in prof.items() if v[1] > 0}
        assert set(launched) <= {"stage_residual", solver, "recover", "lattice"}
        assert all(v[0] > 0.0 for v in launched.values())
        # the classes' times are disjoint intervals of the timed region
        assert sum(v[0] for v in launched.values()) <= total * 1.0001 + 1e-3
        # profiling is off again: after a reset, later steps add nothing
        m.profile(2)
        m.rk3_step(dt, 1)
        assert all(v[1] == 0 for v in m.profile(0).values())
