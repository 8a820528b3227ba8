"""The facet solve that allocates nothing (dg_facet_solve_noalloc).

It serves callers that cannot call cudaMalloc (code running inside another
framework's memory pool or budget, or where allocating is forbidden), so they
cannot create a dg_mesh either: they hold the condensed facet operator, the
right-hand side and the solution in memory they own, and the library keeps its
work vectors in a static device array.

What the test checks: the existing entry point dg_get_pressure solves the mesh's
facet system S lam = g for the pressure functional and returns lam on the
facets. The no-allocation solve is given the library's own facet operator S
(dg_host_facet_operator) and g = S lam, and must return that lam (in the energy
norm of S, the norm in which the velocity error is measured): an S-inverse
consistency check of the new entry point against the existing one, on two calls
in a row that share the static scratch, from a zero and from a random initial
guess.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1808_04669_gb300 import build
    build.build()
    import paper_1808_04669_gb300 as pkg
    return pkg


def facet_values_to_coefficients(pf, k):
    """Coefficients in the facet basis sqrt(2m+1) P_m(2t-1) from the values at t = i/k (dgdf.h conventions)."""
    t = np.arange(k + 1) / k
    V = np.stack([np.sqrt(2 * m + 1) * np.polynomial.legendre.Legendre.basis(m)(2 * t - 1) for m in range(k + 1)], 1)
    return np.linalg.solve(V, pf.T).T


def apply_S(nbr, st, blk, x):
    nf, nl = x.shape
    y = np.einsum("fij,fj->fi", blk[st, 0], x)
    for b in range(4):
        y += np.einsum("fij,fj->fi", blk[st, b + 1], x[nbr[:, b]])
    return y


def energy_rel(nbr, st, blk, a, ref):
    # lam is defined up to the constant multiplier (mode 0 on every facet, the kernel of S): remove it first
    d = a - ref
    d[:, 0] -= d[:, 0].mean()
    return float(np.sqrt(abs((d * apply_S(nbr, st, blk, d)).sum()) / (ref * apply_S(nbr, st, blk, ref)).sum()))


@pytest.mark.parametrize("N,k", [(6, 2), (5, 3)])
def test_noalloc_solve_matches_mesh_solver_on_two_calls(g, N, k):
    import torch
    vid, X = synth.split_square_mesh(N)
    mesh = g.DGMesh(vid, X, k, 1e-2)
    rng = np.random.default_rng(N * 10 + k)
    mesh.set_velocity(rng.standard_normal((mesh.n_tri, mesh.n_lat, 2)))
    mesh.project_divfree()
    lams = []
    _, pf = mesh.get_pressure()                            # existing entry point, first state
    lams.append(facet_values_to_coefficients(pf, k))
    mesh.rk3_step(0.01, 1)
    _, pf = mesh.get_pressure()                            # existing entry point, second state
    lams.append(facet_values_to_coefficients(pf, k))

    nbr, st, blk, binv = g.host_facet_operator(vid, X, k)
    dev = torch.device("cuda")
    nbr_d = torch.from_numpy(nbr).to(dev)
    st_d = torch.from_numpy(st).to(dev)
    blk_d = torch.from_numpy(np.ascontiguousarray(blk)).to(dev)
    binv_d = torch.from_numpy(np.ascontiguousarray(binv)).to(dev)
    iters = []
    for lam_ex in lams:                                    # two calls in a row on the shared scratch
        rhs = apply_S(nbr, st, blk, lam_ex)
        g_d = torch.from_numpy(np.ascontiguousarray(rhs)).to(dev)
        lam_d = torch.zeros_like(g_d)
        it, rr = g.facet_solve_noalloc(k, nbr_d, st_d, blk_d, binv_d, g_d, lam_d)
        torch.cuda.synchronize()
        lam = lam_d.cpu().numpy()
        assert it > 0 and rr <= 1e-13
        assert energy_rel(nbr, st, blk, lam, lam_ex) < TOL64
        iters.append(it)
    # lam is also the initial guess: a random start converges to the same solution, and a start
    # at the solution itself needs (almost) no iterations
    lam_ex = lams[1]
    g_d = torch.from_numpy(np.ascontiguousarray(apply_S(nbr, st, blk, lam_ex))).to(dev)
    lam_d = torch.from_numpy(rng.standard_normal(lam_ex.shape)).to(dev)
    it, rr = g.facet_solve_noalloc(k, nbr_d, st_d, blk_d, binv_d, g_d, lam_d)
    torch.cuda.synchronize()
    assert rr <= 1e-13 and energy_rel(nbr, st, blk, lam_d.cpu().numpy(), lam_ex) < TOL64
    lam_d = torch.from_numpy(np.ascontiguousarray(lam_ex)).to(dev)
    it0, rr = g.facet_solve_noalloc(k, nbr_d, st_d, blk_d, binv_d, g_d, lam_d)
    torch.cuda.synchronize()
    assert it0 < iters[1] and energy_rel(nbr, st, blk, lam_d.cpu().numpy(), lam_ex) < TOL64


def test_noalloc_wrapper_rejects_mismatched_shapes(g):
    import torch
    vid, X = synth.split_square_mesh(4)
    k = 2
    nbr, st, blk, binv = g.host_facet_operator(vid, X, k)
    dev = torch.device("cuda")
    t = {n: torch.from_numpy(np.ascontiguousarray(a)).to(dev) for n, a in
         (("nbr", nbr), ("st", st), ("blk", blk), ("binv", binv))}
    nf = nbr.shape[0]
    good_g = torch.zeros(nf, k + 1, dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):     # g one facet short
        g.facet_solve_noalloc(k, t["nbr"], t["st"], t["blk"], t["binv"], good_g[:-1], torch.zeros_like(good_g))
    with pytest.raises(ValueError):     # blocks of the wrong degree
        g.facet_solve_noalloc(k + 1, t["nbr"], t["st"], t["blk"], t["binv"], good_g, torch.zeros_like(good_g))
    with pytest.raises(ValueError):     # stencil ids for fewer facets
        g.facet_solve_noalloc(k, t["nbr"], t["st"][:-1], t["blk"], t["binv"], good_g, torch.zeros_like(good_g))


def test_noalloc_rejects_sizes_beyond_its_scratch(g):
    import torch
    from paper_1808_04669_gb300 import DGError
    k = 2
    n_facet = (1 << 18) // (k + 1) + 1
    small_i = torch.zeros(4, dtype=torch.int32, device="cuda")
    small_d = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(DGError) as e:
        g.lib()
        import ctypes
        V = ctypes.c_void_p
        from paper_1808_04669_gb300._native import check
        check(g.lib().dg_facet_solve_noalloc(k, n_facet, V(small_i.data_ptr()), V(small_i.data_ptr()),
                                             V(small_d.data_ptr()), V(small_d.data_ptr()), V(small_d.data_ptr()),
                                             V(small_d.data_ptr()), 1e-13, 100, None, None, None),
              "dg_facet_solve_noalloc")
    assert e.value.code == -1 and "exceeds the static scratch limit" in str(e.value)
