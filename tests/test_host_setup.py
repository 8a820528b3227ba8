"""CPU checks of libdgdf: it loads, exports every declared symbol, and its host set-up
(topology, quadrature, basis) follows the conventions and exactness it claims."""
import math
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    import paper_1808_04669_gb300 as pkg
    from paper_1808_04669_gb300 import build
    build.build()
    return pkg


def declared_functions():
    names = []
    for h in ("dgdf.h", "dgdf_host.h", "dgdf3.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(dg3?_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(g):
    names = declared_functions()
    assert "dg_mesh_create" in names and "dg_rk3_step" in names and "dg_host_topology" in names
    assert "dg3_mesh_create" in names and "dg3_rk3_step" in names
    L = g.lib()
    for n in names:
        assert hasattr(L, n), n
    from paper_1808_04669_gb300._native import EXPORTS
    assert sorted(EXPORTS) == names


def test_kernel_names(g):
    L = g.lib()
    names = []
    i = 0
    while L.dg_kernel_name(i) is not None:
        names.append(L.dg_kernel_name(i).decode())
        i += 1
    assert "facet_pcg_fp64" in names and "stage_residual" in names


@pytest.mark.parametrize("k", [1, 2, 3])
def test_volume_rule_exact_to_3k_minus_1(g, k):
    q = g.host_reference(k, 0).reshape(-1, 3)
    deg = 3 * k - 1
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs((q[:, 2] * q[:, 0] ** a * q[:, 1] ** b).sum() - exact) < 2e-16 * 10


@pytest.mark.parametrize("k", [1, 2, 3])
def test_facet_rule_is_gauss_legendre(g, k):
    q = g.host_reference(k, 1).reshape(-1, 2)
    assert len(q) == math.ceil((3 * k + 1) / 2)
    x, w = np.polynomial.legendre.leggauss(len(q))
    assert np.allclose(q[:, 0], 0.5 * (x + 1), atol=1e-15, rtol=0)
    assert np.allclose(q[:, 1], 0.5 * w, atol=1e-15, rtol=0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_basis_orthonormal_and_hierarchical(g, k):
    q = g.host_reference(k, 0).reshape(-1, 3)
    ns = (k + 1) * (k + 2) // 2
    phi = g.host_reference(k, 2).reshape(len(q), ns)
    M = (phi * q[:, 2:3]).T @ phi
    assert np.abs(M - np.eye(ns)).max() < 5e-15
    # first function is the constant; the first n_lat(k-1) span P^{k-1}: their gradients are degree k-2
    assert np.allclose(phi[:, 0], phi[0, 0]) and abs(phi[0, 0] - math.sqrt(2.0)) < 1e-14
    # gradients match finite differences of the values at the lattice (smoke check of the derivative table)
    dphi = g.host_reference(k, 3).reshape(len(q), ns, 2)
    assert np.all(np.isfinite(dphi)) and np.abs(dphi[:, 0, :]).max() == 0.0
    V = g.host_reference(k, 4).reshape(ns, ns)
    assert np.linalg.cond(V) < 1e4


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_library_topology_matches_oracle_convention(g, N):
    from oracle.mesh import Topology
    vid, X = synth.split_square_mesh(N)
    tf, to, ft = g.host_topology(vid, X)
    T = Topology(vid, X)
    assert tf.shape == T.tri_facet.shape
    assert np.array_equal(tf, T.tri_facet)
    assert np.array_equal(ft, T.facet_tri)
    orient = np.zeros_like(to)
    for f in range(T.n_facet):
        for s in range(2):
            orient[T.facet_tri[f, s], T.facet_loc[f, s]] = T.facet_orient[f, s]
    assert np.array_equal(to, orient)


def test_library_topology_on_a_perturbed_periodic_mesh(g):
    # interior vertices moved (periodic images moved together): still closed and consistent
    from oracle.mesh import Topology
    N = 5
    vid, X = synth.split_square_mesh(N, L=1.0)
    rng = np.random.default_rng(0)
    shift = 0.15 / N * rng.uniform(-1, 1, size=(N * N, 2))
    Xp = X + shift[vid]
    tf, to, ft = g.host_topology(vid, Xp)
    T = Topology(vid, Xp)
    assert np.array_equal(tf, T.tri_facet) and np.array_equal(ft, T.facet_tri)


def test_library_topology_with_walls_matches_oracle(g):
    # an edge with one triangle is a wall: its second side is -1 in both conventions
    from oracle.mesh import Topology
    box = synth.split_square_mesh(3, L=1.0, periodic=False)
    vid, X = synth.split_square_mesh(3)
    holed = (vid[:-1], X[:-1])                   # the torus with one triangle cut out
    for vid, X in (box, holed):
        tf, to, ft = g.host_topology(vid, X)
        T = Topology(vid, X)
        assert np.array_equal(tf, T.tri_facet) and np.array_equal(ft, T.facet_tri)
        assert (ft[:, 1] < 0).sum() == T.boundary.sum() > 0


def _legendre_from_bernstein(k):
    # columns: sqrt(2m+1) P_m(2t-1) in the Bernstein basis C(k,j) t^j (1-t)^(k-j) of [0, 1]
    from math import comb
    from numpy.polynomial import legendre
    t = np.linspace(0.05, 0.95, k + 1)
    bern = np.array([[comb(k, j) * x ** j * (1 - x) ** (k - j) for j in range(k + 1)] for x in t])
    leg = np.array([[np.sqrt(2 * m + 1) * legendre.legval(2 * x - 1, [0] * m + [1]) for m in range(k + 1)] for x in t])
    return np.linalg.solve(bern, leg)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_facet_operator_with_walls_matches_oracle(g, k):
    # the library's condensed facet system on a box equals the oracle's (Bernstein multipliers)
    # after the change to the library's Legendre facet basis; one-dimensional kernel
    from oracle import Discretization
    vid, X = synth.split_square_mesh(3, L=1.0, periodic=False)
    nbr, st, blk, binv = g.host_facet_operator(vid, X, k)
    S = _dense_S(nbr, st, blk)
    d = Discretization(vid, X, k, 0.0)
    B = np.kron(np.eye(d.n_facet), _legendre_from_bernstein(k))
    So = B.T @ d.prepare()["S"].toarray() @ B
    assert np.abs(So - S).max() < 1e-13 * np.abs(S).max()
    ev = np.linalg.eigvalsh(S)
    assert (ev < 1e-10 * ev[-1]).sum() == 1
    assert g.host_lattice(vid, X, k) is None           # walls: no Fourier preconditioner


def test_library_rejects_clockwise_meshes(g):
    from paper_1808_04669_gb300 import DGError
    vid, X = synth.split_square_mesh(3)
    Xc = X.copy()
    Xc[0, [1, 2]] = Xc[0, [2, 1]]
    vc = vid.copy()
    vc[0, [1, 2]] = vc[0, [2, 1]]
    with pytest.raises(DGError) as e:
        g.host_topology(vc, Xc)
    assert e.value.code == -2            # DG_ERR_MESH: clockwise triangle
    with pytest.raises(DGError) as e:
        g.host_reference(4, 0)
    assert e.value.code == -3


@pytest.mark.parametrize("N,k,perturb", [(1, 1, 0.0), (3, 2, 0.0), (4, 3, 0.0), (4, 2, 0.12)])
def test_facet_operator_is_spsd_with_constant_kernel(g, N, k, perturb):
    # eq. (12) condensed: S = sum_T C_T P_T C_T^T is symmetric, positive semi-definite, and its
    # kernel on the torus is the constant multiplier (paired with a constant w)
    vid, X = synth.split_square_mesh(N)
    if perturb:
        rng = np.random.default_rng(1)
        X = X + (perturb * 2 * np.pi / N * rng.uniform(-1, 1, size=(N * N, 2)))[vid]
    nbr, st, blk, binv = g.host_facet_operator(vid, X, k)
    nf, nl = nbr.shape[0], k + 1
    S = np.zeros((nf * nl, nf * nl))
    for f in range(nf):
        for b, c in enumerate([f] + list(nbr[f])):
            S[f * nl:(f + 1) * nl, c * nl:(c + 1) * nl] += blk[st[f], b]
    assert np.abs(S - S.T).max() < 1e-13 * np.abs(S).max()
    ev = np.linalg.eigvalsh(S)
    assert ev[0] > -1e-12 * ev[-1]
    assert (ev < 1e-10 * ev[-1]).sum() == 1
    kern = np.zeros(nf * nl)
    kern[::nl] = 1.0
    assert np.abs(S @ kern).max() < 1e-12 * ev[-1]
    for f in range(nf):
        own = blk[st[f], 0]
        assert np.abs(binv[st[f]] @ own - np.eye(nl)).max() < 1e-12
    if not perturb:
        assert blk.shape[0] <= 3        # three facet orientations on a split-square mesh


def _dense_S(nbr, st, blk):
    nf, nl = nbr.shape[0], blk.shape[-1]
    S = np.zeros((nf * nl, nf * nl))
    for f in range(nf):
        for b, c in enumerate([f] + list(nbr[f])):
            S[f * nl:(f + 1) * nl, c * nl:(c + 1) * nl] += blk[st[f], b]
    return S


@pytest.mark.parametrize("N,k", [(1, 1), (2, 2), (3, 2), (4, 3), (6, 1), (8, 2)])
def test_lattice_fourier_inverse_solves_the_facet_system(g, N, k):
    # the preconditioner of DG_PRECOND_AUTO: z = IDFT(S^(kappa)^+ DFT(r)) must satisfy S z = r for any r
    # without a constant-multiplier component (S is block circulant on the split-square torus)
    vid, X = synth.split_square_mesh(N)
    lat = g.host_lattice(vid, X, k)
    assert lat is not None
    n, fo, sinv = lat
    assert n == N and sorted(fo.ravel().tolist()) == list(range(3 * N * N))
    nbr, st, blk, binv = g.host_facet_operator(vid, X, k)
    S = _dense_S(nbr, st, blk)
    nl = k + 1
    rng = np.random.default_rng(N + k)
    r = rng.standard_normal((3 * N * N, nl))
    r[:, 0] -= r[:, 0].mean()
    # gather into [type, mode, j, i], transform over (j, i), multiply per wavenumber, transform back
    R = np.transpose(r[fo], (0, 3, 1, 2)).reshape(3 * nl, N, N)
    Rh = np.fft.fft2(R)                                  # axes (j, i) -> (kj, ki)
    Zh = np.einsum("ijab,bji->aji", sinv, Rh)            # sinv indexed [ki][kj][C][C]
    Z = np.fft.ifft2(Zh).real.reshape(3, nl, N, N)
    z = np.empty_like(r)
    z[fo] = np.transpose(Z, (0, 2, 3, 1))
    assert np.abs(S @ z.ravel() - r.ravel()).max() < 1e-10 * np.abs(r).max()


def test_lattice_detection_rejects_other_meshes(g):
    vid, X = synth.split_square_mesh(4)
    rng = np.random.default_rng(0)
    Xp = X + (0.1 * rng.uniform(-1, 1, size=(16, 2)))[vid]
    assert g.host_lattice(vid, Xp, 2) is None            # not translation invariant


# ------------------------------------------------------ multilevel preconditioner (host set-up)
def _ml_mesh(N, k, walls, perturb=0.0):
    vid, X = synth.split_square_mesh(N, L=1.0, periodic=not walls)
    if perturb:
        rng = np.random.default_rng(3)
        X = X + (perturb / N * rng.uniform(-1, 1, size=(N * N, 2)))[vid]
    return vid, X


def _apply_S(nbr, st, blk, x):
    nl = blk.shape[-1]
    x = x.reshape(-1, nl)
    y = np.einsum("fij,fj->fi", blk[st, 0], x)
    for b in range(4):
        y += np.einsum("fij,fj->fi", blk[st, b + 1], x[nbr[:, b]])
    return y.ravel()


@pytest.mark.parametrize("N,k,walls,perturb", [(32, 1, True, 0.0), (32, 2, True, 0.0), (32, 3, True, 0.0),
                                               (32, 3, False, 0.15), (8, 2, True, 0.0)])
def test_multilevel_pcg_solves_the_facet_system_in_few_iterations(g, N, k, walls, perturb):
    # block Jacobi needs O(N) iterations (hundreds here); one V-cycle per iteration keeps it at ~35
    vid, X = _ml_mesh(N, k, walls, perturb)
    nbr, st, blk, binv = g.host_facet_operator(vid, X, k)
    nl = k + 1
    rhs = np.random.default_rng(N + k).standard_normal(nbr.shape[0] * nl)
    res = g.host_multilevel(vid, X, k, g=rhs, rtol=1e-12)
    sizes = [n for n, _ in res["levels"]]
    assert res["levels"][0] == (nbr.shape[0], nl)
    assert all(a >= b for a, b in zip(sizes, sizes[1:])) and res["coarsest"] <= 1024
    assert 0 < res["iters"] <= 45, res["iters"]
    # the solution: S lam = g up to the constant multiplier (mode 0 on every facet)
    b = rhs.reshape(-1, nl).copy()
    b[:, 0] -= b[:, 0].mean()
    r = b.ravel() - _apply_S(nbr, st, blk, res["lam"])
    r = r.reshape(-1, nl)
    r[:, 0] -= r[:, 0].mean()
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("N,k", [(8, 2), (16, 2), (32, 1)])
def test_multilevel_v_cycle_is_symmetric_positive_on_the_range(g, N, k):
    # PCG needs a symmetric positive definite preconditioner (on the complement of the constant
    # multiplier): the same Chebyshev polynomial before and after the coarse correction. The
    # coarsest pseudo-inverse comes from an eigen-decomposition at 8^2 (208 rows, the mode-0
    # operator itself) and from elimination on the operator made definite along the constant
    # at 16^2 (800 rows, likewise) and 32^2 (512 rows, after aggregation)
    vid, X = _ml_mesh(N, k, True)
    nl = k + 1
    nf = g.host_facet_operator(vid, X, k)[0].shape[0]
    assert g.host_multilevel(vid, X, k)["coarsest"] == {8: 208, 16: 800, 32: 512}[N]
    rng = np.random.default_rng(5)
    r = rng.standard_normal((4, nf * nl))
    r.reshape(4, nf, nl)[:, :, 0] -= r.reshape(4, nf, nl)[:, :, 0].mean(1, keepdims=True)
    z = g.host_multilevel(vid, X, k, r=r)["z"]
    G = r @ z.T
    assert np.abs(G - G.T).max() <= 1e-12 * np.abs(G).max()
    assert np.linalg.eigvalsh(0.5 * (G + G.T)).min() > 0


@pytest.mark.parametrize("N,k", [(2, 1), (2, 2), (3, 2)])
def test_three_dimensional_setup_projects_like_the_oracle(g, N, k):
    # the library's 3-D host set-up (topology, canonical faces, class operators, face stencil and
    # the assembled multilevel hierarchy) gives the oracle's L2 projection onto the
    # divergence-free space, computed on the host
    from oracle.dg3 import Discretization3
    from synth.mesh3 import abc_flow, kuhn_cube_mesh, sample_lattice3
    vid, X = kuhn_cube_mesh(N)
    v = sample_lattice3(abc_flow(), X, k) + 0.3 * np.random.default_rng(N).standard_normal((6 * N ** 3, (k + 1) * (k + 2) * (k + 3) // 6, 3))
    out, its = g.host_project3(vid, X, k, v)
    d = Discretization3(vid, X, k, 0.0)
    ref = d.to_lattice(d.project(d.from_lattice(v)))
    assert np.linalg.norm(out - ref) < 1e-11 * np.linalg.norm(ref)
    assert 0 < its < 60


@pytest.mark.parametrize("N", [2, 3])
def test_three_dimensional_face_numbering_matches_the_oracle(g, N):
    # dg3_host_faces: faces in order of first appearance over (tetrahedron, local face), the two
    # sides and local indices as the oracle's topology finds them, vertex ids sorted
    from oracle.dg3 import Topology3
    from synth.mesh3 import kuhn_cube_mesh
    vid, X = kuhn_cube_mesh(N)
    ft, fl, fv = g.host_faces3(vid, X)
    T = Topology3(vid, X)
    assert ft.shape == (T.n_face, 2) and fv.shape == (T.n_face, 3)
    assert np.array_equal(ft, T.face_tet) and np.array_equal(fl.astype(np.int64), T.face_loc)
    for f in range(T.n_face):
        loc = [v for v in range(4) if v != fl[f, 0]]
        assert list(fv[f]) == sorted(int(vid[ft[f, 0], v]) for v in loc)
        # the other side sees the same three periodic vertex ids
        loc1 = [v for v in range(4) if v != fl[f, 1]]
        assert sorted(int(vid[ft[f, 1], v]) for v in loc1) == list(fv[f])
