"""GB300-native explicit divergence-free DG (Fu, arXiv:1808.04669): Python binding of libdgdf.

The library (C ABI in include/dgdf.h) holds the whole hot path: the SSP-RK3
stage residual, the hybrid-mixed facet solve and the recovery run as CUDA
kernels for sm_103a. This module only marshals arguments: numpy arrays are
passed as host pointers, torch CUDA tensors as device pointers on their stream.
"""
import ctypes

import numpy as np

from . import _native
from ._native import DGError, DGParams, check, lib

FP64 = 0
MIXED = 1
# explicit schemes of DGMesh.step
SSPRK3 = 0
EULER = 1
RK4 = 2
PRECOND_AUTO = 0
PRECOND_BLOCK_JACOBI = 1
PRECOND_MULTILEVEL = 2


def _ptr(a):
    """(pointer, on_device) of a C-contiguous float64 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("need a C-contiguous float64 array")
        return a.ctypes.data_as(ctypes.c_void_p), 0
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("need a contiguous float64 tensor")
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(type(a))


class DGMesh:
    """One mesh and its state, owned by libdgdf (dg_mesh_create ... dg_mesh_destroy)."""

    def __init__(self, tri_vertex_ids, tri_coords, k, nu, alpha=2.0, precision=FP64, cg_rtol=1e-13,
                 cg_maxit=20000, stream=None, precond=PRECOND_AUTO, boundary=None, inflow=None):
        """boundary: kind of every triangle edge [n_tri, 3] (0 wall, 1 inflow, 2 outflow; edge e
        is opposite vertex e; read on boundary edges), or None for walls (dg_mesh_create_ex);
        inflow: u_in at the k+1 equispaced points of every edge [n_tri, 3, k+1, 2] (set_inflow)."""
        L = lib()
        vid = np.ascontiguousarray(tri_vertex_ids, dtype=np.int64)
        X = np.ascontiguousarray(tri_coords, dtype=np.float64)
        if vid.ndim != 2 or vid.shape[1] != 3 or X.shape != (vid.shape[0], 3, 2):
            raise ValueError("tri_vertex_ids [n,3] and tri_coords [n,3,2] expected")
        kinds = None
        if boundary is not None:
            kinds = np.ascontiguousarray(boundary, dtype=np.int8)
            if kinds.shape != (vid.shape[0], 3):
                raise ValueError("boundary [n_tri, 3] expected")
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except Exception:
                stream = 0
        self.params = DGParams(int(k), float(nu), float(alpha), int(precision), float(cg_rtol), int(cg_maxit),
                               ctypes.c_void_p(int(stream)), int(precond))
        h = ctypes.c_void_p()
        check(L.dg_mesh_create_ex(vid.shape[0], vid.ctypes.data_as(ctypes.c_void_p),
                                  X.ctypes.data_as(ctypes.c_void_p),
                                  None if kinds is None else kinds.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.byref(self.params), ctypes.byref(h)), "dg_mesh_create_ex")
        self._h = h
        info = self.info()
        self.n_tri, self.n_facet, self.k, self.n_lat = (int(v) for v in info[:4])
        self.n_class, self.n_stencil = int(info[4]), int(info[5])
        self.n_vel_dofs, self.n_lam_dofs = int(info[6]), int(info[7])
        self.nw = self.k * (self.k + 1) // 2
        if inflow is not None:
            self.set_inflow(inflow)

    def set_inflow(self, vals):
        """Inflow velocity at the k+1 equispaced points of every triangle edge, in the triangle's
        counter-clockwise direction [n_tri, 3, k+1, 2] (dg_set_inflow; read on inflow edges)."""
        v = np.ascontiguousarray(vals, dtype=np.float64)
        if v.shape != (self.n_tri, 3, self.k + 1, 2):
            raise ValueError("inflow values [n_tri, 3, k+1, 2] expected")
        check(lib().dg_set_inflow(self._h, v.ctypes.data_as(ctypes.c_void_p)), "dg_set_inflow")

    def close(self):
        if getattr(self, "_h", None):
            lib().dg_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self):
        out = (ctypes.c_int64 * 8)()
        check(lib().dg_mesh_info(self._h, out), "dg_mesh_info")
        return list(out)

    def set_velocity(self, vals):
        if isinstance(vals, np.ndarray):
            vals = np.ascontiguousarray(vals, dtype=np.float64)
        p, dev = _ptr(vals)
        check(lib().dg_set_velocity(self._h, p, dev), "dg_set_velocity")

    def get_velocity(self, out=None):
        if out is None:
            out = np.empty((self.n_tri, self.n_lat, 2))
        p, dev = _ptr(out)
        check(lib().dg_get_velocity(self._h, p, dev), "dg_get_velocity")
        return out

    def project_divfree(self):
        check(lib().dg_project_divfree(self._h), "dg_project_divfree")

    def rk3_step(self, dt, nsteps=1):
        check(lib().dg_rk3_step(self._h, float(dt), int(nsteps)), "dg_rk3_step")

    def step(self, dt, nsteps=1, scheme=SSPRK3):
        """nsteps steps of SSPRK3, EULER or RK4 (dg_step)."""
        check(lib().dg_step(self._h, int(scheme), float(dt), int(nsteps)), "dg_step")

    def get_pressure(self, with_facet=True, out=None):
        if out is None:
            pe = np.empty((self.n_tri, self.nw))
            pf = np.empty((self.n_facet, self.k + 1)) if with_facet else None
        else:
            pe, pf = out
        p1, dev = _ptr(pe)
        p2 = _ptr(pf)[0] if pf is not None else None
        check(lib().dg_get_pressure(self._h, p1, p2, dev), "dg_get_pressure")
        return pe, pf

    def eval_residual(self, out=None):
        if out is None:
            out = np.empty((self.n_tri, self.n_lat, 2))
        p, dev = _ptr(out)
        check(lib().dg_eval_residual(self._h, p, dev), "dg_eval_residual")
        return out

    def diagnostics(self):
        out = (ctypes.c_double * 8)()
        check(lib().dg_get_diagnostics(self._h, out), "dg_get_diagnostics")
        keys = ("energy", "enstrophy", "max_div", "max_jump", "last_iters", "total_iters", "solves", "last_relres")
        return dict(zip(keys, list(out)))

    def set_coefficients(self, coef):
        if isinstance(coef, np.ndarray):
            coef = np.ascontiguousarray(coef, dtype=np.float64)
        p, dev = _ptr(coef)
        check(lib().dg_set_coefficients(self._h, p, dev), "dg_set_coefficients")

    def get_coefficients(self, out=None):
        if out is None:
            out = np.empty((self.n_tri, 2 * self.n_lat))
        p, dev = _ptr(out)
        check(lib().dg_get_coefficients(self._h, p, dev), "dg_get_coefficients")
        return out

    def set_viscosity(self, nu):
        check(lib().dg_set_viscosity(self._h, float(nu)), "dg_set_viscosity")

    def rk3_vjp(self, dt, nsteps, ubar, checkpoint_every=0, out=None):
        """(u0bar, nubar) for the cotangent ubar of the state after nsteps steps (see dg_rk3_vjp)."""
        if isinstance(ubar, np.ndarray):
            ubar = np.ascontiguousarray(ubar, dtype=np.float64)
        if out is None:
            out = np.empty((self.n_tri, 2 * self.n_lat)) if isinstance(ubar, np.ndarray) else ubar.new_empty(ubar.shape)
        p1, dev = _ptr(ubar)
        p2, _ = _ptr(out)
        nb = ctypes.c_double()
        check(lib().dg_rk3_vjp(self._h, float(dt), int(nsteps), int(checkpoint_every), p1, p2, ctypes.byref(nb), dev),
              "dg_rk3_vjp")
        return out, nb.value

    def solver_stats(self):
        out = (ctypes.c_double * 8)()
        check(lib().dg_get_solver_stats(self._h, out), "dg_get_solver_stats")
        keys = ("last_iters", "total_iters", "solves", "last_relres", "last_sweeps", "total_sweeps",
                "precond_kind", "blocks")
        d = dict(zip(keys, list(out)))
        d["lattice"] = 1.0 if d["precond_kind"] == 1.0 else 0.0
        d["preconditioner"] = {0.0: "block Jacobi", 1.0: "lattice FFT", 2.0: "multilevel"}[d["precond_kind"]]
        return d

    def set_tensor_cores(self, enable):
        """Tensor-core (tcgen05) recovery on or off (dg_set_tensor_cores)."""
        check(lib().dg_set_tensor_cores(self._h, int(bool(enable))), "dg_set_tensor_cores")

    def set_energy_watchdog(self, rel_tol):
        """Flag growth of ||u||^2 by more than rel_tol in a step (dg_set_energy_watchdog); 0 turns it off."""
        check(lib().dg_set_energy_watchdog(self._h, float(rel_tol)), "dg_set_energy_watchdog")

    def solver_history(self, enable=None):
        """Per-iteration (relres, r.z, p.Sp, alpha) of the last multilevel solve (dg_solver_history);
        enable=True/False starts/stops recording."""
        mode = 2 if enable is None else (1 if enable else 0)
        out = np.zeros(4 * 512)
        n = ctypes.c_int(0)
        check(lib().dg_solver_history(self._h, mode, out.ctypes.data_as(ctypes.c_void_p), out.size, ctypes.byref(n)),
              "dg_solver_history")
        return out.reshape(512, 4)[:min(n.value + 1, 512)]

    def test_multilevel_apply(self, r):
        """One device V-cycle z = M r of the multilevel preconditioner (dg_test_multilevel_apply)."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty_like(r)
        check(lib().dg_test_multilevel_apply(self._h, r.ctypes.data_as(ctypes.c_void_p),
                                             z.ctypes.data_as(ctypes.c_void_p), 0), "dg_test_multilevel_apply")
        return z

    def test_barrier_fault(self, spin_limit=0, skip_block=-1):
        """Failure-detection test hook (dg_test_barrier_fault): bounded barrier waits of the solvers."""
        check(lib().dg_test_barrier_fault(self._h, int(spin_limit), int(skip_block)), "dg_test_barrier_fault")

    def profile(self, enable):
        n = 16
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        check(lib().dg_profile(self._h, int(enable), ms, cnt, n), "dg_profile")
        res = {}
        for i in range(n):
            name = lib().dg_kernel_name(i)
            if name is None:
                break
            res[name.decode()] = (ms[i], int(cnt[i]))
        return res


class DGMesh3:
    """One closed tetrahedral mesh and its state (include/dgdf3.h: dg3_mesh_create ... dg3_mesh_destroy),
    FP64, k = 1 or 2; multilevel PCG by default, block Jacobi with precond=PRECOND_BLOCK_JACOBI."""

    def __init__(self, tet_vertex_ids, tet_coords, k, nu, alpha=2.0, cg_rtol=1e-13, cg_maxit=20000, stream=None,
                 precond=PRECOND_AUTO):
        L = lib()
        vid = np.ascontiguousarray(tet_vertex_ids, dtype=np.int64)
        X = np.ascontiguousarray(tet_coords, dtype=np.float64)
        if vid.ndim != 2 or vid.shape[1] != 4 or X.shape != (vid.shape[0], 4, 3):
            raise ValueError("tet_vertex_ids [n,4] and tet_coords [n,4,3] expected")
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except Exception:
                stream = 0
        self.params = DGParams(int(k), float(nu), float(alpha), FP64, float(cg_rtol), int(cg_maxit),
                               ctypes.c_void_p(int(stream)), int(precond))
        h = ctypes.c_void_p()
        check(L.dg3_mesh_create(vid.shape[0], vid.ctypes.data_as(ctypes.c_void_p), X.ctypes.data_as(ctypes.c_void_p),
                                ctypes.byref(self.params), ctypes.byref(h)), "dg3_mesh_create")
        self._h = h
        info = self.info()
        self.n_tet, self.n_face, self.k, self.n_lat = (int(v) for v in info[:4])
        self.n_class, self.n_stencil = int(info[4]), int(info[5])
        self.n_vel_dofs, self.n_lam_dofs = int(info[6]), int(info[7])

    def close(self):
        if getattr(self, "_h", None):
            lib().dg3_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        out = (ctypes.c_int64 * 8)()
        check(lib().dg3_mesh_info(self._h, out), "dg3_mesh_info")
        return list(out)

    def set_velocity(self, vals):
        if isinstance(vals, np.ndarray):
            vals = np.ascontiguousarray(vals, dtype=np.float64)
        p, dev = _ptr(vals)
        check(lib().dg3_set_velocity(self._h, p, dev), "dg3_set_velocity")

    def get_velocity(self, out=None):
        if out is None:
            out = np.empty((self.n_tet, self.n_lat, 3))
        p, dev = _ptr(out)
        check(lib().dg3_get_velocity(self._h, p, dev), "dg3_get_velocity")
        return out

    def project_divfree(self):
        check(lib().dg3_project_divfree(self._h), "dg3_project_divfree")

    def rk3_step(self, dt, nsteps=1):
        check(lib().dg3_rk3_step(self._h, float(dt), int(nsteps)), "dg3_rk3_step")

    def eval_residual(self, out=None):
        if out is None:
            out = np.empty((self.n_tet, self.n_lat, 3))
        p, dev = _ptr(out)
        check(lib().dg3_eval_residual(self._h, p, dev), "dg3_eval_residual")
        return out

    def get_pressure(self, with_face=True):
        """(p_elem [n_tet, n_lat3(k-1)], p_face [n_face, (k+1)(k+2)/2] or None) of the current
        state, mean-free (dg3_get_pressure)."""
        k = self.k
        pe = np.empty((self.n_tet, k * (k + 1) * (k + 2) // 6))
        pf = np.empty((self.n_face, (k + 1) * (k + 2) // 2)) if with_face else None
        p, dev = _ptr(pe)
        q = _ptr(pf)[0] if pf is not None else None
        check(lib().dg3_get_pressure(self._h, p, q, dev), "dg3_get_pressure")
        return pe, pf

    def diagnostics(self):
        out = (ctypes.c_double * 8)()
        check(lib().dg3_get_diagnostics(self._h, out), "dg3_get_diagnostics")
        keys = ("energy", "enstrophy", "max_div", "max_jump", "last_iters", "last_relres", "total_iters", "solves")
        return dict(zip(keys, list(out)))


class DGBatch:
    """An ensemble of DGMesh members advanced together (dg_batch_create / dg_batch_rk3_step)."""

    def __init__(self, meshes, stream=None):
        L = lib()
        self.meshes = list(meshes)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        arr = (ctypes.c_void_p * len(self.meshes))(*[m._h.value for m in self.meshes])
        h = ctypes.c_void_p()
        check(L.dg_batch_create(len(self.meshes), arr, ctypes.c_void_p(int(stream)), ctypes.byref(h)),
              "dg_batch_create")
        self._h = h

    def rk3_step(self, dt, nsteps=1):
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (len(self.meshes),)))
        check(lib().dg_batch_rk3_step(self._h, d.ctypes.data_as(ctypes.c_void_p), int(nsteps)), "dg_batch_rk3_step")

    def set_lanes(self, lanes):
        """Parallel branches of the captured step: 0 = autotune on the next call, or 1, 2, 4, 8, 16."""
        check(lib().dg_batch_set_lanes(self._h, int(lanes)), "dg_batch_set_lanes")

    def tuning(self):
        """(lanes in use, {lanes: measured ms per step}) (dg_batch_get_tuning)."""
        ln = ctypes.c_int(0)
        ms = (ctypes.c_double * 5)()
        check(lib().dg_batch_get_tuning(self._h, ctypes.byref(ln), ms), "dg_batch_get_tuning")
        return ln.value, {c: ms[i] for i, c in enumerate((1, 2, 4, 8, 16)) if ms[i] >= 0}

    def close(self):
        if getattr(self, "_h", None):
            lib().dg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def host_topology(tri_vertex_ids, tri_coords):
    """Facet topology computed by the library's host set-up (no GPU): (tri_facet, tri_orient, facet_tri)."""
    L = lib()
    vid = np.ascontiguousarray(tri_vertex_ids, dtype=np.int64)
    X = np.ascontiguousarray(tri_coords, dtype=np.float64)
    nf = ctypes.c_int64()
    V = ctypes.c_void_p
    check(L.dg_host_topology(vid.shape[0], vid.ctypes.data_as(V), X.ctypes.data_as(V), ctypes.byref(nf),
                             None, None, None), "dg_host_topology")
    tf = np.empty((vid.shape[0], 3), dtype=np.int32)
    to = np.empty((vid.shape[0], 3), dtype=np.int8)
    ft = np.empty((nf.value, 2), dtype=np.int32)
    check(L.dg_host_topology(vid.shape[0], vid.ctypes.data_as(V), X.ctypes.data_as(V), ctypes.byref(nf),
                             tf.ctypes.data_as(V), to.ctypes.data_as(V), ft.ctypes.data_as(V)), "dg_host_topology")
    return tf, to, ft


def host_reference(k, table):
    """Reference tables of the library's host set-up (see include/dgdf_host.h)."""
    L = lib()
    n = ctypes.c_int64()
    check(L.dg_host_reference(int(k), int(table), None, 0, ctypes.byref(n)), "dg_host_reference")
    out = np.empty(n.value)
    check(L.dg_host_reference(int(k), int(table), out.ctypes.data_as(ctypes.c_void_p), n.value, ctypes.byref(n)),
          "dg_host_reference")
    return out


def host_facet_operator(tri_vertex_ids, tri_coords, k, alpha=2.0):
    """The library's condensed facet system (include/dgdf_host.h): (facet_nbr, stencil, blocks, binv)."""
    L = lib()
    vid = np.ascontiguousarray(tri_vertex_ids, dtype=np.int64)
    X = np.ascontiguousarray(tri_coords, dtype=np.float64)
    V = ctypes.c_void_p
    nf, ns = ctypes.c_int64(), ctypes.c_int64()
    args = (vid.shape[0], vid.ctypes.data_as(V), X.ctypes.data_as(V), int(k), float(alpha), ctypes.byref(nf),
            ctypes.byref(ns))
    check(L.dg_host_facet_operator(*args, None, None, None, None, 0), "dg_host_facet_operator")
    nl = k + 1
    nbr = np.empty((nf.value, 4), dtype=np.int32)
    st = np.empty(nf.value, dtype=np.int32)
    blk = np.empty((ns.value, 5, nl, nl))
    binv = np.empty((ns.value, nl, nl))
    check(L.dg_host_facet_operator(*args, nbr.ctypes.data_as(V), st.ctypes.data_as(V), blk.ctypes.data_as(V),
                                   binv.ctypes.data_as(V), ns.value), "dg_host_facet_operator")
    return nbr, st, blk, binv


def host_lattice(tri_vertex_ids, tri_coords, k, alpha=2.0):
    """The lattice structure and inverse Fourier symbol of the facet operator (include/dgdf_host.h).

    Returns (N, facet_of [3][N][N], sinv [N][N][C][C] complex) or None if the mesh is not a lattice.
    """
    L = lib()
    vid = np.ascontiguousarray(tri_vertex_ids, dtype=np.int64)
    X = np.ascontiguousarray(tri_coords, dtype=np.float64)
    V = ctypes.c_void_p
    N = ctypes.c_int64()
    args = (vid.shape[0], vid.ctypes.data_as(V), X.ctypes.data_as(V), int(k), float(alpha), ctypes.byref(N))
    rc = L.dg_host_lattice(*args, None, None, 0)
    if rc == -3:
        return None
    check(rc, "dg_host_lattice")
    n = N.value
    C = 3 * (k + 1)
    fo = np.empty((3, n, n), dtype=np.int32)
    s = np.empty((n, n, C, C, 2))
    check(L.dg_host_lattice(*args, fo.ctypes.data_as(V), s.ctypes.data_as(V), s.size), "dg_host_lattice")
    return n, fo, s[..., 0] + 1j * s[..., 1]


def host_multilevel(tri_vertex_ids, tri_coords, k, alpha=2.0, r=None, g=None, rtol=1e-13):
    """The multilevel preconditioner of the facet system built on the host (include/dgdf_host.h).

    Returns a dict with the level sizes; with r ([nr, n_facet (k+1)]) also z = M r; with g also
    the PCG solution lam and its iteration count.
    """
    L = lib()
    vid = np.ascontiguousarray(tri_vertex_ids, dtype=np.int64)
    X = np.ascontiguousarray(tri_coords, dtype=np.float64)
    V = ctypes.c_void_p
    info = (ctypes.c_int64 * 34)()
    nr, rp, zp, z = 0, None, None, None
    if r is not None:
        r = np.ascontiguousarray(np.atleast_2d(r), dtype=np.float64)
        nr = r.shape[0]
        z = np.empty_like(r)
        rp, zp = r.ctypes.data_as(V), z.ctypes.data_as(V)
    gp, lp, lam, it = None, None, None, ctypes.c_int64(0)
    if g is not None:
        g = np.ascontiguousarray(g, dtype=np.float64).ravel()
        lam = np.empty_like(g)
        gp, lp = g.ctypes.data_as(V), lam.ctypes.data_as(V)
    check(L.dg_host_multilevel(vid.shape[0], vid.ctypes.data_as(V), X.ctypes.data_as(V), int(k), float(alpha), info,
                               nr, rp, zp, gp, lp, float(rtol), ctypes.byref(it)), "dg_host_multilevel")
    nlev = int(info[0])
    return {"levels": [(int(info[2 + 2 * l]), int(info[3 + 2 * l])) for l in range(nlev)], "coarsest": int(info[1]),
            "z": z, "lam": lam, "iters": int(it.value) if g is not None else None}


def host_faces3(tet_vertex_ids, tet_coords):
    """Face numbering of the 3-D set-up (include/dgdf_host.h, dg3_host_faces): (face_tet [n_face, 2],
    face_loc [n_face, 2], face_vid [n_face, 3] sorted periodic vertex ids)."""
    vid = np.ascontiguousarray(tet_vertex_ids, dtype=np.int64)
    X = np.ascontiguousarray(tet_coords, dtype=np.float64)
    V = ctypes.c_void_p
    nf = ctypes.c_int64(0)
    check(lib().dg3_host_faces(vid.shape[0], vid.ctypes.data_as(V), X.ctypes.data_as(V), ctypes.byref(nf),
                               None, None, None), "dg3_host_faces")
    ft = np.empty((nf.value, 2), dtype=np.int64)
    fl = np.empty((nf.value, 2), dtype=np.int8)
    fv = np.empty((nf.value, 3), dtype=np.int64)
    check(lib().dg3_host_faces(vid.shape[0], vid.ctypes.data_as(V), X.ctypes.data_as(V), None,
                               ft.ctypes.data_as(V), fl.ctypes.data_as(V), fv.ctypes.data_as(V)), "dg3_host_faces")
    return ft, fl, fv


def host_project3(tet_vertex_ids, tet_coords, k, vals, alpha=2.0):
    """Host-side L2 projection of a 3-D field onto the divergence-free space from the library's own
    set-up (include/dgdf_host.h, dg3_host_project): (lattice values, PCG iterations)."""
    vid = np.ascontiguousarray(tet_vertex_ids, dtype=np.int64)
    X = np.ascontiguousarray(tet_coords, dtype=np.float64)
    v = np.ascontiguousarray(vals, dtype=np.float64)
    out = np.empty_like(v)
    it = ctypes.c_int64()
    check(lib().dg3_host_project(vid.shape[0], vid.ctypes.data_as(ctypes.c_void_p), X.ctypes.data_as(ctypes.c_void_p),
                                 int(k), float(alpha), v.ctypes.data_as(ctypes.c_void_p),
                                 out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(it)), "dg3_host_project")
    return out, int(it.value)


def facet_solve_noalloc(k, facet_nbr, stencil, blocks, binv, g, lam, rtol=1e-13, maxit=20000, stream=None):
    """dg_facet_solve_noalloc on caller-owned CUDA tensors (torch); lam is updated in place.

    For callers that cannot allocate: the library allocates nothing here (see include/dgdf.h).
    Returns (iterations, relative residual).
    """
    import torch
    for t, dt in ((facet_nbr, torch.int32), (stencil, torch.int32), (blocks, torch.float64), (binv, torch.float64),
                  (g, torch.float64), (lam, torch.float64)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError("need contiguous CUDA tensors of the documented dtypes")
    # the kernel trusts these sizes: a short array would be read or written past its end
    nl = int(k) + 1
    nf = facet_nbr.shape[0] if facet_nbr.dim() == 2 else -1
    if facet_nbr.dim() != 2 or facet_nbr.shape[1] != 4:
        raise ValueError("facet_nbr must be [n_facet, 4]")
    if tuple(stencil.shape) != (nf,):
        raise ValueError("stencil must be [n_facet]")
    if g.numel() != nf * nl or lam.numel() != nf * nl:
        raise ValueError("g and lam must hold n_facet * (k + 1) values")
    if blocks.dim() != 4 or tuple(blocks.shape[1:]) != (5, nl, nl):
        raise ValueError("blocks must be [n_stencil, 5, k + 1, k + 1]")
    if tuple(binv.shape) != (blocks.shape[0], nl, nl):
        raise ValueError("binv must be [n_stencil, k + 1, k + 1] with the n_stencil of blocks")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    it = ctypes.c_int()
    rr = ctypes.c_double()
    V = ctypes.c_void_p
    check(lib().dg_facet_solve_noalloc(int(k), int(facet_nbr.shape[0]), V(facet_nbr.data_ptr()), V(stencil.data_ptr()),
                                       V(blocks.data_ptr()), V(binv.data_ptr()), V(g.data_ptr()), V(lam.data_ptr()),
                                       float(rtol), int(maxit), V(int(stream)), ctypes.byref(it), ctypes.byref(rr)),
          "dg_facet_solve_noalloc")
    return it.value, rr.value


__all__ = ["DGMesh", "DGMesh3", "DGBatch", "DGError", "FP64", "MIXED", "PRECOND_AUTO", "PRECOND_BLOCK_JACOBI", "PRECOND_MULTILEVEL", "host_topology", "host_reference", "host_facet_operator", "host_lattice", "host_multilevel", "host_project3", "host_faces3", "facet_solve_noalloc",
           "lib"]
