"""ctypes binding of libdgdf (include/dgdf.h, include/dgdf_host.h, include/dgdf3.h): argument marshalling only.

The library must have been built in-tree (``paper_1808_04669_gb300.build``);
there is no fallback: a missing library raises ImportError.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgdf.so")

DG_OK = 0
STATUS = {0: "DG_OK", -1: "DG_ERR_INVALID_ARG", -2: "DG_ERR_MESH", -3: "DG_ERR_UNSUPPORTED", -4: "DG_ERR_CUDA",
          -5: "DG_ERR_NOT_CONVERGED", -6: "DG_ERR_NONFINITE", -7: "DG_ERR_OOM", -8: "DG_ERR_UNSTABLE"}

EXPORTS = ["dg_mesh_create", "dg_mesh_create_ex", "dg_set_inflow", "dg_mesh_destroy", "dg_mesh_info", "dg_set_velocity", "dg_get_velocity",
           "dg_project_divfree", "dg_rk3_step", "dg_step", "dg_batch_create", "dg_batch_destroy", "dg_batch_rk3_step", "dg_batch_set_lanes", "dg_batch_get_tuning", "dg_get_pressure", "dg_eval_residual", "dg_set_coefficients", "dg_get_coefficients",
           "dg_set_viscosity", "dg_rk3_vjp", "dg_get_diagnostics", "dg_get_solver_stats", "dg_facet_solve_noalloc",
           "dg_set_energy_watchdog", "dg_set_tensor_cores", "dg_solver_history", "dg_test_multilevel_apply", "dg_test_barrier_fault", "dg_profile", "dg_kernel_name", "dg_last_error", "dg_host_topology", "dg_host_reference",
           "dg_host_facet_operator", "dg_host_lattice", "dg_host_multilevel",
           "dg3_mesh_create", "dg3_mesh_destroy", "dg3_mesh_info", "dg3_set_velocity", "dg3_get_velocity",
           "dg3_project_divfree", "dg3_rk3_step", "dg3_eval_residual", "dg3_get_pressure", "dg3_get_diagnostics",
           "dg3_host_project", "dg3_host_faces"]


class DGParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("nu", ctypes.c_double), ("alpha", ctypes.c_double),
                ("precision", ctypes.c_int), ("cg_rtol", ctypes.c_double), ("cg_maxit", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("precond", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdgdf.so is not built (run paper_1808_04669_gb300.build.build()): %s" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, I64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    sig = {
        "dg_mesh_create": (ctypes.c_int, [I64, P, P, ctypes.POINTER(DGParams), ctypes.POINTER(ctypes.c_void_p)]),
        "dg_mesh_create_ex": (ctypes.c_int, [I64, P, P, P, ctypes.POINTER(DGParams), ctypes.POINTER(ctypes.c_void_p)]),
        "dg_set_inflow": (ctypes.c_int, [P, P]),
        "dg_mesh_destroy": (ctypes.c_int, [P]),
        "dg3_mesh_create": (ctypes.c_int, [I64, P, P, ctypes.POINTER(DGParams), ctypes.POINTER(ctypes.c_void_p)]),
        "dg3_mesh_destroy": (ctypes.c_int, [P]),
        "dg3_mesh_info": (ctypes.c_int, [P, P]),
        "dg3_set_velocity": (ctypes.c_int, [P, P, ctypes.c_int]),
        "dg3_get_velocity": (ctypes.c_int, [P, P, ctypes.c_int]),
        "dg3_project_divfree": (ctypes.c_int, [P]),
        "dg3_rk3_step": (ctypes.c_int, [P, D, I64]),
        "dg3_eval_residual": (ctypes.c_int, [P, P, ctypes.c_int]),
        "dg3_get_pressure": (ctypes.c_int, [P, P, P, ctypes.c_int]),
        "dg3_host_faces": (ctypes.c_int, [ctypes.c_int64, P, P, P, P, P, P]),
        "dg3_get_diagnostics": (ctypes.c_int, [P, P]),
        "dg3_host_project": (ctypes.c_int, [I64, P, P, ctypes.c_int, D, P, P, P]),
        "dg_mesh_info": (ctypes.c_int, [P, P]),
        "dg_set_velocity": (ctypes.c_int, [P, P, ctypes.c_int]),
        "dg_get_velocity": (ctypes.c_int, [P, P, ctypes.c_int]),
        "dg_project_divfree": (ctypes.c_int, [P]),
        "dg_rk3_step": (ctypes.c_int, [P, D, I64]),
        "dg_step": (ctypes.c_int, [P, ctypes.c_int, D, I64]),
        "dg_batch_create": (ctypes.c_int, [ctypes.c_int, P, P, ctypes.POINTER(ctypes.c_void_p)]),
        "dg_batch_destroy": (ctypes.c_int, [P]),
        "dg_batch_rk3_step": (ctypes.c_int, [P, P, I64]),
        "dg_batch_set_lanes": (ctypes.c_int, [P, ctypes.c_int]),
        "dg_batch_get_tuning": (ctypes.c_int, [P, P, P]),
        "dg_get_pressure": (ctypes.c_int, [P, P, P, ctypes.c_int]),
        "dg_eval_residual": (ctypes.c_int, [P, P, ctypes.c_int]),
        "dg_set_coefficients": (ctypes.c_int, [P, P, ctypes.c_int]),
        "dg_get_coefficients": (ctypes.c_int, [P, P, ctypes.c_int]),
        "dg_set_viscosity": (ctypes.c_int, [P, D]),
        "dg_rk3_vjp": (ctypes.c_int, [P, D, I64, I64, P, P, P, ctypes.c_int]),
        "dg_get_diagnostics": (ctypes.c_int, [P, P]),
        "dg_get_solver_stats": (ctypes.c_int, [P, P]),
        "dg_facet_solve_noalloc": (ctypes.c_int, [ctypes.c_int, I64, P, P, P, P, P, P, D, ctypes.c_int, P, P, P]),
        "dg_set_energy_watchdog": (ctypes.c_int, [P, D]),
        "dg_test_barrier_fault": (ctypes.c_int, [P, I64, ctypes.c_int]),
        "dg_test_multilevel_apply": (ctypes.c_int, [P, P, P, ctypes.c_int]),
        "dg_solver_history": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int, P]),
        "dg_set_tensor_cores": (ctypes.c_int, [P, ctypes.c_int]),
        "dg_profile": (ctypes.c_int, [P, ctypes.c_int, P, P, ctypes.c_int]),
        "dg_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
        "dg_last_error": (ctypes.c_char_p, []),
        "dg_host_topology": (ctypes.c_int, [I64, P, P, P, P, P, P]),
        "dg_host_reference": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, I64, P]),
        "dg_host_facet_operator": (ctypes.c_int, [I64, P, P, ctypes.c_int, D, P, P, P, P, P, P, I64]),
        "dg_host_lattice": (ctypes.c_int, [I64, P, P, ctypes.c_int, D, P, P, P, I64]),
        "dg_host_multilevel": (ctypes.c_int, [I64, P, P, ctypes.c_int, D, P, ctypes.c_int, P, P, P, P, D, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class DGError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().dg_last_error().decode(errors="replace")
        super().__init__("%s failed: %s (%s)" % (where, STATUS.get(code, code), msg))
        self.code = code


def check(code, where):
    if code != DG_OK:
        raise DGError(code, where)
    return code
