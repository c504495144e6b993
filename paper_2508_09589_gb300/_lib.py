"""ctypes declarations of the C ABI in include/st.h (argument marshalling only).

The native library libst.so is built in-tree by paper_2508_09589_gb300.build.
Loading fails loudly when it is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libst.so")

ST_OK = 0
STATUS = {0: "ST_OK", -1: "ST_ERR_ARG", -2: "ST_ERR_OOM", -3: "ST_ERR_NOT_CONVERGED", -4: "ST_ERR_NUMERIC",
          -5: "ST_ERR_TIMEOUT", -6: "ST_ERR_CUDA", -7: "ST_ERR_BUSY", -8: "ST_ERR_STATE", -9: "ST_ERR_NOT_FOUND",
          -10: "ST_ERR_CANCELLED"}
BC = {"patch_left": 0, "patch_bottom": 1, "all_walls": 2, "none": 3}
LAYOUT = {"extruded": 0, "spacetime": 1}
SMOOTHER = {"gmres": 0, "jacobi": 1}
MEM_HOST, MEM_DEVICE = 0, 1
PREC = {"mixed": 0, "fp64": 1}
SRC = {"uniform": 0, "sin_t": 1, "gaussian": 2}
OBJ = {"compliance": 0, "pnorm": 1}
WHICH = {"T": 0, "lambda": 1, "rhs": 2, "adj_rhs": 3}
COARSEN = {"semi": 0, "full": 1}
COARSE = {"auto": 0, "dense": 1, "gmres": 2}


class Material(C.Structure):
    _fields_ = [("C_ins", C.c_double), ("C_con", C.c_double), ("k_ins", C.c_double), ("k_con", C.c_double),
                ("p_c", C.c_int), ("p_k", C.c_int)]


class MeshDesc(C.Structure):
    _fields_ = [("ndim_space", C.c_int), ("n", C.c_int * 3), ("n_t", C.c_int), ("ext", C.c_double * 3),
                ("tau", C.c_double), ("mat", Material), ("bc", C.c_int), ("bc_width", C.c_double),
                ("lambda_crit", C.c_double), ("coarse_dof_cap", C.c_longlong), ("max_levels", C.c_int),
                ("coarsening", C.c_int), ("device", C.c_int), ("coarse_solver", C.c_int),
                ("coarse_max_it", C.c_int), ("coarse_rtol", C.c_double), ("march_blocks", C.c_int),
                ("smoother", C.c_int), ("smoother_omega", C.c_double)]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int), ("q0", C.c_double), ("a", C.c_double), ("b", C.c_double), ("f", C.c_double)]


class Options(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_it", C.c_int), ("restart", C.c_int), ("precision", C.c_int),
                ("warm_start", C.c_int), ("smooth_steps", C.c_int), ("use_graphs", C.c_int)]


class Objective(C.Structure):
    _fields_ = [("kind", C.c_int), ("P", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("outer_its", C.c_int), ("restarts", C.c_int), ("converged", C.c_int), ("rel_res", C.c_double),
                ("rel_res_est", C.c_double), ("seconds", C.c_double), ("norm_f", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MeshInfo(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("n_nodes", C.c_longlong), ("n_elem", C.c_longlong),
                ("device_bytes", C.c_longlong)]


class LevelInfo(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("n_t", C.c_int), ("n_nodes", C.c_longlong), ("to_next", C.c_int),
                ("h", C.c_double * 3), ("dt", C.c_double)]


class Request(C.Structure):
    _fields_ = [("mesh", MeshDesc), ("gamma", C.POINTER(C.c_double)), ("layout", C.c_int), ("count", C.c_size_t),
                ("source", Source), ("objective", Objective), ("options", Options), ("want_gradient", C.c_int)]


class MmaParams(C.Structure):
    _fields_ = [("s0", C.c_double), ("incr", C.c_double), ("decr", C.c_double), ("move", C.c_double),
                ("raa", C.c_double), ("lam_max", C.c_double)]


class TopOptParams(C.Structure):
    _fields_ = [("vf", C.c_double), ("r_x", C.c_double), ("r_t", C.c_double), ("beta", C.c_double),
                ("eta", C.c_double), ("objective", C.c_int), ("P", C.c_int), ("obj_scale", C.c_double),
                ("filter_rtol", C.c_double), ("filter_max_it", C.c_int), ("warm_start", C.c_int),
                ("mma", MmaParams)]


class TopOptStats(C.Structure):
    _fields_ = [("iteration", C.c_int), ("phi", C.c_double), ("chi", C.c_double), ("lam", C.c_double),
                ("change", C.c_double), ("forward", Stats), ("adjoint", Stats), ("filter_its", C.c_int),
                ("seconds", C.c_double), ("filter_seconds", C.c_double), ("design_seconds", C.c_double),
                ("mma_seconds", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("forward", "adjoint")}
        d["forward"] = self.forward.as_dict()
        d["adjoint"] = self.adjoint.as_dict()
        return d


class Bdf1Stats(C.Structure):
    _fields_ = [("steps", C.c_int), ("outer_its", C.c_longlong), ("max_outer_its", C.c_int),
                ("max_rel_res", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TO_FIELD = {"gamma": 0, "gamma_tilde": 1, "gamma_bar": 2, "dphi": 3, "dchi": 4}


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("phi", C.c_double), ("forward", Stats), ("adjoint", Stats),
                ("latency_s", C.c_double), ("queue_s", C.c_double), ("footprint", C.c_longlong),
                ("batch", C.c_int)]


class ServerDesc(C.Structure):
    _fields_ = [("hbm_budget", C.c_longlong), ("max_inflight", C.c_int), ("device", C.c_int),
                ("max_batch", C.c_int), ("batch_nodes", C.c_longlong)]


_lib = None

# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "st_version": (C.c_char_p, []),
    "st_last_error": (C.c_char_p, []),
    "st_mesh_desc_default": (None, [C.POINTER(MeshDesc)]),
    "st_options_default": (None, [C.POINTER(Options)]),
    "st_plan_hierarchy": (C.c_int, [C.POINTER(MeshDesc), C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "st_create_mesh": (C.c_int, [C.POINTER(MeshDesc), C.POINTER(C.c_void_p)]),
    "st_destroy_mesh": (C.c_int, [C.c_void_p]),
    "st_mesh_info_get": (C.c_int, [C.c_void_p, C.POINTER(MeshInfo)]),
    "st_level_info_get": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(LevelInfo)]),
    "st_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "st_synchronize": (C.c_int, [C.c_void_p]),
    "st_set_design": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_size_t, C.c_int]),
    "st_solve_forward": (C.c_int, [C.c_void_p, C.POINTER(Source), C.POINTER(Options), C.POINTER(Stats)]),
    "st_solve_adjoint": (C.c_int, [C.c_void_p, C.POINTER(Objective), C.POINTER(Options), C.POINTER(C.c_double),
                                   C.POINTER(Stats)]),
    "st_filter": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_double, C.c_double,
                            C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "st_heaviside": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_double,
                               C.c_double]),
    "st_solve_forward_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(Options), C.c_void_p,
                                         C.c_void_p]),
    "st_solve_adjoint_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(Options), C.c_void_p,
                                         C.c_void_p, C.c_void_p]),
    "st_sensitivities": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
    "st_get_state": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_int]),
    "st_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
    "st_op_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "st_op_diag": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "st_restrict": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "st_prolong": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "st_smooth": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "st_vcycle": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "st_level_elements": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    "st_coarse_inverse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "st_apply_timer": (C.c_int, [C.c_void_p, C.c_int]),
    "st_apply_timer_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "st_server_create": (C.c_int, [C.POINTER(ServerDesc), C.POINTER(C.c_void_p)]),
    "st_server_destroy": (C.c_int, [C.c_void_p]),
    "st_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "st_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "st_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(Result), C.c_void_p, C.c_size_t, C.POINTER(C.c_int)]),
    "st_footprint_bytes": (C.c_longlong, [C.POINTER(MeshDesc), C.c_int, C.c_int]),
    "st_kernel_launches": (C.c_longlong, []),
    "st_fp64_fma_rate": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "st_residual_norm_noalloc": (C.c_int, [C.POINTER(MeshDesc), C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p]),
    "st_mma_params_default": (None, [C.POINTER(MmaParams)]),
    "st_mma_create": (C.c_int, [C.c_longlong, C.POINTER(MmaParams), C.POINTER(C.c_void_p)]),
    "st_mma_destroy": (C.c_int, [C.c_void_p]),
    "st_mma_update": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_double,
                                C.c_double, C.c_void_p, C.POINTER(C.c_double)]),
    "st_topopt_params_default": (None, [C.POINTER(TopOptParams)]),
    "st_topopt_create": (C.c_int, [C.c_void_p, C.POINTER(TopOptParams), C.c_void_p, C.c_int, C.c_size_t, C.c_int,
                                   C.POINTER(C.c_void_p)]),
    "st_topopt_destroy": (C.c_int, [C.c_void_p]),
    "st_topopt_step": (C.c_int, [C.c_void_p, C.POINTER(Source), C.POINTER(Options), C.POINTER(TopOptStats)]),
    "st_topopt_get": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_int]),
    "st_bdf1_create": (C.c_int, [C.POINTER(MeshDesc), C.POINTER(C.c_void_p)]),
    "st_bdf1_destroy": (C.c_int, [C.c_void_p]),
    "st_bdf1_set_design": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_size_t, C.c_int]),
    "st_bdf1_forward": (C.c_int, [C.c_void_p, C.POINTER(Source), C.POINTER(Options), C.c_void_p, C.c_size_t,
                                  C.c_int, C.POINTER(Bdf1Stats)]),
    "st_bdf1_adjoint": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Options), C.POINTER(C.c_double), C.c_void_p,
                                  C.c_size_t, C.c_int, C.POINTER(Bdf1Stats)]),
    "st_bdf1_sensitivities": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]),
}


def lib():
    """Load libst.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"native library missing: {LIB_PATH} (run paper_2508_09589_gb300.build.build())")
    L = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class STError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().st_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")


def check(code: int, where: str, allow=()):
    if code != ST_OK and code not in allow:
        raise STError(code, where)
    return code
