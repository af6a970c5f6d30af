"""ctypes declarations of the C ABI in include/ifeast.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as ct
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libifeast.so")

IFEAST_OK = 0
IFEAST_ERR_INVALID_ARG = 1
IFEAST_ERR_OOM = 2
IFEAST_ERR_CUDA = 3
IFEAST_ERR_NOT_CONVERGED = 4
IFEAST_ERR_M0_TOO_SMALL = 5
IFEAST_STATUS_NO_EIGENVALUES = 6
IFEAST_ERR_BREAKDOWN = 7
IFEAST_ERR_TIMEOUT = 8
IFEAST_ERR_STATE = 9
IFEAST_ERR_UNSUPPORTED = 10

GL_HALF, TRAP_HALF, TRAP_FULL, USER = 0, 1, 2, 3
INNER_GMRES, INNER_MINRES = 0, 1
FP64, FP32, FP16, BF16 = 0, 1, 2, 3
INNERS = {"gmres": INNER_GMRES, "minres": INNER_MINRES}
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp16": FP16, "bf16": BF16}

RULES = {"gl_half": GL_HALF, "trap_half": TRAP_HALF, "trap_full": TRAP_FULL, "user": USER}


class Csr(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("nnz", ct.c_int64), ("rowptr", ct.c_void_p),
                ("colidx", ct.c_void_p), ("val", ct.c_void_p)]


class Contour(ct.Structure):
    _fields_ = [("rule", ct.c_int), ("nc", ct.c_int), ("emin", ct.c_double), ("emax", ct.c_double),
                ("user_zw", ct.c_void_p)]


class Opts(ct.Structure):
    _fields_ = [("inner_solver", ct.c_int), ("inner_max_iters", ct.c_int), ("alpha", ct.c_double),
                ("max_outer", ct.c_int), ("tol", ct.c_double), ("precision", ct.c_int),
                ("verbose", ct.c_int), ("nonsymmetric", ct.c_int), ("minres_two_pass", ct.c_int),
                ("correction_rf", ct.c_double), ("time_limit_ms", ct.c_double),
                ("node_chunk", ct.c_int), ("plain_loads", ct.c_int),
                ("nonsym_correction", ct.c_int)]


class Stats(ct.Structure):
    _fields_ = [("outer_iters", ct.c_int), ("found", ct.c_int), ("RF", ct.c_double),
                ("total_matvecs", ct.c_int64), ("seq_matvecs", ct.c_int64),
                ("max_inner", ct.c_int), ("shifted_cholesky", ct.c_int), ("solve_ms", ct.c_double)]


class ServerOpts(ct.Structure):
    _fields_ = [("mem_budget_bytes", ct.c_size_t), ("max_active", ct.c_int), ("device", ct.c_int)]


class RequestInfo(ct.Structure):
    _fields_ = [("status", ct.c_int), ("found", ct.c_int), ("outer_iters", ct.c_int),
                ("RF", ct.c_double), ("submit_to_start_ms", ct.c_double),
                ("submit_to_done_ms", ct.c_double), ("workspace_bytes", ct.c_size_t)]


# name -> (restype, argtypes)
SIGNATURES = {
    "ifeast_default_opts": (None, [ct.POINTER(Opts)]),
    "ifeast_contour_nodes": (ct.c_int, [ct.POINTER(Contour), ct.c_void_p]),
    "ifeast_workspace_bytes": (ct.c_int, [ct.c_int64, ct.c_int64, ct.c_int, ct.POINTER(Contour),
                                          ct.POINTER(Opts), ct.POINTER(ct.c_size_t)]),
    "ifeast_workspace_bytes_generalized": (ct.c_int, [ct.c_int64, ct.c_int64, ct.c_int64, ct.c_int,
                                                      ct.POINTER(Contour), ct.POINTER(Opts),
                                                      ct.POINTER(ct.c_size_t)]),
    "ifeast_create": (ct.c_int, [ct.POINTER(Csr), ct.c_void_p, ct.POINTER(Contour), ct.c_int,
                                 ct.POINTER(Opts), ct.c_void_p, ct.c_size_t, ct.c_void_p,
                                 ct.POINTER(ct.c_void_p)]),
    "ifeast_solve": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_uint64, ct.c_void_p]),
    "ifeast_initial_subspace": (ct.c_int, [ct.c_int64, ct.c_int, ct.c_uint64, ct.c_void_p,
                                           ct.c_void_p]),
    "ifeast_eigenpairs": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_int), ct.c_void_p,
                                     ct.c_void_p, ct.c_void_p, ct.c_int]),
    "ifeast_ritz_all": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "ifeast_eigenpairs_complex": (ct.c_int, [ct.c_void_p, ct.c_int, ct.POINTER(ct.c_int),
                                             ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "ifeast_rayleigh_ritz_nonsym": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                               ct.c_void_p, ct.c_void_p]),
    "ifeast_stats": (ct.c_int, [ct.c_void_p, ct.POINTER(Stats)]),
    "ifeast_strerror": (ct.c_char_p, [ct.c_int]),
    "ifeast_destroy": (None, [ct.c_void_p]),
    "ifeast_apply_filter": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_double,
                                       ct.c_void_p]),
    "ifeast_apply_filter_residual": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                                ct.c_void_p, ct.c_double, ct.c_void_p]),
    "ifeast_rayleigh_ritz": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                        ct.c_void_p]),
    "ifeast_spmm_shift": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_int,
                                     ct.c_void_p]),
    "ifeast_set_profiling": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "ifeast_kernel_times": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "ifeast_kernel_launches": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int]),
    "ifeast_kernel_name": (ct.c_char_p, [ct.c_int]),
    "ifeast_server_create": (ct.c_int, [ct.POINTER(ServerOpts), ct.POINTER(ct.c_void_p)]),
    "ifeast_server_submit": (ct.c_int, [ct.c_void_p, ct.POINTER(Csr), ct.POINTER(Contour), ct.c_int,
                                        ct.POINTER(Opts), ct.c_void_p, ct.POINTER(ct.c_int64)]),
    "ifeast_server_wait": (ct.c_int, [ct.c_void_p, ct.c_int64, ct.c_int, ct.POINTER(ct.c_int),
                                      ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                      ct.POINTER(RequestInfo)]),
    "ifeast_server_destroy": (None, [ct.c_void_p]),
    "ifeast_rayleigh_ritz_noalloc": (ct.c_int, [ct.c_int64, ct.c_int64, ct.c_void_p, ct.c_void_p,
                                                ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p,
                                                ct.c_void_p, ct.c_void_p, ct.c_void_p]),
}

_lib = None


def load(path: str | None = None):
    """Loads libifeast.so (built by paper_1706_00692_gb300.build). Raises if it
    is missing: there is no fallback implementation."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libifeast.so not found at {p}; run paper_1706_00692_gb300.build.build()")
    lib = ct.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib
