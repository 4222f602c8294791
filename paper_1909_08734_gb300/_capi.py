"""ctypes declarations of the C ABI in include/cpm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcpm_gb300.so")

# status codes
CPM_OK = 0
CPM_ERR_INVALID_ARG = 1
CPM_ERR_OOM = 2
CPM_ERR_CUDA = 3
CPM_ERR_SINGULAR = 4
CPM_ERR_NOT_CONVERGED = 5
CPM_ERR_BREAKDOWN = 6
CPM_ERR_NAN = 7
CPM_ERR_TIMEOUT = 8
CPM_ERR_BUDGET = 9
CPM_ERR_STENCIL = 10
# enums
CPM_SPHERE, CPM_TORUS, CPM_TRIMESH = 0, 1, 2
CPM_TUNE_SOLVE_CTAS_PER_SM, CPM_TUNE_SOLVE_KSEG, CPM_TUNE_SOLVE_PREFETCH, CPM_TUNE_SOLVE_STAGGER = 0, 1, 2, 3
CPM_RAS, CPM_ORAS, CPM_ORAS_R3 = 0, 1, 2
CPM_FP64, CPM_FP32, CPM_BF16 = 0, 1, 2
CPM_SETUP_SIMT_LU = 0x100
(CPM_SET_OWN, CPM_SET_SIGMA, CPM_SET_LAST, CPM_SET_GHOST, CPM_SET_BC_A, CPM_SET_BC_G,
 CPM_SET_BC_GEN, CPM_SET_BC_NEARX) = range(8)


class cpm_surface(C.Structure):
    _fields_ = [("kind", C.c_int), ("R", C.c_double), ("r", C.c_double),
                ("verts", C.POINTER(C.c_double)), ("n_verts", C.c_int64),
                ("tris", C.POINTER(C.c_int32)), ("n_tris", C.c_int64)]


class cpm_band_info(C.Structure):
    _fields_ = [("n_active", C.c_int64), ("n_ghost", C.c_int64), ("p", C.c_int), ("h", C.c_double),
                ("lambda_", C.c_double), ("ijk", C.POINTER(C.c_int32)), ("cp", C.POINTER(C.c_double)),
                ("nbr", C.POINTER(C.c_int32)), ("base", C.POINTER(C.c_int32)),
                ("pencil", C.POINTER(C.c_int32)), ("weights", C.POINTER(C.c_double)),
                ("tri", C.POINTER(C.c_int32))]


class oras_info(C.Structure):
    _fields_ = [("n_sub", C.c_int), ("n_active", C.c_int64), ("n_nodes", C.c_int64),
                ("precision", C.c_int), ("transmission", C.c_int), ("max_n", C.c_int64),
                ("sum_n", C.c_int64), ("sum_n2", C.c_int64), ("sum_sigma", C.c_int64),
                ("factor_bytes", C.c_int64), ("device_bytes", C.c_int64),
                ("setup_ms_assemble", C.c_double), ("setup_ms_factor", C.c_double),
                ("kernel_launches", C.c_int64), ("solve_ctas_per_sm", C.c_int),
                ("solve_kseg", C.c_int), ("solve_prefetch", C.c_int), ("solve_stagger", C.c_int),
                ("peak_device_bytes", C.c_int64), ("tile_rows", C.c_int64),
                ("solve_offdiag_tiles", C.c_int64)]


class oras_plan_info(C.Structure):
    _fields_ = [("setup_peak_bytes", C.c_int64), ("resident_bytes", C.c_int64),
                ("factor_bytes", C.c_int64), ("vector_bytes", C.c_int64), ("sum_n2", C.c_int64),
                ("max_tiles", C.c_int)]


class cpm_gmres_opts(C.Structure):
    _fields_ = [("restart", C.c_int), ("tol", C.c_double), ("max_it", C.c_int),
                ("use_graph", C.c_int), ("zero_guess", C.c_int)]


class cpm_gmres_result(C.Structure):
    _fields_ = [("iterations", C.c_int), ("relres", C.c_double), ("status", C.c_int)]


_P = C.c_void_p
_SIGS = {
    "cpm_build_band": (C.c_int, [C.POINTER(cpm_surface), C.c_double, C.c_int, C.c_double, C.POINTER(_P)]),
    "cpm_build_band_algorithmic": (C.c_int, [C.POINTER(cpm_surface), C.c_double, C.c_int, C.POINTER(_P)]),
    "cpm_build_band_device": (C.c_int, [C.POINTER(cpm_surface), C.c_double, C.c_int, C.c_double, _P,
                                        C.POINTER(_P)]),
    "cpm_band_info_get": (C.c_int, [_P, C.POINTER(cpm_band_info)]),
    "cpm_band_destroy": (None, [_P]),
    "cpm_partition": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64), C.c_int, C.c_int, C.POINTER(_P)]),
    "cpm_partition_graph": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64), C.c_int, C.c_int, C.POINTER(_P)]),
    "cpm_partition_labels": (C.c_int, [_P, C.POINTER(C.POINTER(C.c_int32))]),
    "cpm_partition_set": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.POINTER(C.c_int32)),
                                    C.POINTER(C.c_int64)]),
    "cpm_partition_cross_points": (C.c_int, [_P, C.POINTER(C.POINTER(C.c_int32)), C.POINTER(C.c_int64)]),
    "cpm_partition_destroy": (None, [_P]),
    "cpm_partition_from_labels": (C.c_int, [_P, C.c_int, _P, C.c_int, C.POINTER(_P)]),
    "cpm_partition_save": (C.c_int, [_P, C.c_char_p]),
    "cpm_partition_load": (C.c_int, [_P, C.c_char_p, C.POINTER(_P)]),
    "cpm_local_coo": (C.c_int, [_P, _P, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int,
                                C.POINTER(C.c_int64), C.POINTER(C.c_int64), _P, _P, _P]),
    "cpm_local_order": (C.c_int, [_P, _P, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int,
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int), _P, _P, _P, _P]),
    "oras_setup": (C.c_int, [_P, _P, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int, _P,
                             C.POINTER(_P)]),
    "oras_info_get": (C.c_int, [_P, C.POINTER(oras_info)]),
    "oras_plan": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(oras_plan_info)]),
    "oras_local_sizes": (C.c_int, [_P, _P]),
    "cpm_op_apply": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "cpm_op_apply_noalloc": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int64, C.c_int, C.c_double,
                                       C.c_double, _P, _P, _P]),
    "oras_apply": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "oras_check_status": (C.c_int, [_P, _P]),
    "oras_tune": (C.c_int, [_P, C.c_int, C.c_int]),
    "oras_autotune": (C.c_int, [_P, _P]),
    "cpm_gmres_solve": (C.c_int, [_P, _P, _P, C.c_int, C.POINTER(cpm_gmres_opts),
                                  C.POINTER(cpm_gmres_result), _P]),
    "oras_stationary_solve": (C.c_int, [_P, _P, _P, C.c_int, C.c_double, C.c_int,
                                        C.POINTER(cpm_gmres_result), _P]),
    "cpm_vec_axpby": (C.c_int, [C.c_int64, C.c_double, _P, C.c_double, _P, _P]),
    "cpm_selftest_bounded_wait": (C.c_int, [_P, C.c_double, _P]),
    "cpm_selftest_zero_operator": (C.c_int, [_P]),
    "oras_setup_selftest_singular": (C.c_int, [_P, _P, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int,
                                               C.c_int, _P]),
    "cpm_probe_fp64": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]),
    "oras_destroy": (None, [_P]),
    "cpm_status_string": (C.c_char_p, [C.c_int]),
    "cpm_last_error": (C.c_char_p, []),
}

_lib = None


def load() -> C.CDLL:
    """Load the in-tree CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
