"""ctypes view of the C ABI declared in include/mvgd.h (argument marshalling only).

Loads the in-tree ``_build/libmvgd.so``.  There is no fallback: if the library
is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

_P = C.c_void_p
LIB_PATH = Path(__file__).resolve().parent / "_build" / "libmvgd.so"

# status codes (mvgd_status)
OK, EINVAL, EWORKSPACE, EDEGENERATE, ENOCONV, EBREAKDOWN, ENONFINITE, ECANCELLED, ETIMEOUT, ECUDA = range(10)
DELTA_QUARTER_RANGE, DELTA_MEAN_NN = 0, 1
ROW_MVGD, ROW_LS = 0, 1  # mvgd_row_variant
FP64, FP32_REFINE = 0, 1
ELL_COL, ELL_VAL, ELL_VAL_LO = 0, 1, 2
SPMV_F64, SPMV_F32, SPMV_F64_HILO = 0, 1, 2

EXPORTS = (
    "mvgd_status_string", "mvgd_version", "mvgd_knn_workspace_bytes", "mvgd_knn", "mvgd_ell_bytes",
    "mvgd_assemble_workspace_bytes", "mvgd_assemble", "mvgd_spmv", "mvgd_solve_workspace_bytes", "mvgd_solve",
    "mvgd_request_workspace_bytes", "mvgd_request_init", "mvgd_iterate_workspace_bytes", "mvgd_iterate",
    "mvgd_request_finish", "mvgd_assemble_batch_workspace_bytes", "mvgd_assemble_batch", "mvgd_request_poll",
    "mvgd_knn_noalloc", "mvgd_amg_workspace_bytes", "mvgd_amg_setup", "mvgd_amg_describe",
    "mvgd_amg_apply_workspace_bytes", "mvgd_amg_apply", "mvgd_trace_enable", "mvgd_trace_read",
    "mvgd_row_signs", "mvgd_dirichlet_rows", "mvgd_block_gram_workspace_bytes", "mvgd_block_gram",
    "mvgd_block_combine", "mvgd_block_zero_rows", "mvgd_gs_power_workspace_bytes", "mvgd_gs_power",
    "mvgd_neumann_ghosts_workspace_bytes", "mvgd_neumann_ghosts", "mvgd_neumann_fold_workspace_bytes",
    "mvgd_neumann_fold", "mvgd_neumann_rhs", "mvgd_set_wait_limit", "mvgd_test_withhold_arrival",
    "mvgd_block_chol_inverse", "mvgd_ritz_values", "mvgd_set_launch_tuning",
)
PRECOND_NONE, PRECOND_ROWSCALE, PRECOND_AMG = 0, 1, 2
AMG_AGG, AMG_COARSEST, AMG_MAX_WIDTH = 8, 512, 64  # MVGD_AMG_* in include/mvgd.h


class DeltaRule(C.Structure):
    _fields_ = [("kind", C.c_int32), ("m", C.c_int32), ("scale", C.c_double), ("variant", C.c_int32),
                ("arith", C.c_int32)]


class Ell(C.Structure):
    _fields_ = [("n", C.c_int64), ("k", C.c_int32), ("prec", C.c_int32), ("order", _P), ("col", _P),
                ("val", _P), ("val_lo", _P)]


class SolveOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("maxit", C.c_int32), ("inner_maxit", C.c_int32),
                ("inner_rtol", C.c_double), ("max_outer", C.c_int32), ("precond", C.c_int32), ("amg", _P)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("outer", C.c_int32), ("relres", C.c_double), ("status", C.c_int32),
                ("reserved", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("workspace", _P), ("n", C.c_int64), ("nrhs", C.c_int32), ("k", C.c_int32)]


def requests(items) -> C.Array:
    """ctypes array of mvgd_request from (workspace tensor or pointer, n, nrhs, k) tuples."""
    arr = (Request * len(items))()
    for i, (ws, n, q, k) in enumerate(items):
        ptr = ws if isinstance(ws, int) else ws.data_ptr()
        arr[i] = Request(C.c_void_p(ptr), int(n), int(q), int(k))
    return arr


class AmgInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("levels", C.c_int32), ("stride", C.c_int32), ("status", C.c_int32),
                ("width_max", C.c_int32), ("col", _P), ("val", _P), ("val64", _P), ("cnt", _P), ("dinv", _P),
                ("cinv", _P), ("cinv64", _P)]


class AssembleItem(C.Structure):
    _fields_ = [("pts", _P), ("nbr", _P), ("L", Ell), ("h", _P), ("row_status", _P)]


class MvgdError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn}: {status_string(status)}")


_lib = None


def load(path: str | os.PathLike | None = None) -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"libmvgd.so not built ({p}); run paper_1603_04100_gb300.build.build()")
    L = C.CDLL(str(p))
    L.mvgd_status_string.argtypes = [C.c_int]; L.mvgd_status_string.restype = C.c_char_p
    L.mvgd_version.argtypes = []; L.mvgd_version.restype = C.c_int32
    L.mvgd_knn_workspace_bytes.argtypes = [C.c_int64, C.c_int32]; L.mvgd_knn_workspace_bytes.restype = C.c_size_t
    L.mvgd_knn.argtypes = [_P, C.c_int64, C.c_int32, _P, _P, C.c_double, _P, C.c_size_t, _P]
    L.mvgd_knn.restype = C.c_int
    L.mvgd_ell_bytes.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_int32]; L.mvgd_ell_bytes.restype = C.c_size_t
    L.mvgd_assemble_workspace_bytes.argtypes = [C.c_int64]; L.mvgd_assemble_workspace_bytes.restype = C.c_size_t
    L.mvgd_assemble.argtypes = [_P, C.c_int64, C.c_int32, _P, DeltaRule, C.POINTER(Ell), _P, _P, _P, _P,
                                C.c_size_t, _P]
    L.mvgd_assemble.restype = C.c_int
    L.mvgd_spmv.argtypes = [C.POINTER(Ell), C.c_int32, C.c_int32, C.c_double, C.c_double, _P, C.c_double, _P, _P]
    L.mvgd_spmv.restype = C.c_int
    L.mvgd_solve_workspace_bytes.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    L.mvgd_solve_workspace_bytes.restype = C.c_size_t
    L.mvgd_solve.argtypes = [C.POINTER(Ell), C.c_int32, C.c_double, _P, _P, C.POINTER(SolveOpts), _P, _P, _P,
                             C.c_size_t, _P]
    L.mvgd_solve.restype = C.c_int
    L.mvgd_request_workspace_bytes.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    L.mvgd_request_workspace_bytes.restype = C.c_size_t
    L.mvgd_request_init.argtypes = [_P, C.c_size_t, C.POINTER(Ell), C.c_int32, C.c_double, _P, _P,
                                    C.POINTER(SolveOpts), _P]
    L.mvgd_request_init.restype = C.c_int
    L.mvgd_iterate_workspace_bytes.argtypes = [C.c_int32, C.c_int64]
    L.mvgd_iterate_workspace_bytes.restype = C.c_size_t
    L.mvgd_iterate.argtypes = [C.POINTER(Request), C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, _P, C.c_size_t,
                               _P]
    L.mvgd_iterate.restype = C.c_int
    L.mvgd_request_finish.argtypes = [_P, C.c_int64, C.c_int32, _P, _P, _P]
    L.mvgd_request_finish.restype = C.c_int
    L.mvgd_assemble_batch_workspace_bytes.argtypes = [C.POINTER(C.c_int64), C.c_int32]
    L.mvgd_assemble_batch_workspace_bytes.restype = C.c_size_t
    L.mvgd_assemble_batch.argtypes = [C.POINTER(AssembleItem), C.c_int32, DeltaRule, _P, _P, C.c_size_t, _P]
    L.mvgd_assemble_batch.restype = C.c_int
    L.mvgd_request_poll.argtypes = [C.POINTER(C.c_void_p), C.c_int32, _P, _P]
    L.mvgd_request_poll.restype = C.c_int
    L.mvgd_knn_noalloc.argtypes = [_P, C.c_int64, C.c_int32, _P, _P, C.c_double, _P]
    L.mvgd_knn_noalloc.restype = C.c_int
    L.mvgd_amg_workspace_bytes.argtypes = [C.c_int64, C.c_int32]
    L.mvgd_amg_workspace_bytes.restype = C.c_size_t
    L.mvgd_amg_setup.argtypes = [C.POINTER(Ell), C.c_double, _P, C.c_size_t, _P]
    L.mvgd_amg_setup.restype = C.c_int
    L.mvgd_amg_describe.argtypes = [_P, C.c_int32, C.POINTER(AmgInfo)]
    L.mvgd_amg_describe.restype = C.c_int
    L.mvgd_amg_apply_workspace_bytes.argtypes = [C.c_int64, C.c_int32]
    L.mvgd_amg_apply_workspace_bytes.restype = C.c_size_t
    L.mvgd_amg_apply.argtypes = [_P, C.c_int64, C.c_int32, _P, _P, _P, C.c_size_t, _P]
    L.mvgd_amg_apply.restype = C.c_int
    L.mvgd_trace_enable.argtypes = [C.c_int32]
    L.mvgd_trace_enable.restype = C.c_int
    L.mvgd_trace_read.argtypes = [C.POINTER(C.c_uint64), C.c_int32]
    L.mvgd_trace_read.restype = C.c_int32
    L.mvgd_row_signs.argtypes = [C.POINTER(Ell), _P, _P]
    L.mvgd_row_signs.restype = C.c_int
    L.mvgd_dirichlet_rows.argtypes = [C.POINTER(Ell), _P, _P, _P]
    L.mvgd_dirichlet_rows.restype = C.c_int
    L.mvgd_block_gram_workspace_bytes.argtypes = [C.c_int32, C.c_int32]
    L.mvgd_block_gram_workspace_bytes.restype = C.c_size_t
    L.mvgd_block_gram.argtypes = [_P, C.c_int32, _P, C.c_int32, C.c_int64, C.c_int32, _P, _P, C.c_size_t, _P]
    L.mvgd_block_gram.restype = C.c_int
    L.mvgd_block_combine.argtypes = [_P, C.c_int32, _P, C.c_int32, C.c_int64, C.c_int32, _P, _P]
    L.mvgd_block_combine.restype = C.c_int
    L.mvgd_block_zero_rows.argtypes = [_P, C.c_int32, C.c_int64, C.c_int32, _P, _P]
    L.mvgd_block_zero_rows.restype = C.c_int
    L.mvgd_gs_power_workspace_bytes.argtypes = [C.c_int64, C.c_int32]
    L.mvgd_gs_power_workspace_bytes.restype = C.c_size_t
    L.mvgd_gs_power.argtypes = [C.POINTER(Ell), C.c_double, _P, C.c_int32, _P, _P, _P, _P, C.c_size_t, _P]
    L.mvgd_gs_power.restype = C.c_int
    L.mvgd_neumann_ghosts_workspace_bytes.argtypes = [C.c_int64]
    L.mvgd_neumann_ghosts_workspace_bytes.restype = C.c_size_t
    L.mvgd_neumann_ghosts.argtypes = [_P, C.c_int64, C.c_int32, _P, _P, C.c_int32, _P, _P, _P, _P, _P, _P, _P,
                                      C.c_size_t, _P]
    L.mvgd_neumann_ghosts.restype = C.c_int
    L.mvgd_neumann_fold_workspace_bytes.argtypes = [C.c_int64]
    L.mvgd_neumann_fold_workspace_bytes.restype = C.c_size_t
    L.mvgd_neumann_fold.argtypes = [C.POINTER(Ell), _P, C.POINTER(Ell), _P, C.c_size_t, _P]
    L.mvgd_neumann_fold.restype = C.c_int
    L.mvgd_neumann_rhs.argtypes = [C.POINTER(Ell), C.c_int64, _P, _P, _P, _P, _P]
    L.mvgd_neumann_rhs.restype = C.c_int
    L.mvgd_block_chol_inverse.argtypes = [_P, C.c_int32, _P]
    L.mvgd_block_chol_inverse.restype = C.c_int
    L.mvgd_ritz_values.argtypes = [_P, C.c_int32, _P, _P]
    L.mvgd_ritz_values.restype = C.c_int
    L.mvgd_set_launch_tuning.argtypes = [C.c_int32, C.c_int32, C.c_int32]
    L.mvgd_set_launch_tuning.restype = C.c_int
    L.mvgd_set_wait_limit.argtypes = [C.c_int64]
    L.mvgd_set_wait_limit.restype = C.c_int
    L.mvgd_test_withhold_arrival.argtypes = [C.c_int32]
    L.mvgd_test_withhold_arrival.restype = C.c_int
    _lib = L
    return L


def status_string(s: int) -> str:
    return load().mvgd_status_string(int(s)).decode()


def check(fn: str, status: int) -> int:
    if status != OK:
        raise MvgdError(fn, status)
    return status
