"""ctypes declarations of the C ABI in include/ntvs.h and include/ntvs_fbp.h (argument
marshalling only).

Every function of the header is bound here under its C name.  The library is the
in-tree ``libntvs.so`` built by ``paper_1803_01112_gb300._build``; importing this module
fails loudly when it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libntvs.so")

NTVS_OK = 0
NTVS_ERR_ARG = -1
NTVS_ERR_CSR = -2
NTVS_ERR_OOM = -3
NTVS_ERR_CUDA = -4
NTVS_ERR_TIMEOUT = -5
NTVS_ERR_STATE = -6

NTVS_F64, NTVS_F32, NTVS_F16, NTVS_BF16 = 0, 1, 2, 3
NTVS_I32 = 4
NTVS_MEM_HOST, NTVS_MEM_DEVICE = 0, 1
NTVS_CSR32, NTVS_DELTA16 = 0, 1
NTVS_SCHED_AUTO, NTVS_SCHED_PLAIN, NTVS_SCHED_WINDOW, NTVS_SCHED_PIPELINE, NTVS_SCHED_ONTHEFLY = 0, 1, 2, 3, 4
NTVS_STEP_NTVS, NTVS_STEP_OTVS, NTVS_STEP_DECOUPLED = 0, 1, 2
NTVS_HOOK_STARVE_PIPE, NTVS_HOOK_STARVE_CHECK, NTVS_HOOK_STARVE_BATCH = 1, 2, 4

ERROR_NAMES = {NTVS_ERR_ARG: "NTVS_ERR_ARG", NTVS_ERR_CSR: "NTVS_ERR_CSR", NTVS_ERR_OOM: "NTVS_ERR_OOM",
               NTVS_ERR_CUDA: "NTVS_ERR_CUDA", NTVS_ERR_TIMEOUT: "NTVS_ERR_TIMEOUT",
               NTVS_ERR_STATE: "NTVS_ERR_STATE"}


class ntvs_system(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_blocks", ctypes.c_int32), ("n_rows", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("block_ptr", ctypes.c_void_p),
                ("val_dtype", ctypes.c_int32), ("mem_kind", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("schedule", ctypes.c_int32)]


class ntvs_histories(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("n_blocks", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("n_rows", ctypes.c_int64), ("hist", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("block_ptr", ctypes.c_void_p), ("n_seg", ctypes.c_int32), ("mem_kind", ctypes.c_int32),
                ("min_len", ctypes.c_double)]


class ntvs_paths(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("n_blocks", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("n_rows", ctypes.c_int64), ("paths", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("block_ptr", ctypes.c_void_p), ("n_seg", ctypes.c_int32), ("mem_kind", ctypes.c_int32),
                ("min_len", ctypes.c_double)]


class ntvs_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("alpha", ctypes.c_double), ("beta0", ctypes.c_double),
                ("eps_tv", ctypes.c_double), ("N", ctypes.c_int32), ("tv_check", ctypes.c_int32),
                ("max_retries", ctypes.c_int32), ("step_rule", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("gamma", ctypes.c_double)]


class ntvs_stats(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("ell_prev", ctypes.c_int64), ("n_steps", ctypes.c_int64),
                ("n_accepted", ctypes.c_int64), ("n_tries", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_rows", ctypes.c_int64), ("n_blocks", ctypes.c_int32), ("compute_dtype", ctypes.c_int32),
                ("last_tv", ctypes.c_double), ("n_launches", ctypes.c_int64),
                ("drop_schedule", ctypes.c_int32), ("lanes_per_row", ctypes.c_int32),
                ("n_escaped", ctypes.c_int64), ("voxel_tile_x", ctypes.c_int32),
                ("voxel_tile_y", ctypes.c_int32)]


class ntvs_profile(ctypes.Structure):
    _fields_ = [("drop_block_ms", ctypes.c_double), ("drop_block_launches", ctypes.c_int64),
                ("drop_apply_ms", ctypes.c_double), ("drop_apply_launches", ctypes.c_int64),
                ("tv_ms", ctypes.c_double), ("tv_launches", ctypes.c_int64)]


class ntvs_batch_stats(ctypes.Structure):
    _fields_ = [("members", ctypes.c_int32), ("lanes_per_row", ctypes.c_int32), ("cycles", ctypes.c_int64),
                ("n_launches", ctypes.c_int64), ("kernels_per_cycle", ctypes.c_int64), ("total_rows", ctypes.c_int64),
                ("total_nnz", ctypes.c_int64), ("total_voxels", ctypes.c_int64), ("rows_per_item", ctypes.c_int32),
                ("window_floats", ctypes.c_int32), ("ctas", ctypes.c_int32), ("lanes_per_row_min", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("lanes_per_row_all", ctypes.c_int32)]


vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
P = ctypes.POINTER

# int (*ntvs_allreduce_fn)(void* buf, int64_t n, int dtype, void* cuda_stream, void* user)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, vp, i64, ctypes.c_int, vp, vp)

class ntvs_fbp_geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_theta", ctypes.c_int32), ("n_t", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("theta0", ctypes.c_double)]


# name -> (restype, argtypes); the list is the whole of both headers
SIGNATURES = {
    "ntvs_version": (ctypes.c_char_p, []),
    "ntvs_last_error": (ctypes.c_char_p, []),
    "ntvs_create": (ctypes.c_int, [P(vp), ctypes.c_int, vp]),
    "ntvs_destroy": (ctypes.c_int, [vp]),
    "ntvs_load_system": (ctypes.c_int, [vp, P(ntvs_system)]),
    "ntvs_set_params": (ctypes.c_int, [vp, P(ntvs_params)]),
    "ntvs_load_paths": (ctypes.c_int, [vp, P(ntvs_paths)]),
    "ntvs_load_histories": (ctypes.c_int, [vp, P(ntvs_histories)]),
    "ntvs_set_image": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int]),
    "ntvs_get_image": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int]),
    "ntvs_run": (ctypes.c_int, [vp, ctypes.c_int]),
    "ntvs_sync": (ctypes.c_int, [vp]),
    "ntvs_get_tv": (ctypes.c_int, [vp, P(d)]),
    "ntvs_get_stats": (ctypes.c_int, [vp, P(ntvs_stats)]),
    "ntvs_get_block_resid": (ctypes.c_int, [vp, vp, ctypes.c_int]),
    "ntvs_get_trace": (ctypes.c_int, [vp, vp, vp, vp, i64, P(i64)]),
    "ntvs_get_state": (ctypes.c_int, [vp, P(i64), P(i64)]),
    "ntvs_set_state": (ctypes.c_int, [vp, i64, i64]),
    "ntvs_set_ell_override": (ctypes.c_int, [vp, vp, i64]),
    "ntvs_set_profiling": (ctypes.c_int, [vp, ctypes.c_int]),
    "ntvs_set_voxel_tile": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
    "ntvs_set_compute_dtype": (ctypes.c_int, [vp, ctypes.c_int]),
    "ntvs_set_fault_hook": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.c_int]),
    "ntvs_get_profile": (ctypes.c_int, [vp, P(ntvs_profile)]),
    "ntvs_tv_gradient": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, P(d)]),
    "ntvs_perturb": (ctypes.c_int, [vp, d]),
    "ntvs_perturb_checked": (ctypes.c_int, [vp, d, P(ctypes.c_int), P(d), P(d)]),
    "ntvs_drop_block": (ctypes.c_int, [vp, ctypes.c_int]),
    "ntvs_drop_sweep": (ctypes.c_int, [vp]),
    "ntvs_forward_project": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int]),
    "ntvs_drop_block_partial": (ctypes.c_int, [vp, ctypes.c_int, i64, i64, vp, ctypes.c_int, ctypes.c_int, P(d)]),
    "ntvs_apply_delta": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int]),
    "ntvs_get_hit_counts": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
    "ntvs_set_hit_counts": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
    "ntvs_set_allreduce": (ctypes.c_int, [vp, ALLREDUCE_FN, vp]),
    "ntvs_batch_create": (ctypes.c_int, [P(vp), ctypes.c_int, vp]),
    "ntvs_batch_destroy": (ctypes.c_int, [vp]),
    "ntvs_batch_add": (ctypes.c_int, [vp, P(ntvs_system), P(ntvs_params), vp, ctypes.c_int, ctypes.c_int,
                                      P(ctypes.c_int)]),
    "ntvs_batch_add_paths": (ctypes.c_int, [vp, P(ntvs_paths), P(ntvs_params), vp, ctypes.c_int, ctypes.c_int,
                                            P(ctypes.c_int)]),
    "ntvs_batch_set_schedule": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
    "ntvs_batch_set_fault_hook": (ctypes.c_int, [vp, i64, ctypes.c_int]),
    "ntvs_batch_sync": (ctypes.c_int, [vp]),
    "ntvs_batch_get_member": (ctypes.c_int, [vp, ctypes.c_int, vp]),
    "ntvs_batch_get_rows": (ctypes.c_int, [vp, ctypes.c_int, P(i64), P(i64), vp, vp, vp]),
    "ntvs_batch_get_tuning": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, P(ctypes.c_int)]),
    "ntvs_batch_finalize": (ctypes.c_int, [vp, ctypes.c_int]),
    "ntvs_batch_run": (ctypes.c_int, [vp, ctypes.c_int]),
    "ntvs_batch_get_image": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int]),
    "ntvs_batch_get_tv": (ctypes.c_int, [vp, ctypes.c_int, P(d)]),
    "ntvs_batch_get_stats": (ctypes.c_int, [vp, P(ntvs_batch_stats)]),
    "ntvs_tv_value_static": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]),
    # include/ntvs_fbp.h: the initial iterate
    "ntvs_fbp_bin": (ctypes.c_int, [P(ntvs_fbp_geom), vp, vp, i64, vp, vp, vp]),
    "ntvs_fbp_filter": (ctypes.c_int, [P(ntvs_fbp_geom), vp, vp, vp]),
    "ntvs_fbp_backproject": (ctypes.c_int, [P(ntvs_fbp_geom), vp, vp, vp]),
    "ntvs_median_filter": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, d, vp]),
    "ntvs_hull": (ctypes.c_int, [vp, i64, d, vp]),
    "ntvs_fbp_workspace_bytes": (i64, [P(ntvs_fbp_geom)]),
    "ntvs_initial_iterate": (ctypes.c_int, [P(ntvs_fbp_geom), vp, vp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            d, vp, i64, vp, vp]),
}

_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class NtvsError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().ntvs_last_error().decode(errors="replace")
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code: int, where: str) -> None:
    if code != NTVS_OK:
        raise NtvsError(code, where)
