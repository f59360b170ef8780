"""NTVS proton-CT reconstruction on GB300 (sm_103a): Python binding of the C ABI.

Total variation superiorization with N normalized TV perturbation steps of size
beta0*alpha^ell interleaved with block-DROP feasibility-seeking sweeps, with or without
the TV reduction check (arXiv 1803.01112, Sec. III-B, Appendix C).

Every step of the computation runs in the CUDA kernels of ``libntvs.so``; this module
only marshals arguments (numpy arrays = host memory, CUDA torch tensors = device
memory).  The module-level ``ntvs_*`` functions carry the C names of include/ntvs.h;
``Reconstructor`` is a small object wrapper over them.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import _ffi
from ._ffi import (NTVS_BF16, NTVS_CSR32, NTVS_DELTA16, NTVS_F16, NTVS_F32, NTVS_F64, NTVS_MEM_DEVICE,
                   NTVS_MEM_HOST, NTVS_STEP_DECOUPLED, NTVS_STEP_NTVS, NTVS_STEP_OTVS, NtvsError, check, lib)

__all__ = ["Reconstructor", "NtvsError", "build", "lib", "NTVS_F64", "NTVS_F32", "NTVS_F16", "NTVS_BF16",
           "NTVS_CSR32", "NTVS_DELTA16", "NTVS_STEP_NTVS", "NTVS_STEP_OTVS", "NTVS_STEP_DECOUPLED"]

_NP_DT = {np.dtype(np.float64): NTVS_F64, np.dtype(np.float32): NTVS_F32, np.dtype(np.float16): NTVS_F16}


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _dtype_code(a) -> int:
    if _is_torch(a):
        import torch
        m = {torch.float64: NTVS_F64, torch.float32: NTVS_F32, torch.float16: NTVS_F16, torch.bfloat16: NTVS_BF16}
        return m[a.dtype]
    return _NP_DT[np.dtype(a.dtype)]


def _ptr_kind(a, dtype=None):
    """(pointer, mem_kind) of a contiguous numpy array (host) or CUDA torch tensor (device)."""
    if a is None:
        return None, NTVS_MEM_HOST
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and a.dtype != dtype[1]:
            raise TypeError(f"expected {dtype[1]}, got {a.dtype}")
        return a.data_ptr(), (NTVS_MEM_DEVICE if a.is_cuda else NTVS_MEM_HOST)
    if not (a.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be C-contiguous")
    if dtype is not None and np.dtype(a.dtype) != np.dtype(dtype[0]):
        raise TypeError(f"expected {np.dtype(dtype[0])}, got {a.dtype}")
    return a.ctypes.data, NTVS_MEM_HOST


# ----------------------------------------------------------------- C-named functions
def ntvs_version() -> str:
    return lib().ntvs_version().decode()


def ntvs_last_error() -> str:
    return lib().ntvs_last_error().decode()


def ntvs_create(device: int = 0, stream: Optional[int] = None) -> int:
    """stream: None -> the context owns a stream; a cudaStream_t handle otherwise.  The
    handle 0 (torch's default stream) is passed as cudaStreamLegacy, since NULL means
    "own stream" in the C ABI."""
    h = ctypes.c_void_p()
    if stream is not None and int(stream) == 0:
        stream = 1   # cudaStreamLegacy
    check(lib().ntvs_create(ctypes.byref(h), device, stream), "ntvs_create")
    return h.value


def ntvs_destroy(ctx: int) -> None:
    check(lib().ntvs_destroy(ctx), "ntvs_destroy")


def ntvs_load_system(ctx: int, nx: int, ny: int, nz: int, row_ptr, col, val, b, n_blocks: int = 1,
                     block_ptr=None, storage: int = NTVS_CSR32, schedule: int = 0) -> None:
    """Arrays are all numpy (host, copied) or all CUDA torch tensors (device, borrowed:
    they must stay alive while the context uses them)."""
    import_torch = _is_torch(row_ptr)
    rp, kind = _ptr_kind(row_ptr)
    cp, kc = _ptr_kind(col)
    vptr, kv = _ptr_kind(val)
    bptr, kb = _ptr_kind(b)
    if len({kind, kc, kv, kb}) != 1:
        raise ValueError("row_ptr, col, val and b must all be host arrays or all device tensors")
    vdt = _dtype_code(val)
    want_b = np.float64 if vdt == NTVS_F64 else np.float32
    if import_torch:
        import torch
        for a, t, nm in ((row_ptr, torch.int64, "row_ptr"), (col, torch.int32, "col"),
                         (b, torch.float64 if vdt == NTVS_F64 else torch.float32, "b")):
            if a.dtype != t:
                raise TypeError(f"{nm} must be {t}")
    else:
        for a, t, nm in ((row_ptr, np.int64, "row_ptr"), (col, np.int32, "col"), (b, want_b, "b")):
            if np.dtype(a.dtype) != np.dtype(t):
                raise TypeError(f"{nm} must be {np.dtype(t)}")
    bp = None
    if block_ptr is not None:
        bp = np.ascontiguousarray(block_ptr, dtype=np.int64)
        n_blocks = bp.size - 1
    s = _ffi.ntvs_system(nx, ny, nz, n_blocks, (row_ptr.numel() if import_torch else row_ptr.size) - 1,
                         rp, cp, vptr, bptr, None if bp is None else bp.ctypes.data, vdt, kind, storage, schedule)
    check(lib().ntvs_load_system(ctx, ctypes.byref(s)), "ntvs_load_system")


def ntvs_load_paths(ctx: int, nx: int, ny: int, nz: int, voxel, paths, b, n_blocks: int = 1, block_ptr=None,
                    n_seg: int = 16, min_len: float = 1e-4) -> None:
    """paths: float32 [M, 10] records, b: float32 [M]; numpy (host) or CUDA tensors (device)."""
    pp, kind = _ptr_kind(paths)
    bp_, kb = _ptr_kind(b)
    if kind != kb:
        raise ValueError("paths and b must both be host arrays or both device tensors")
    nrows = (paths.shape[0])
    bp = None
    if block_ptr is not None:
        bp = np.ascontiguousarray(block_ptr, dtype=np.int64)
        n_blocks = bp.size - 1
    dx, dy, dz = voxel
    st = _ffi.ntvs_paths(nx, ny, nz, n_blocks, dx, dy, dz, nrows, pp, bp_, None if bp is None else bp.ctypes.data,
                         n_seg, kind, min_len)
    check(lib().ntvs_load_paths(ctx, ctypes.byref(st)), "ntvs_load_paths")


def ntvs_load_histories(ctx: int, nx: int, ny: int, nz: int, voxel, hist, b, n_blocks: int = 1, block_ptr=None,
                        n_seg: int = 16, min_len: float = 1e-4) -> None:
    """hist: float32 [M, 12] (P_in, P_out, d_in, d_out), b: float32 [M]; numpy (host) or CUDA tensors."""
    hp, kind = _ptr_kind(hist)
    bp_, kb = _ptr_kind(b)
    if kind != kb:
        raise ValueError("hist and b must both be host arrays or both device tensors")
    bp = None
    if block_ptr is not None:
        bp = np.ascontiguousarray(block_ptr, dtype=np.int64)
        n_blocks = bp.size - 1
    dx, dy, dz = voxel
    st = _ffi.ntvs_histories(nx, ny, nz, n_blocks, dx, dy, dz, hist.shape[0], hp, bp_,
                             None if bp is None else bp.ctypes.data, n_seg, kind, min_len)
    check(lib().ntvs_load_histories(ctx, ctypes.byref(st)), "ntvs_load_histories")


def ntvs_set_params(ctx: int, lam: float, N: int, alpha: float, beta0: float = 1.0, tv_check: bool = False,
                    seed: int = 0, eps_tv: float = 1e-8, max_retries: int = 64, step_rule: int = 0,
                    gamma: float = 0.5) -> None:
    p = _ffi.ntvs_params(lam, alpha, beta0, eps_tv, N, int(bool(tv_check)), max_retries, int(step_rule), seed,
                         gamma)
    check(lib().ntvs_set_params(ctx, ctypes.byref(p)), "ntvs_set_params")


def ntvs_set_image(ctx: int, x) -> None:
    ptr, kind = _ptr_kind(x)
    check(lib().ntvs_set_image(ctx, ptr, _dtype_code(x), kind), "ntvs_set_image")


def ntvs_get_image(ctx: int, out) -> None:
    ptr, kind = _ptr_kind(out)
    check(lib().ntvs_get_image(ctx, ptr, _dtype_code(out), kind), "ntvs_get_image")


def ntvs_run(ctx: int, k_iters: int) -> None:
    check(lib().ntvs_run(ctx, k_iters), "ntvs_run")


def ntvs_sync(ctx: int) -> None:
    check(lib().ntvs_sync(ctx), "ntvs_sync")


def ntvs_get_tv(ctx: int) -> float:
    v = ctypes.c_double()
    check(lib().ntvs_get_tv(ctx, ctypes.byref(v)), "ntvs_get_tv")
    return v.value


def ntvs_get_stats(ctx: int) -> dict:
    st = _ffi.ntvs_stats()
    check(lib().ntvs_get_stats(ctx, ctypes.byref(st)), "ntvs_get_stats")
    return {f: getattr(st, f) for f, _ in _ffi.ntvs_stats._fields_}


def ntvs_get_block_resid(ctx: int, n_blocks: int) -> np.ndarray:
    out = np.zeros(max(n_blocks, 1), np.float64)
    check(lib().ntvs_get_block_resid(ctx, out.ctypes.data, out.size), "ntvs_get_block_resid")
    return out[:n_blocks]


def ntvs_get_trace(ctx: int, cap: int = 1 << 16):
    ell = np.zeros(cap, np.int64)
    tries = np.zeros(cap, np.int32)
    acc = np.zeros(cap, np.int32)
    n = ctypes.c_int64()
    check(lib().ntvs_get_trace(ctx, ell.ctypes.data, tries.ctypes.data, acc.ctypes.data, cap, ctypes.byref(n)),
          "ntvs_get_trace")
    return ell, tries, acc, n.value


def ntvs_get_state(ctx: int):
    k, e = ctypes.c_int64(), ctypes.c_int64()
    check(lib().ntvs_get_state(ctx, ctypes.byref(k), ctypes.byref(e)), "ntvs_get_state")
    return k.value, e.value


def ntvs_set_state(ctx: int, k: int, ell_prev: int) -> None:
    check(lib().ntvs_set_state(ctx, k, ell_prev), "ntvs_set_state")


def ntvs_set_profiling(ctx: int, on: bool) -> None:
    check(lib().ntvs_set_profiling(ctx, int(bool(on))), "ntvs_set_profiling")


def ntvs_get_profile(ctx: int) -> dict:
    pr = _ffi.ntvs_profile()
    check(lib().ntvs_get_profile(ctx, ctypes.byref(pr)), "ntvs_get_profile")
    return {f: getattr(pr, f) for f, _ in _ffi.ntvs_profile._fields_}


def ntvs_set_voxel_tile(ctx: int, tx: int, ty: int) -> None:
    check(lib().ntvs_set_voxel_tile(ctx, int(tx), int(ty)), "ntvs_set_voxel_tile")


def ntvs_set_compute_dtype(ctx: int, dtype: int) -> None:
    check(lib().ntvs_set_compute_dtype(ctx, int(dtype)), "ntvs_set_compute_dtype")


def ntvs_forward_project(ctx: int, x, out) -> None:
    """out[i] = <a_i, x> for every row (x: V values, out: M values; F32/F64, host or device)."""
    xp, xk = _ptr_kind(x)
    op, ok = _ptr_kind(out)
    check(lib().ntvs_forward_project(ctx, xp, _dtype_code(x), xk, op, _dtype_code(out), ok), "ntvs_forward_project")


def ntvs_drop_block_partial(ctx: int, t: int, out, r0: int = -1, r1: int = -1) -> float:
    """delta of rows [r0, r1) of block t (default: the whole block) into `out` (V values,
    F32/F64, numpy = host or CUDA tensor = device), not applied; returns the rows' residual
    sum of squares."""
    ptr, kind = _ptr_kind(out)
    ss = ctypes.c_double()
    check(lib().ntvs_drop_block_partial(ctx, int(t), int(r0), int(r1), ptr, _dtype_code(out), kind, ctypes.byref(ss)),
          "ntvs_drop_block_partial")
    return ss.value


def ntvs_apply_delta(ctx: int, t: int, delta) -> None:
    ptr, kind = _ptr_kind(delta)
    check(lib().ntvs_apply_delta(ctx, int(t), ptr, _dtype_code(delta), kind), "ntvs_apply_delta")


def _require_int32(a, what):
    name = str(a.dtype)
    if not name.endswith("int32"):
        raise TypeError(f"{what} must be int32, got {name}")


def ntvs_get_hit_counts(ctx: int, t: int, out) -> None:
    _require_int32(out, "hit counts")
    ptr, kind = _ptr_kind(out)
    check(lib().ntvs_get_hit_counts(ctx, int(t), ptr, kind), "ntvs_get_hit_counts")


def ntvs_set_hit_counts(ctx: int, t: int, counts) -> None:
    _require_int32(counts, "hit counts")
    ptr, kind = _ptr_kind(counts)
    check(lib().ntvs_set_hit_counts(ctx, int(t), ptr, kind), "ntvs_set_hit_counts")


def shard_rows(row_ptr, col, val, b, block_ptr, rank: int, world: int):
    """Rank `rank`'s rows of a system split over `world` ranks for row-sharded DROP: the
    rows of every block t are cut into `world` contiguous, nearly equal runs and the rank
    keeps run `rank` of each.  Returns (row_ptr, col, val, b, block_ptr) of the shard (host
    arrays; block t of the shard holds the rank's rows of block t)."""
    rp = np.asarray(row_ptr, np.int64)
    bp = np.asarray(block_ptr, np.int64)
    keep, nbp = [], [0]
    for t in range(bp.size - 1):
        n = int(bp[t + 1] - bp[t])
        lo, hi = int(bp[t]) + n * rank // world, int(bp[t]) + n * (rank + 1) // world
        keep.append(np.arange(lo, hi, dtype=np.int64))
        nbp.append(nbp[-1] + hi - lo)
    rows = np.concatenate(keep) if keep else np.zeros(0, np.int64)
    lens = rp[rows + 1] - rp[rows]
    srp = np.zeros(rows.size + 1, np.int64)
    np.cumsum(lens, out=srp[1:])
    idx = np.concatenate([np.arange(rp[i], rp[i + 1], dtype=np.int64) for i in rows]) if rows.size else \
        np.zeros(0, np.int64)
    return srp, np.ascontiguousarray(col[idx]), np.ascontiguousarray(val[idx]), np.ascontiguousarray(b[rows]), \
        np.asarray(nbp, np.int64)


def ntvs_set_allreduce(ctx: int, fn, user=None) -> None:
    """fn: an _ffi.ALLREDUCE_FN (keep a reference while the context uses it) or None."""
    check(lib().ntvs_set_allreduce(ctx, fn if fn is not None else _ffi.ALLREDUCE_FN(), user), "ntvs_set_allreduce")


class _DeviceArray:
    """A raw device buffer described through __cuda_array_interface__ (no copy)."""
    _TYPESTR = {NTVS_F32: "<f4", NTVS_F64: "<f8", _ffi.NTVS_I32: "<i4"}

    def __init__(self, ptr: int, n: int, dtype: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": self._TYPESTR[dtype],
                                         "data": (int(ptr), False), "version": 2}


def torch_allreduce(group=None, device: Optional[int] = None):
    """An all-reduce callback for ntvs_set_allreduce backed by torch.distributed (NCCL on
    GPUs): the library's buffer is wrapped as a tensor and summed over `group` on the
    context's stream.  Keep the returned object alive while the context uses it."""
    import torch
    import torch.distributed as dist
    dev = torch.cuda.current_device() if device is None else device

    def cb(buf, n, dtype, stream, user):
        try:
            t = torch.as_tensor(_DeviceArray(buf, n, dtype), device=f"cuda:{dev}")
            with torch.cuda.stream(torch.cuda.ExternalStream(stream, device=f"cuda:{dev}")):
                dist.all_reduce(t, group=group)
            return 0
        except Exception:   # reported to the library as a failed collective
            return 1

    return _ffi.ALLREDUCE_FN(cb)


def ntvs_set_fault_hook(ctx: int, wait_ns: int, flags: int) -> None:
    check(lib().ntvs_set_fault_hook(ctx, int(wait_ns), int(flags)), "ntvs_set_fault_hook")


def ntvs_set_ell_override(ctx: int, ell) -> None:
    if ell is None:
        check(lib().ntvs_set_ell_override(ctx, None, 0), "ntvs_set_ell_override")
        return
    a = np.ascontiguousarray(ell, np.int64)
    check(lib().ntvs_set_ell_override(ctx, a.ctypes.data, a.size), "ntvs_set_ell_override")


def ntvs_tv_gradient(ctx: int, out=None):
    gn = ctypes.c_double()
    if out is None:
        check(lib().ntvs_tv_gradient(ctx, None, NTVS_F64, NTVS_MEM_HOST, ctypes.byref(gn)), "ntvs_tv_gradient")
    else:
        ptr, kind = _ptr_kind(out)
        check(lib().ntvs_tv_gradient(ctx, ptr, _dtype_code(out), kind, ctypes.byref(gn)), "ntvs_tv_gradient")
    return gn.value


def ntvs_perturb(ctx: int, beta: float) -> None:
    check(lib().ntvs_perturb(ctx, beta), "ntvs_perturb")


def ntvs_perturb_checked(ctx: int, beta: float):
    a, px, pz = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    check(lib().ntvs_perturb_checked(ctx, beta, ctypes.byref(a), ctypes.byref(px), ctypes.byref(pz)),
          "ntvs_perturb_checked")
    return bool(a.value), px.value, pz.value


def ntvs_drop_block(ctx: int, t: int) -> None:
    check(lib().ntvs_drop_block(ctx, t), "ntvs_drop_block")


def ntvs_drop_sweep(ctx: int) -> None:
    check(lib().ntvs_drop_sweep(ctx), "ntvs_drop_sweep")


def _system_struct(nx, ny, nz, row_ptr, col, val, b, n_blocks=1, block_ptr=None, storage=NTVS_CSR32, schedule=0):
    rp, kind = _ptr_kind(row_ptr)
    cp, _ = _ptr_kind(col)
    vptr, _ = _ptr_kind(val)
    bptr, _ = _ptr_kind(b)
    bp = None
    if block_ptr is not None:
        bp = np.ascontiguousarray(block_ptr, dtype=np.int64)
        n_blocks = bp.size - 1
    nrows = (row_ptr.numel() if _is_torch(row_ptr) else row_ptr.size) - 1
    st = _ffi.ntvs_system(nx, ny, nz, n_blocks, nrows, rp, cp, vptr, bptr, None if bp is None else bp.ctypes.data,
                          _dtype_code(val), kind, storage, schedule)
    return st, bp


def ntvs_batch_create(device: int = 0, stream: Optional[int] = None) -> int:
    h = ctypes.c_void_p()
    if stream is not None and int(stream) == 0:
        stream = 1   # cudaStreamLegacy
    check(lib().ntvs_batch_create(ctypes.byref(h), device, stream), "ntvs_batch_create")
    return h.value


def ntvs_batch_destroy(bt: int) -> None:
    check(lib().ntvs_batch_destroy(bt), "ntvs_batch_destroy")


def ntvs_batch_add(bt: int, shape, row_ptr, col, val, b, n_blocks: int, params: "Params", x0, block_ptr=None) -> int:
    nx, ny, nz = shape
    st, _keep = _system_struct(nx, ny, nz, row_ptr, col, val, b, n_blocks, block_ptr)
    p = _params_struct(params)
    xp, xk = _ptr_kind(x0)
    idx = ctypes.c_int()
    check(lib().ntvs_batch_add(bt, ctypes.byref(st), ctypes.byref(p), xp, _dtype_code(x0), xk, ctypes.byref(idx)),
          "ntvs_batch_add")
    return idx.value


def _params_struct(params: "Params"):
    return _ffi.ntvs_params(params.lam, params.alpha, params.beta0, params.eps_tv, params.N,
                            int(bool(params.tv_check)), params.max_retries, int(params.step_rule), params.seed,
                            params.gamma)


def ntvs_batch_add_paths(bt: int, shape, voxel, paths, b, n_blocks: int, params: "Params", x0, block_ptr=None,
                         n_seg: int = 16, min_len: float = 1e-4) -> int:
    """A member from path records (float32 [M, 10]) and b (float32 [M]); numpy or CUDA tensors."""
    nx, ny, nz = shape
    pp, kind = _ptr_kind(paths)
    bp_, kb = _ptr_kind(b)
    if kind != kb:
        raise ValueError("paths and b must both be host arrays or both device tensors")
    bp = None
    if block_ptr is not None:
        bp = np.ascontiguousarray(block_ptr, dtype=np.int64)
        n_blocks = bp.size - 1
    dx, dy, dz = voxel
    st = _ffi.ntvs_paths(nx, ny, nz, n_blocks, dx, dy, dz, paths.shape[0], pp, bp_,
                         None if bp is None else bp.ctypes.data, n_seg, kind, min_len)
    p = _params_struct(params)
    xp, xk = _ptr_kind(x0)
    idx = ctypes.c_int()
    check(lib().ntvs_batch_add_paths(bt, ctypes.byref(st), ctypes.byref(p), xp, _dtype_code(x0), xk,
                                     ctypes.byref(idx)), "ntvs_batch_add_paths")
    return idx.value


def ntvs_batch_set_schedule(bt: int, rows_per_item: int = 0, window_floats: int = -1) -> None:
    check(lib().ntvs_batch_set_schedule(bt, rows_per_item, window_floats), "ntvs_batch_set_schedule")


def ntvs_batch_set_fault_hook(bt: int, wait_ns: int = 0, flags: int = 0) -> None:
    check(lib().ntvs_batch_set_fault_hook(bt, int(wait_ns), flags), "ntvs_batch_set_fault_hook")


def ntvs_batch_sync(bt: int) -> None:
    check(lib().ntvs_batch_sync(bt), "ntvs_batch_sync")


def ntvs_batch_get_member(bt: int, index: int) -> dict:
    out = np.zeros(5, np.int64)
    check(lib().ntvs_batch_get_member(bt, index, out.ctypes.data), "ntvs_batch_get_member")
    return dict(zip(("k", "ell_prev", "n_steps", "n_accepted", "n_tries"), (int(v) for v in out)))


def ntvs_batch_get_sizes(bt: int, index: int):
    """(rows, stored entries) of a member."""
    M, nnz = ctypes.c_int64(), ctypes.c_int64()
    check(lib().ntvs_batch_get_rows(bt, index, ctypes.byref(M), ctypes.byref(nnz), None, None, None),
          "ntvs_batch_get_rows")
    return M.value, nnz.value


def ntvs_batch_get_rows(bt: int, index: int):
    """(row_ptr, col, val) of a member's stored rows (canonical voxel indices)."""
    M, nnz = ctypes.c_int64(), ctypes.c_int64()
    check(lib().ntvs_batch_get_rows(bt, index, ctypes.byref(M), ctypes.byref(nnz), None, None, None),
          "ntvs_batch_get_rows")
    rp = np.empty(M.value + 1, np.int64)
    col = np.empty(nnz.value, np.int32)
    val = np.empty(nnz.value, np.float32)
    check(lib().ntvs_batch_get_rows(bt, index, None, None, rp.ctypes.data, col.ctypes.data, val.ctypes.data),
          "ntvs_batch_get_rows")
    return rp, col, val


def ntvs_batch_get_tuning(bt: int) -> list:
    """[(rows_per_item, window_floats, ctas_per_sm, lanes_per_row_all, ms_per_cycle)] timed at
    finalize (lanes_per_row_all 0: each member's own)."""
    n = ctypes.c_int()
    check(lib().ntvs_batch_get_tuning(bt, None, None, 0, ctypes.byref(n)), "ntvs_batch_get_tuning")
    cand = np.zeros(4 * max(n.value, 1), np.int32)
    ms = np.zeros(max(n.value, 1), np.float32)
    check(lib().ntvs_batch_get_tuning(bt, cand.ctypes.data, ms.ctypes.data, n.value, ctypes.byref(n)),
          "ntvs_batch_get_tuning")
    return [tuple(int(v) for v in cand[4 * i:4 * i + 4]) + (float(ms[i]),) for i in range(n.value)]


def ntvs_batch_finalize(bt: int, max_cycles: int) -> None:
    check(lib().ntvs_batch_finalize(bt, max_cycles), "ntvs_batch_finalize")


def ntvs_batch_run(bt: int, k_iters: int) -> None:
    check(lib().ntvs_batch_run(bt, k_iters), "ntvs_batch_run")


def ntvs_batch_get_image(bt: int, index: int, out) -> None:
    ptr, kind = _ptr_kind(out)
    check(lib().ntvs_batch_get_image(bt, index, ptr, _dtype_code(out), kind), "ntvs_batch_get_image")


def ntvs_batch_get_tv(bt: int, index: int) -> float:
    v = ctypes.c_double()
    check(lib().ntvs_batch_get_tv(bt, index, ctypes.byref(v)), "ntvs_batch_get_tv")
    return v.value


def ntvs_batch_get_stats(bt: int) -> dict:
    st = _ffi.ntvs_batch_stats()
    check(lib().ntvs_batch_get_stats(bt, ctypes.byref(st)), "ntvs_batch_get_stats")
    return {f: getattr(st, f) for f, _ in _ffi.ntvs_batch_stats._fields_}


def ntvs_tv_value_static(x, shape, out, stream: Optional[int] = None) -> None:
    """phi(x) into out[0] without any allocation (see include/ntvs.h): x and out are CUDA
    tensors owned by the caller (x float64/float32 of nx*ny*nz values, out one float64)."""
    nx, ny, nz = shape
    ptr, kind = _ptr_kind(x)
    optr, okind = _ptr_kind(out)
    if kind != NTVS_MEM_DEVICE or okind != NTVS_MEM_DEVICE:
        raise ValueError("x and out must be CUDA tensors")
    check(lib().ntvs_tv_value_static(ptr, _dtype_code(x), nx, ny, nz, optr, stream), "ntvs_tv_value_static")


# ----------------------------------------------------------------- initial iterate (include/ntvs_fbp.h)
def fbp_geom(nx: int, ny: int, nz: int, dx: float, dy: float, dz: float, n_theta: int, n_t: int, dt: float,
             theta0: float = 0.0) -> "_ffi.ntvs_fbp_geom":
    """Geometry of the initial-iterate pipeline (ntvs_fbp_geom of include/ntvs_fbp.h)."""
    return _ffi.ntvs_fbp_geom(nx, ny, nz, n_theta, n_t, 0, dx, dy, dz, dt, theta0)


def _cuda(a, dtype, name: str, numel: Optional[int] = None) -> int:
    """Device pointer of a contiguous CUDA tensor of the given torch dtype (and size)."""
    if not _is_torch(a) or not a.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not a.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if a.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {a.dtype}")
    if numel is not None and a.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {a.numel()}")
    return a.data_ptr()


def _fbp_sizes(g):
    return g.nz * g.n_theta * g.n_t, g.nx * g.ny * g.nz


def ntvs_fbp_bin(g, paths, wepl, sino, count, stream: Optional[int] = None) -> None:
    """Step 1: sino (float64) and count (int32), [nz, n_theta, n_t], from paths (float32
    [M, 10]) and wepl (float64 [M]); CUDA tensors."""
    import torch
    S, _ = _fbp_sizes(g)
    M = int(wepl.numel())
    pp = _cuda(paths, torch.float32, "paths", 10 * M)
    wp = _cuda(wepl, torch.float64, "wepl")
    check(lib().ntvs_fbp_bin(ctypes.byref(g), pp, wp, M, _cuda(sino, torch.float64, "sino", S),
                             _cuda(count, torch.int32, "count", S), stream), "ntvs_fbp_bin")


def ntvs_fbp_filter(g, sino, q, stream: Optional[int] = None) -> None:
    """Step 2: q = Ram-Lak filter of sino along t (float64 CUDA tensors of nz*n_theta*n_t)."""
    import torch
    S, _ = _fbp_sizes(g)
    check(lib().ntvs_fbp_filter(ctypes.byref(g), _cuda(sino, torch.float64, "sino", S),
                                _cuda(q, torch.float64, "q", S), stream), "ntvs_fbp_filter")


def ntvs_fbp_backproject(g, q, img, stream: Optional[int] = None) -> None:
    """Step 3: img (float64, nz*ny*nx) = back-projection of the filtered sinogram q."""
    import torch
    S, V = _fbp_sizes(g)
    check(lib().ntvs_fbp_backproject(ctypes.byref(g), _cuda(q, torch.float64, "q", S),
                                     _cuda(img, torch.float64, "img", V), stream), "ntvs_fbp_backproject")


def ntvs_median_filter(inp, out, shape, radius: int = 2, ball: bool = False, use_hull: bool = False,
                       tau: float = 0.0, stream: Optional[int] = None) -> None:
    """Step 4 (and the hull when use_hull): out = median filter of inp (float64 CUDA
    tensors of nx*ny*nz voxels, shape = (nx, ny, nz))."""
    import torch
    nx, ny, nz = shape
    V = nx * ny * nz
    check(lib().ntvs_median_filter(_cuda(inp, torch.float64, "inp", V), _cuda(out, torch.float64, "out", V),
                                   nx, ny, nz, radius, int(ball), int(use_hull), tau, stream), "ntvs_median_filter")


def ntvs_hull(img, tau: float, stream: Optional[int] = None) -> None:
    """Step 5 in place: voxels <= tau become 0 (float64 CUDA tensor)."""
    import torch
    check(lib().ntvs_hull(_cuda(img, torch.float64, "img"), int(img.numel()), tau, stream), "ntvs_hull")


def ntvs_fbp_workspace_bytes(g) -> int:
    n = int(lib().ntvs_fbp_workspace_bytes(ctypes.byref(g)))
    if n < 0:
        check(n, "ntvs_fbp_workspace_bytes")
    return n


def ntvs_initial_iterate(g, paths, wepl, out, median_radius: int = 2, median_ball: bool = False,
                         use_hull: bool = False, tau: float = 0.0, workspace=None,
                         stream: Optional[int] = None) -> None:
    """Steps 1-5 into out (float64 CUDA tensor of nz*ny*nx voxels).  workspace: a uint8
    CUDA tensor of at least ntvs_fbp_workspace_bytes(g) bytes, allocated here when None."""
    import torch
    _, V = _fbp_sizes(g)
    M = int(wepl.numel())
    need = ntvs_fbp_workspace_bytes(g)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=out.device)
    wsp = _cuda(workspace, torch.uint8, "workspace")
    check(lib().ntvs_initial_iterate(ctypes.byref(g), _cuda(paths, torch.float32, "paths", 10 * M),
                                     _cuda(wepl, torch.float64, "wepl"), M, median_radius, int(median_ball),
                                     int(use_hull), tau, wsp, int(workspace.numel()),
                                     _cuda(out, torch.float64, "out", V), stream), "ntvs_initial_iterate")


# ----------------------------------------------------------------- object wrapper
@dataclass
class Params:
    lam: float = 1e-4
    N: int = 0
    alpha: float = 0.75
    beta0: float = 1.0
    tv_check: bool = False
    seed: int = 0
    eps_tv: float = 1e-8
    max_retries: int = 64
    step_rule: int = 0      # NTVS_STEP_NTVS / NTVS_STEP_OTVS / NTVS_STEP_DECOUPLED
    gamma: float = 0.5      # decoupled rule: beta_{k,n} = beta0 alpha^n gamma^k

    @staticmethod
    def otvs(lam: float = 1e-4, **kw) -> "Params":
        """The paper's OTVS (Appendix B): one checked step per cycle, beta = (1/2)^ell with
        ell counting every try since the start of the run."""
        return Params(lam=lam, N=1, alpha=0.5, beta0=1.0, tv_check=True, step_rule=NTVS_STEP_OTVS, **kw)


class Batch:
    """Independent reconstructions advanced together (see ntvs_batch_* in include/ntvs.h)."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self._bt = ntvs_batch_create(device, stream)
        self.shapes = []

    def add(self, shape, row_ptr, col, val, b, n_blocks: int, params: "Params", x0, block_ptr=None) -> int:
        i = ntvs_batch_add(self._bt, shape, row_ptr, col, val, b, n_blocks, params, x0, block_ptr)
        self.shapes.append(tuple(shape))
        return i

    def add_paths(self, shape, voxel, paths, b, n_blocks: int, params: "Params", x0, block_ptr=None,
                  n_seg: int = 16, min_len: float = 1e-4) -> int:
        i = ntvs_batch_add_paths(self._bt, shape, voxel, paths, b, n_blocks, params, x0, block_ptr, n_seg, min_len)
        self.shapes.append(tuple(shape))
        return i

    def set_schedule(self, rows_per_item: int = 0, window_floats: int = -1):
        ntvs_batch_set_schedule(self._bt, rows_per_item, window_floats)
        return self

    def set_fault_hook(self, wait_ns: int = 0, flags: int = 0):
        ntvs_batch_set_fault_hook(self._bt, wait_ns, flags)
        return self

    def finalize(self, max_cycles: int = 1024):
        ntvs_batch_finalize(self._bt, max_cycles)
        return self

    def sync(self):
        ntvs_batch_sync(self._bt)
        return self

    def member(self, index: int) -> dict:
        return ntvs_batch_get_member(self._bt, index)

    def rows(self, index: int):
        return ntvs_batch_get_rows(self._bt, index)

    def sizes(self, index: int):
        return ntvs_batch_get_sizes(self._bt, index)

    def tuning(self) -> list:
        return ntvs_batch_get_tuning(self._bt)

    def run(self, k: int):
        ntvs_batch_run(self._bt, k)
        return self

    def get_image(self, index: int, dtype=np.float64) -> np.ndarray:
        out = np.empty(int(np.prod(self.shapes[index])), dtype)
        ntvs_batch_get_image(self._bt, index, out)
        return out

    def tv(self, index: int) -> float:
        return ntvs_batch_get_tv(self._bt, index)

    def stats(self) -> dict:
        return ntvs_batch_get_stats(self._bt)

    def close(self):
        if self._bt:
            ntvs_batch_destroy(self._bt)
            self._bt = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Reconstructor:
    """One reconstruction context on one GPU (see include/ntvs.h for the semantics)."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self._ctx = ntvs_create(device, stream)
        self._keep = ()
        self.shape = None
        self.n_blocks = 0

    @property
    def handle(self) -> int:
        return self._ctx

    def close(self) -> None:
        if self._ctx:
            ntvs_destroy(self._ctx)
            self._ctx = None
            self._keep = ()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, shape, row_ptr, col, val, b, n_blocks: int = 1, block_ptr=None, storage: int = NTVS_CSR32,
             schedule: int = 0):
        nx, ny, nz = shape
        ntvs_load_system(self._ctx, nx, ny, nz, row_ptr, col, val, b, n_blocks, block_ptr, storage, schedule)
        self._keep = (row_ptr, col, val, b) if _is_torch(row_ptr) and row_ptr.is_cuda else ()
        self.shape = (nx, ny, nz)
        self.n_blocks = (len(block_ptr) - 1) if block_ptr is not None else n_blocks
        return self

    def load_histories(self, shape, voxel, hist, b, n_blocks: int = 1, block_ptr=None, n_seg: int = 16,
                       min_len: float = 1e-4):
        """System from per-history tracking data [M, 12] (entry/exit points and directions)."""
        nx, ny, nz = shape
        ntvs_load_histories(self._ctx, nx, ny, nz, voxel, hist, b, n_blocks, block_ptr, n_seg, min_len)
        self._keep = (b,) if _is_torch(b) and b.is_cuda else ()
        self.shape = (nx, ny, nz)
        self.n_blocks = (len(block_ptr) - 1) if block_ptr is not None else n_blocks
        return self

    def load_paths(self, shape, voxel, paths, b, n_blocks: int = 1, block_ptr=None, n_seg: int = 16,
                   min_len: float = 1e-4):
        nx, ny, nz = shape
        ntvs_load_paths(self._ctx, nx, ny, nz, voxel, paths, b, n_blocks, block_ptr, n_seg, min_len)
        self._keep = (paths, b) if _is_torch(paths) and paths.is_cuda else ()
        self.shape = (nx, ny, nz)
        self.n_blocks = (len(block_ptr) - 1) if block_ptr is not None else n_blocks
        return self

    def set_params(self, p: Params = None, **kw):
        p = p or Params(**kw)
        ntvs_set_params(self._ctx, p.lam, p.N, p.alpha, p.beta0, p.tv_check, p.seed, p.eps_tv, p.max_retries,
                        p.step_rule, p.gamma)
        return self

    def set_image(self, x):
        ntvs_set_image(self._ctx, x)
        return self

    def get_image(self, dtype=np.float64) -> np.ndarray:
        out = np.empty(int(np.prod(self.shape)), dtype)
        ntvs_get_image(self._ctx, out)
        return out

    def run(self, k: int):
        ntvs_run(self._ctx, k)
        return self

    def sync(self):
        ntvs_sync(self._ctx)
        return self

    def tv(self) -> float:
        return ntvs_get_tv(self._ctx)

    def stats(self) -> dict:
        return ntvs_get_stats(self._ctx)

    def block_resid(self) -> np.ndarray:
        return ntvs_get_block_resid(self._ctx, self.n_blocks)

    def trace(self):
        ell, tries, acc, n = ntvs_get_trace(self._ctx)
        st = self.stats()
        ns = st["n_steps"]
        return ell[:n].copy(), tries[:ns].copy(), acc[:ns].copy()

    def state(self):
        return ntvs_get_state(self._ctx)

    def set_state(self, k: int, ell_prev: int):
        ntvs_set_state(self._ctx, k, ell_prev)
        return self

    def set_profiling(self, on: bool = True):
        ntvs_set_profiling(self._ctx, on)
        return self

    def profile(self) -> dict:
        return ntvs_get_profile(self._ctx)

    def set_ell_override(self, ell):
        ntvs_set_ell_override(self._ctx, ell)
        return self

    def set_voxel_tile(self, tx: int, ty: int):
        """Internal voxel tile of the FP32 path, applied at the next load."""
        ntvs_set_voxel_tile(self._ctx, tx, ty)
        return self

    def set_compute_dtype(self, dtype: int):
        """Arithmetic (NTVS_F32 or NTVS_F64) of FP32-stored systems, applied at the next load."""
        ntvs_set_compute_dtype(self._ctx, dtype)
        return self

    def forward_project(self, x, out=None):
        """A x for the loaded system (every row), as float64 unless `out` is given."""
        if out is None:
            out = np.empty(int(self.stats()["n_rows"]), np.float64)
        ntvs_forward_project(self._ctx, x, out)
        return out

    def drop_block_partial(self, t: int, out=None, r0: int = -1, r1: int = -1):
        """(delta, residual sum of squares) of rows [r0, r1) of block t, not applied."""
        if out is None:
            out = np.empty(int(np.prod(self.shape)), np.float64)
        ss = ntvs_drop_block_partial(self._ctx, t, out, r0, r1)
        return out, ss

    def apply_delta(self, t: int, delta):
        ntvs_apply_delta(self._ctx, t, delta)
        return self

    def hit_counts(self, t: int, out=None):
        if out is None:
            out = np.empty(int(np.prod(self.shape)), np.int32)
        ntvs_get_hit_counts(self._ctx, t, out)
        return out

    def set_hit_counts(self, t: int, counts):
        ntvs_set_hit_counts(self._ctx, t, counts)
        return self

    def set_allreduce(self, fn):
        """Row-sharded mode with all-reduce callback fn (an _ffi.ALLREDUCE_FN, e.g.
        torch_allreduce()); None leaves it."""
        ntvs_set_allreduce(self._ctx, fn)
        self._allreduce = fn   # the library calls it until it is replaced
        return self

    def set_fault_hook(self, wait_ns: int = 0, flags: int = 0):
        """Budget of every bounded device wait and the test flags that starve one."""
        ntvs_set_fault_hook(self._ctx, wait_ns, flags)
        return self

    def tv_gradient(self, dtype=np.float64):
        out = np.empty(int(np.prod(self.shape)), dtype)
        gn = ntvs_tv_gradient(self._ctx, out)
        return out, gn

    def perturb(self, beta: float):
        ntvs_perturb(self._ctx, beta)
        return self

    def perturb_checked(self, beta: float):
        return ntvs_perturb_checked(self._ctx, beta)

    def drop_block(self, t: int):
        ntvs_drop_block(self._ctx, t)
        return self

    def drop_sweep(self):
        ntvs_drop_sweep(self._ctx)
        return self
