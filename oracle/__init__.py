"""FP64 CPU oracle for NTVS (arXiv 1803.01112) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of
``bench.py`` may import this package.  The product library never uses it and shares
no code with it.  The arithmetic is in ``ntvs_oracle.c`` and ``fbp_oracle.c`` (plain
single-threaded C, double precision); this module is argument marshalling.

Pins (what fixes each function independently of itself) live in ``tests/test_oracle_*.py``:
  * orc_splitmix64 / orc_rand_ell : published SplitMix64 outputs, an independent
    Python SplitMix64, and the N=1 no-check identity ell_k = k (Sec. III-B).
  * orc_tv       : phi(const) = 0, closed form of a step edge, homogeneity and shift
    invariance, the 1D total variation.
  * orc_tv_grad  : central finite differences of phi_eps, and a hand-expanded 2x2x1 case.
  * orc_drop_block / orc_drop_sweep : exact hyperplane projection of one-row blocks,
    the one-row closed form, fixed points of consistent systems, convergence to the
    numpy least-squares solution, a hand-computed 3-voxel 4-row block.
  * orc_drop_block_at : equals orc_drop_block on every voxel of small cases.
  * orc_fbp_* / orc_median / orc_hull / orc_initial_iterate (fbp_oracle.c): analytic
    disc projections reconstruct to the disc, hand-worked bins and angle folds,
    hand-made median cases and scipy's median filter on interior voxels, the noise-free
    phantom reconstructed end to end.
  * orc_ntvs     : N = 0 is plain DROP; the check variant without rejections equals
    the variant without the check; accepted steps never raise phi; ell_k >= k.
    OTVS and decoupled step rules: closed forms of the total shift of a two-voxel image
    (every step moves both voxels by beta/sqrt(2)), including OTVS rejections worked by
    hand; OTVS ell_k equals the running count of tries; decoupled with gamma = alpha
    equals NTVS with ell_k = k replayed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ntvs_oracle.c")
_SRC_FBP = os.path.join(_HERE, "fbp_oracle.c")   # the initial iterate (FBP, median, hull)
_SO = os.path.join(_HERE, "libntvs_oracle.so")
_SO_OMP = os.path.join(_HERE, "libntvs_oracle_omp.so")   # timing build on all host cores


def build_command(out: str = _SO, omp: bool = False):
    return ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared"] + (["-fopenmp"] if omp else []) + \
        ["-o", out, _SRC, _SRC_FBP, "-lm"]


def build(force: bool = False, omp: bool = False) -> str:
    so = _SO_OMP if omp else _SO
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_FBP))
    if force or not os.path.exists(so) or os.path.getmtime(so) < newest:
        subprocess.run(build_command(so, omp), check=True)
    return so


class _Params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("alpha", ctypes.c_double), ("beta0", ctypes.c_double),
                ("eps_tv", ctypes.c_double), ("N", ctypes.c_int32), ("tv_check", ctypes.c_int32),
                ("max_retries", ctypes.c_int32), ("step_rule", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("gamma", ctypes.c_double)]


class _Trace(ctypes.Structure):
    _fields_ = [("ell_k", ctypes.c_void_p), ("ell_step", ctypes.c_void_p), ("tries", ctypes.c_void_p),
                ("accepted", ctypes.c_void_p), ("tv", ctypes.c_void_p), ("resid_ss", ctypes.c_void_p),
                ("beta_step", ctypes.c_void_p)]


class FbpGeom(ctypes.Structure):
    """Geometry of the initial-iterate pipeline: image grid (in-plane centred on the
    origin, slice iz over z in [iz dz, (iz+1) dz)), n_theta angle bins of width pi/n_theta
    from theta0, and n_t lateral bins of width dt centred on t = 0."""
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("n_theta", ctypes.c_int32), ("n_t", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("theta0", ctypes.c_double)]


def fbp_geom(nx, ny, nz, dx, dy, dz, n_theta, n_t, dt, theta0=0.0) -> FbpGeom:
    return FbpGeom(nx, ny, nz, n_theta, n_t, 0, dx, dy, dz, dt, theta0)


_L = {}


def _lib(omp: bool = False):
    """The checker (single-threaded) or, with omp, the OpenMP timing build of the same source."""
    if omp not in _L:
        L = ctypes.CDLL(build(omp=omp))
        vp, i64, u64, d, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int32
        L.orc_splitmix64.argtypes = [u64, u64]; L.orc_splitmix64.restype = u64
        L.orc_rand_ell.argtypes = [u64, i64, i64]; L.orc_rand_ell.restype = i64
        L.orc_tv.argtypes = [vp, i32, i32, i32, d]; L.orc_tv.restype = d
        L.orc_tv_grad.argtypes = [vp, i32, i32, i32, d, vp]; L.orc_tv_grad.restype = None
        L.orc_drop_block.argtypes = [vp, vp, vp, vp, i64, i64, i64, d, vp, vp]; L.orc_drop_block.restype = None
        L.orc_drop_sweep.argtypes = [vp, vp, vp, vp, vp, i32, i64, d, vp, vp]; L.orc_drop_sweep.restype = None
        L.orc_drop_block_at.argtypes = [vp, vp, vp, vp, i64, i64, i64, d, vp, i64, vp, vp]
        L.orc_drop_block_at.restype = None
        L.orc_ntvs.argtypes = [vp, vp, vp, vp, vp, i32, i32, i32, i32, ctypes.POINTER(_Params),
                               i32, i32, ctypes.POINTER(i64), vp, vp, ctypes.POINTER(_Trace)]
        L.orc_ntvs.restype = i32
        G = ctypes.POINTER(FbpGeom)
        L.orc_fbp_line.argtypes = [vp, vp, vp, vp]; L.orc_fbp_line.restype = i32
        L.orc_fbp_bin_of.argtypes = [vp, G, vp, vp, vp]; L.orc_fbp_bin_of.restype = i32
        L.orc_fbp_bin.argtypes = [vp, vp, i64, G, vp, vp]; L.orc_fbp_bin.restype = None
        L.orc_ramlak.argtypes = [i64, d]; L.orc_ramlak.restype = d
        L.orc_fbp_filter.argtypes = [vp, G, vp]; L.orc_fbp_filter.restype = None
        L.orc_fbp_backproject.argtypes = [vp, G, vp]; L.orc_fbp_backproject.restype = None
        L.orc_median_window.argtypes = [i32, i32, vp]; L.orc_median_window.restype = i32
        L.orc_median.argtypes = [vp, i32, i32, i32, i32, i32, vp]; L.orc_median.restype = None
        L.orc_hull.argtypes = [vp, i64, d]; L.orc_hull.restype = None
        L.orc_initial_iterate.argtypes = [vp, vp, i64, G, i32, i32, i32, d, vp]
        L.orc_initial_iterate.restype = None
        _L[omp] = L
    return _L[omp]


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


# ------------------------------------------------------------------ RNG / schedule
def splitmix64(seed: int, n: int) -> int:
    return int(_lib().orc_splitmix64(seed, n))


def rand_ell(seed: int, k: int, ell_prev: int) -> int:
    return int(_lib().orc_rand_ell(seed, k, ell_prev))


# ------------------------------------------------------------------ TV
def tv(x, shape, eps: float = 0.0) -> float:
    nx, ny, nz = shape
    x = _f64(x).reshape(-1)
    assert x.size == nx * ny * nz
    return float(_lib().orc_tv(x.ctypes.data, nx, ny, nz, eps))


def tv_grad(x, shape, eps: float) -> np.ndarray:
    nx, ny, nz = shape
    x = _f64(x).reshape(-1)
    g = np.empty_like(x)
    _lib().orc_tv_grad(x.ctypes.data, nx, ny, nz, eps, g.ctypes.data)
    return g


# ------------------------------------------------------------------ DROP
def _csr(row_ptr, col, val, b):
    return (np.ascontiguousarray(row_ptr, np.int64), np.ascontiguousarray(col, np.int32),
            _f64(val), _f64(b))


def drop_block(row_ptr, col, val, b, r0: int, r1: int, x, lam: float):
    rp, c, v, bb = _csr(row_ptr, col, val, b)
    x = _f64(x).copy()
    ss = ctypes.c_double(0.0)
    _lib().orc_drop_block(rp.ctypes.data, c.ctypes.data, v.ctypes.data, bb.ctypes.data, r0, r1, x.size,
                          lam, x.ctypes.data, ctypes.byref(ss))
    return x, ss.value


def drop_sweep(row_ptr, col, val, b, block_ptr, x, lam: float):
    rp, c, v, bb = _csr(row_ptr, col, val, b)
    bp = np.ascontiguousarray(block_ptr, np.int64)
    B = bp.size - 1
    x = _f64(x).copy()
    ss = np.zeros(max(B, 1), np.float64)
    _lib().orc_drop_sweep(rp.ctypes.data, c.ctypes.data, v.ctypes.data, bb.ctypes.data, bp.ctypes.data, B,
                          x.size, lam, x.ctypes.data, ss.ctypes.data)
    return x, ss[:B]


def drop_block_at(row_ptr, col, val, b, r0: int, r1: int, x, lam: float, vox) -> np.ndarray:
    rp, c, v, bb = _csr(row_ptr, col, val, b)
    x = _f64(x)
    vox = np.ascontiguousarray(vox, np.int64)
    out = np.empty(vox.size, np.float64)
    _lib().orc_drop_block_at(rp.ctypes.data, c.ctypes.data, v.ctypes.data, bb.ctypes.data, r0, r1, x.size,
                             lam, x.ctypes.data, vox.size, vox.ctypes.data, out.ctypes.data)
    return out


# ------------------------------------------------------------------ NTVS
STEP_NTVS = 0        # ell_k = rand(k, ell_{k-1})                      (Appendix C)
STEP_OTVS = 1        # ell_k = ell_{k-1}: ell never reset               (Appendix B)
STEP_DECOUPLED = 2   # beta_{k,n} = beta0 alpha^n gamma^k, no check      (Sec. VI)


@dataclass
class Params:
    lam: float
    N: int
    alpha: float
    beta0: float = 1.0
    tv_check: bool = False
    seed: int = 0
    eps_tv: float = 1e-8
    max_retries: int = 64
    step_rule: int = STEP_NTVS
    gamma: float = 0.5

    @staticmethod
    def otvs(lam: float, **kw) -> "Params":
        """The paper's OTVS (Appendix B): one checked step per cycle, beta = (1/2)^ell with
        ell counting every try since the start."""
        return Params(lam=lam, N=1, alpha=0.5, beta0=1.0, tv_check=True, step_rule=STEP_OTVS, **kw)


@dataclass
class Result:
    x: np.ndarray
    ell_k: np.ndarray
    ell_step: np.ndarray
    tries: np.ndarray
    accepted: np.ndarray
    tv: np.ndarray
    resid_ss: np.ndarray
    ell_prev: int
    beta_step: np.ndarray


def ntvs(row_ptr, col, val, b, block_ptr, shape, params: Params, K: int, x0,
         k0: int = 0, ell_prev: int = 0, ell_override: Optional[np.ndarray] = None, omp: bool = False) -> Result:
    """K cycles of NTVS from x0 (Appendix C); returns the image and the traces.  omp=True
    runs the OpenMP timing build (all host cores; summation order differs) -- for timing
    only, never as the checker."""
    nx, ny, nz = shape
    rp, c, v, bb = _csr(row_ptr, col, val, b)
    bp = np.ascontiguousarray(block_ptr, np.int64)
    B = bp.size - 1
    x = _f64(x0).reshape(-1).copy()
    N = params.N
    ell_k = np.zeros(max(K, 1), np.int64)
    ell_step = np.zeros(max(K * N, 1), np.int64)
    tries = np.zeros(max(K * N, 1), np.int32)
    accepted = np.zeros(max(K * N, 1), np.int32)
    tvs = np.zeros(max(K, 1), np.float64)
    rss = np.zeros(max(K * B, 1), np.float64)
    bst = np.zeros(max(K * N, 1), np.float64)
    tr = _Trace(ell_k.ctypes.data, ell_step.ctypes.data, tries.ctypes.data, accepted.ctypes.data,
                tvs.ctypes.data, rss.ctypes.data, bst.ctypes.data)
    p = _Params(params.lam, params.alpha, params.beta0, params.eps_tv, N, int(params.tv_check),
                params.max_retries, int(params.step_rule), params.seed, params.gamma)
    ep = ctypes.c_int64(ell_prev)
    ov = None if ell_override is None else np.ascontiguousarray(ell_override, np.int64)
    rc = _lib(omp).orc_ntvs(rp.ctypes.data, c.ctypes.data, v.ctypes.data, bb.ctypes.data, bp.ctypes.data, B,
                         nx, ny, nz, ctypes.byref(p), K, k0, ctypes.byref(ep), _ptr(ov), x.ctypes.data,
                         ctypes.byref(tr))
    if rc != 0:
        raise ValueError("oracle: unknown step rule, or the decoupled rule with the TV check")
    return Result(x, ell_k[:K], ell_step[:K * N].reshape(K, N), tries[:K * N].reshape(K, N),
                  accepted[:K * N].reshape(K, N), tvs[:K], rss[:K * B].reshape(K, B), int(ep.value),
                  bst[:K * N].reshape(K, N))


# ------------------------------------------------------------------ initial iterate (FBP, median, hull)
def _paths32(paths):
    p = np.ascontiguousarray(paths, np.float32)
    assert p.ndim == 2 and p.shape[1] == 10
    return p


def fbp_line(rec):
    """(theta, t, z) of one history's chord line, or None for an empty record."""
    r = np.ascontiguousarray(rec, np.float32).reshape(10)
    th, t, z = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    ok = _lib().orc_fbp_line(r.ctypes.data, ctypes.byref(th), ctypes.byref(t), ctypes.byref(z))
    return (th.value, t.value, z.value) if ok else None


def fbp_bin_of(rec, g: FbpGeom):
    """(slice, angle bin, lateral bin) of one history, or None outside the bins."""
    r = np.ascontiguousarray(rec, np.float32).reshape(10)
    iz, ia, it = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    ok = _lib().orc_fbp_bin_of(r.ctypes.data, ctypes.byref(g), ctypes.byref(iz), ctypes.byref(ia),
                               ctypes.byref(it))
    return (iz.value, ia.value, it.value) if ok else None


def fbp_bin(paths, wepl, g: FbpGeom):
    """Sinogram [nz, n_theta, n_t] of mean WEPL per bin and the history counts."""
    p = _paths32(paths)
    w = _f64(wepl)
    sino = np.empty((g.nz, g.n_theta, g.n_t), np.float64)
    cnt = np.empty((g.nz, g.n_theta, g.n_t), np.int64)
    _lib().orc_fbp_bin(p.ctypes.data, w.ctypes.data, p.shape[0], ctypes.byref(g), sino.ctypes.data,
                       cnt.ctypes.data)
    return sino, cnt


def ramlak(m: int, dt: float) -> float:
    return float(_lib().orc_ramlak(m, dt))


def fbp_filter(sino, g: FbpGeom) -> np.ndarray:
    s = _f64(sino).reshape(g.nz, g.n_theta, g.n_t)
    q = np.empty_like(s)
    _lib().orc_fbp_filter(s.ctypes.data, ctypes.byref(g), q.ctypes.data)
    return q


def fbp_backproject(q, g: FbpGeom) -> np.ndarray:
    qq = _f64(q).reshape(g.nz, g.n_theta, g.n_t)
    img = np.empty(g.nx * g.ny * g.nz, np.float64)
    _lib().orc_fbp_backproject(qq.ctypes.data, ctypes.byref(g), img.ctypes.data)
    return img


def median_window(r: int, ball: bool) -> np.ndarray:
    n = _lib().orc_median_window(r, int(ball), None)
    off = np.empty((n, 3), np.int32)
    _lib().orc_median_window(r, int(ball), off.ctypes.data)
    return off


def median(img, shape, r: int, ball: bool = False) -> np.ndarray:
    nx, ny, nz = shape
    x = _f64(img).reshape(-1)
    assert x.size == nx * ny * nz
    out = np.empty_like(x)
    _lib().orc_median(x.ctypes.data, nx, ny, nz, r, int(ball), out.ctypes.data)
    return out


def hull(img, tau: float) -> np.ndarray:
    x = _f64(img).reshape(-1).copy()
    _lib().orc_hull(x.ctypes.data, x.size, tau)
    return x


def initial_iterate(paths, wepl, g: FbpGeom, median_r: int = 2, median_ball: bool = False,
                    use_hull: bool = False, tau: float = 0.0) -> np.ndarray:
    p = _paths32(paths)
    w = _f64(wepl)
    out = np.empty(g.nx * g.ny * g.nz, np.float64)
    _lib().orc_initial_iterate(p.ctypes.data, w.ctypes.data, p.shape[0], ctypes.byref(g), median_r,
                               int(median_ball), int(use_hull), tau, out.ctypes.data)
    return out
