"""Seeded synthetic proton-CT systems (input generator shared by the CUDA path and the oracle).

The paper's data (Geant4-simulated and experimental CTP404 scans, Sec. III-C) are not
available, so inputs are synthesised with the paper's geometry: 1x1x2.5 mm voxels and
200x200 slices (Sec. III-D), a 150 mm cylinder with 12.2 mm inserts on a 120 mm circle
carrying the simulated RSPs of Table I, parallel projections over a full turn.

Each history contributes one row a_i of intersection lengths through the voxel grid and
one right-hand side b_i = WEPL = (a_i . x*) (1 + sigma z), z ~ N(0,1).  Rows are emitted
angle by angle; inside an angle they are ordered by (z slice, lateral offset).

This module holds no reconstruction arithmetic and imports neither the CUDA library
nor the oracle.  The heavy lifting is in ``ntvs_synth.c`` (OpenMP, counter-based
SplitMix64 so the output does not depend on the thread count).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Callable, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ntvs_synth.c")
_SO = os.path.join(_HERE, "libntvs_synth.so")


def build_command(out: str = _SO):
    # -ffp-contract=off: the same bits on x86-64 and aarch64 hosts (no FMA contraction)
    return ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
            "-o", out, _SRC, "-lm"]


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.run(build_command(), check=True)
    return _SO


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("cyl_r", ctypes.c_double), ("cyl_rsp", ctypes.c_double),
        ("n_ins", ctypes.c_int32),
        ("ins_cx", ctypes.c_void_p), ("ins_cy", ctypes.c_void_p),
        ("ins_r", ctypes.c_void_p), ("ins_rsp", ctypes.c_void_p),
        ("n_hist", ctypes.c_int64), ("n_angles", ctypes.c_int32),
        ("angle_span_deg", ctypes.c_double),
        ("curved", ctypes.c_int32), ("n_seg", ctypes.c_int32),
        ("dev_max", ctypes.c_double), ("noise_sigma", ctypes.c_double),
        ("min_len", ctypes.c_double), ("lateral_width", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        L = ctypes.CDLL(_SO)
        vp = ctypes.c_void_p
        L.syn_phantom.argtypes = [ctypes.POINTER(_Cfg), vp, vp, vp]
        L.syn_plan.argtypes = [ctypes.POINTER(_Cfg), vp, vp, vp, vp]
        L.syn_count.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int64, vp, vp, vp, vp, vp]
        L.syn_fill.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int32,
                               vp, vp]
        L.syn_paths.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int64, vp, vp, vp, vp, vp]
        L.syn_rhs.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int64, vp, vp, vp, vp, vp, vp]
        L.syn_paths.restype = None
        L.syn_rhs.restype = None
        L.syn_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.syn_splitmix64_at.restype = ctypes.c_uint64
        for f in ("syn_phantom", "syn_plan", "syn_count", "syn_fill"):
            getattr(L, f).restype = None
        _lib_handle = L
    return _lib_handle


@dataclasses.dataclass(frozen=True)
class Insert:
    cx: float
    cy: float
    r: float
    rsp: float


@dataclasses.dataclass(frozen=True)
class Spec:
    """Geometry, phantom and acquisition of one synthetic reconstruction problem."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    cyl_r: float
    cyl_rsp: float
    inserts: Tuple[Insert, ...]
    n_hist: int
    n_angles: int
    curved: bool
    n_blocks: int
    seed: int
    angle_span_deg: float = 360.0
    n_seg: int = 16
    dev_max: float = 2.0
    noise_sigma: float = 0.01
    min_len: float = 1e-4
    lateral_width: Optional[float] = None   # default: the cylinder diameter (beam field on the object)

    @property
    def V(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Spec":
        return dataclasses.replace(self, **kw)


def _ring(n, radius, r, rsps, phase_deg=0.0):
    out = []
    for i, rsp in enumerate(rsps):
        a = math.radians(phase_deg + 360.0 * i / n)
        out.append(Insert(radius * math.cos(a), radius * math.sin(a), r, float(rsp)))
    return tuple(out)


# Table I, simulated row: air, air, PMP, LDPE, polystyrene, acrylic, Delrin, Teflon;
# Teflon's 1.828 is clipped to 1.8 so every insert lies in [0, 1.8].
CTP404_SIM_RSP = (0.0013, 0.0013, 0.877, 0.9973, 1.0386, 1.155, 1.356, 1.8)


def spec_slice_2d(seed: int = 1) -> Spec:
    """2D 32x32 slice (1 mm), r=14 mm RSP-1.0 cylinder, 4 inserts (r=3 mm at 8 mm) RSP
    {0.0, 0.3, 1.2, 1.7}, 20k straight histories over 90 angles, 10 blocks."""
    return Spec(name="slice32_2d_straight_20k", nx=32, ny=32, nz=1, dx=1.0, dy=1.0, dz=1.0,
                cyl_r=14.0, cyl_rsp=1.0, inserts=_ring(4, 8.0, 3.0, (0.0, 0.3, 1.2, 1.7)),
                n_hist=20_000, n_angles=90, curved=False, n_blocks=10, seed=seed)


def spec_ctp404_3d(seed: int = 2) -> Spec:
    """200x200x16 voxels of 1x1x2.5 mm, 150 mm cylinder with 8 inserts (12.2 mm on a
    120 mm circle), 10M bent histories over 360 angles, 20 blocks."""
    return Spec(name="ctp404_200x200x16_curved_10M", nx=200, ny=200, nz=16, dx=1.0, dy=1.0, dz=2.5,
                cyl_r=75.0, cyl_rsp=1.0, inserts=_ring(8, 60.0, 6.1, CTP404_SIM_RSP),
                n_hist=10_000_000, n_angles=360, curved=True, n_blocks=20, seed=seed)


def spec_scaled_3d(nx=40, ny=40, nz=4, n_hist=40_000, n_angles=60, n_blocks=5, seed=3,
                   curved=True) -> Spec:
    """The 3D CTP404-like problem at a reduced size (for parity tests): the phantom is
    scaled with the grid so inserts stay several voxels wide."""
    s = nx / 200.0
    return Spec(name=f"ctp404_{nx}x{ny}x{nz}_{'curved' if curved else 'straight'}_{n_hist}",
                nx=nx, ny=ny, nz=nz, dx=1.0, dy=1.0, dz=2.5,
                cyl_r=75.0 * s, cyl_rsp=1.0, inserts=_ring(8, 60.0 * s, max(6.1 * s, 1.5), CTP404_SIM_RSP),
                n_hist=n_hist, n_angles=n_angles, curved=curved, n_blocks=n_blocks, seed=seed,
                dev_max=min(2.0, 2.0 * s * 2))


def spec_batch_member(seed: int, nx: int, ny: int, nz: int, n_hist: int, n_blocks: int = 20) -> Spec:
    """One member of a batched parameter sweep: a cylinder filling the grid with 4-8 random,
    non-overlapping cylindrical inserts of RSP U[0, 1.8]; bent paths over 90 angles."""
    rng = np.random.default_rng(seed)
    R = 0.45 * min(nx, ny)
    ins = []
    for _ in range(200):
        if len(ins) >= int(rng.integers(4, 9)):
            break
        r = float(rng.uniform(0.06, 0.12) * R)
        rho = float(rng.uniform(0.0, 0.75 * R))
        phi = float(rng.uniform(0.0, 2.0 * math.pi))
        cx, cy = rho * math.cos(phi), rho * math.sin(phi)
        if all((cx - i.cx) ** 2 + (cy - i.cy) ** 2 > (r + i.r + 1.0) ** 2 for i in ins) and rho + r < R - 1.0:
            ins.append(Insert(cx, cy, r, float(rng.uniform(0.0, 1.8))))
    return Spec(name=f"member{seed}_{nx}x{ny}x{nz}_{n_hist}", nx=nx, ny=ny, nz=nz, dx=1.0, dy=1.0, dz=2.5,
                cyl_r=R, cyl_rsp=1.0, inserts=tuple(ins), n_hist=n_hist, n_angles=90, curved=True,
                n_blocks=n_blocks, seed=seed)


@dataclasses.dataclass
class System:
    spec: Spec
    row_ptr: np.ndarray     # int64 [M+1]
    col: np.ndarray         # int32 [nnz], voxel index (iz*ny + iy)*nx + ix
    val: np.ndarray         # float64 or float32 [nnz], intersection length (mm)
    b: np.ndarray           # float64 [M], WEPL (mm)
    xstar: np.ndarray       # float64 [V], phantom
    xbar: np.ndarray        # float64 [V], initial iterate (1 inside the cylinder, else 0)
    label: np.ndarray       # int32 [V], insert index / n_ins for background / -1 outside
    angle: np.ndarray       # int32 [M], projection index of each row
    t: np.ndarray           # float64 [M], lateral offset of each history (mm)
    z: np.ndarray           # float64 [M], height of each history (mm)

    @property
    def M(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def block_ptr(self, n_blocks: Optional[int] = None) -> np.ndarray:
        return block_partition(self.M, self.spec.n_blocks if n_blocks is None else n_blocks)


def block_partition(M: int, B: int) -> np.ndarray:
    """Contiguous blocks of ceil(M/B) rows in stored order (the last one may be shorter,
    trailing ones empty when B > M)."""
    per = -(-M // B) if B > 0 else 0
    return np.minimum(np.arange(B + 1, dtype=np.int64) * per, M).astype(np.int64)


def _cfg(spec: Spec, keep):
    ins = spec.inserts
    arrs = [np.ascontiguousarray([getattr(i, f) for i in ins] or [0.0], dtype=np.float64)
            for f in ("cx", "cy", "r", "rsp")]
    keep.extend(arrs)
    w = spec.lateral_width if spec.lateral_width is not None else 2.0 * spec.cyl_r
    return _Cfg(spec.nx, spec.ny, spec.nz, spec.dx, spec.dy, spec.dz, spec.cyl_r, spec.cyl_rsp,
                len(ins), *[a.ctypes.data for a in arrs], spec.n_hist, spec.n_angles,
                spec.angle_span_deg, int(spec.curved), spec.n_seg, spec.dev_max,
                spec.noise_sigma, spec.min_len, w, spec.seed)


def phantom(spec: Spec):
    keep = []
    c = _cfg(spec, keep)
    xstar = np.empty(spec.V, np.float64)
    xbar = np.empty(spec.V, np.float64)
    label = np.empty(spec.V, np.int32)
    _lib().syn_phantom(ctypes.byref(c), xstar.ctypes.data, xbar.ctypes.data, label.ctypes.data)
    return xstar, xbar, label


def generate(spec: Spec, val_dtype=np.float64,
             alloc: Callable[[Sequence[int], np.dtype], np.ndarray] = None,
             rows: Optional[Tuple[int, int]] = None) -> System:
    """Generate the system, or only its rows [r0, r1) when ``rows`` is given (the same rows
    the whole system has there).  ``alloc(shape, dtype)`` provides the col / val / b
    buffers (e.g. views of pinned host memory); default ``np.empty``."""
    val_dtype = np.dtype(val_dtype)
    if val_dtype not in (np.dtype(np.float64), np.dtype(np.float32)):
        raise ValueError("val_dtype must be float64 or float32")
    alloc = alloc or (lambda shape, dt: np.empty(shape, dt))
    keep = []
    c = _cfg(spec, keep)
    L = _lib()
    M = spec.n_hist
    xstar, xbar, label = phantom(spec)
    t = np.empty(M, np.float64)
    z = np.empty(M, np.float64)
    key = np.empty(M, np.uint64)
    angle = np.empty(M, np.int32)
    L.syn_plan(ctypes.byref(c), t.ctypes.data, z.ctypes.data, key.ctypes.data, angle.ctypes.data)
    if rows is not None:
        r0, r1 = rows
        t, z, key, angle = (np.ascontiguousarray(a[r0:r1]) for a in (t, z, key, angle))
        M = r1 - r0
    nnz_row = np.empty(M, np.int64)
    L.syn_count(ctypes.byref(c), M, t.ctypes.data, z.ctypes.data, key.ctypes.data, angle.ctypes.data,
                nnz_row.ctypes.data)
    row_ptr = np.zeros(M + 1, np.int64)
    np.cumsum(nnz_row, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = alloc((nnz,), np.dtype(np.int32))
    val = alloc((nnz,), val_dtype)
    b = np.empty(M, np.float64)
    L.syn_fill(ctypes.byref(c), M, t.ctypes.data, z.ctypes.data, key.ctypes.data, angle.ctypes.data,
               row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data,
               0 if val_dtype == np.float64 else 1, b.ctypes.data, xstar.ctypes.data)
    return System(spec, row_ptr, col, val, b, xstar, xbar, label, angle, t, z)


@dataclasses.dataclass
class Paths:
    """Histories as path records (float32 [M, 10]: P_in xyz, P_out xyz, A_lat, B_lat, A_z,
    B_z; see ntvs_synth.c) with their WEPL b, the phantom and the initial iterate."""
    spec: Spec
    paths: np.ndarray
    b: np.ndarray
    xstar: np.ndarray
    xbar: np.ndarray
    label: np.ndarray

    @property
    def M(self) -> int:
        return int(self.paths.shape[0])


def generate_paths(spec: Spec, rows: Optional[Tuple[int, int]] = None, with_rhs: bool = True) -> Paths:
    """The same histories as ``generate`` (same rows, same b) as path records, without the
    matrix; b is traced row by row without being stored."""
    keep = []
    c = _cfg(spec, keep)
    L = _lib()
    M = spec.n_hist
    xstar, xbar, label = phantom(spec)
    t = np.empty(M, np.float64)
    z = np.empty(M, np.float64)
    key = np.empty(M, np.uint64)
    angle = np.empty(M, np.int32)
    L.syn_plan(ctypes.byref(c), t.ctypes.data, z.ctypes.data, key.ctypes.data, angle.ctypes.data)
    if rows is not None:
        r0, r1 = rows
        t, z, key, angle = (np.ascontiguousarray(a[r0:r1]) for a in (t, z, key, angle))
        M = r1 - r0
    paths = np.empty((M, 10), np.float32)
    L.syn_paths(ctypes.byref(c), M, t.ctypes.data, z.ctypes.data, key.ctypes.data, angle.ctypes.data,
                paths.ctypes.data)
    b = np.zeros(M, np.float64)
    if with_rhs:
        L.syn_rhs(ctypes.byref(c), M, t.ctypes.data, z.ctypes.data, key.ctypes.data, angle.ctypes.data,
                  b.ctypes.data, xstar.ctypes.data)
    return Paths(spec, paths, b, xstar, xbar, label)


def spec_large_onthefly(seed: int = 5, n_hist: int = 60_000_000) -> Spec:
    """256x256x64 voxels of 0.8x0.8x1.25 mm, 720 angles, bent paths, 40 blocks (the grid is
    scaled from the CTP404 layout)."""
    s = 256 * 0.8 / 200.0
    return Spec(name=f"ctp404_256x256x64_onthefly_{n_hist}", nx=256, ny=256, nz=64, dx=0.8, dy=0.8, dz=1.25,
                cyl_r=75.0 * s, cyl_rsp=1.0, inserts=_ring(8, 60.0 * s, 6.1 * s, CTP404_SIM_RSP),
                n_hist=n_hist, n_angles=720, curved=True, n_blocks=40, seed=seed)


def splitmix64_at(seed: int, n: int) -> int:
    return int(_lib().syn_splitmix64_at(seed, n))


def random_image(shape_or_V, seed: int, lo=0.0, hi=2.0) -> np.ndarray:
    """Seeded uniform image (float64) for stencil tests."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape_or_V)
