"""Helpers shared by the GPU tests: build/load the library once, marshal synthetic systems."""
import numpy as np
import pytest

import oracle
import synth


def ntvs_module():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1803_01112_gb300 as ntvs
    from paper_1803_01112_gb300 import _build
    _build.build()
    ntvs.lib()
    return ntvs


def as_stored(s: synth.System, val_dtype):
    """The system as the GPU stores it (values, b in the compute type) and the same
    values upcast to FP64 for the oracle."""
    if val_dtype == np.float64:
        return s.val, s.b, s.val, s.b
    val = s.val.astype(np.float32)
    b = s.b.astype(np.float32)
    return val, b, val.astype(np.float64), b.astype(np.float64)


def load(ntvs, s: synth.System, val_dtype=np.float64, n_blocks=None, block_ptr=None):
    val, b, val64, b64 = as_stored(s, val_dtype)
    r = ntvs.Reconstructor(0)
    shape = (s.spec.nx, s.spec.ny, s.spec.nz)
    B = s.spec.n_blocks if n_blocks is None else n_blocks
    r.load(shape, s.row_ptr, s.col, val, b, n_blocks=B, block_ptr=block_ptr)
    return r, val64, b64


def empty_system(ntvs, shape):
    """A context with geometry but no rows (for TV-only tests)."""
    r = ntvs.Reconstructor(0)
    r.load(shape, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float64), np.zeros(0, np.float64))
    return r


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def stored_image(x, dtype):
    return np.asarray(x, dtype).astype(np.float64)


def oracle_run(s, val64, b64, prm: oracle.Params, K, x0, block_ptr=None, **kw):
    shape = (s.spec.nx, s.spec.ny, s.spec.nz)
    bp = s.block_ptr() if block_ptr is None else block_ptr
    return oracle.ntvs(s.row_ptr, s.col, val64, b64, bp, shape, prm, K, x0, **kw)


def quantize(val, kind):
    """Values as stored in half precision, returned as (array to hand to the library,
    float64 copy of the stored values for the oracle)."""
    import torch
    if kind == "fp16":
        q = np.asarray(val, np.float16)
        return q, q.astype(np.float64)
    if kind == "bf16":
        t = torch.from_numpy(np.asarray(val, np.float32)).to(torch.bfloat16)
        return t, t.to(torch.float64).numpy()
    raise ValueError(kind)


def roi_means(x, spec, frac=0.75):
    """Mean of x over a circle of radius frac * (insert radius) around every insert centre,
    in every slice, plus the background ring midway between the inserts and the cylinder."""
    nx, ny, nz = spec.nx, spec.ny, spec.nz
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    xc = (-0.5 * nx + ix + 0.5) * spec.dx
    yc = (-0.5 * ny + iy + 0.5) * spec.dy
    img = np.asarray(x, np.float64).reshape(nz, ny, nx)
    out = []
    for ins in spec.inserts:
        m = (xc - ins.cx) ** 2 + (yc - ins.cy) ** 2 <= (frac * ins.r) ** 2
        out.append(img[:, m].mean())
    rr = np.hypot(xc, yc)
    ring = np.abs(rr - 0.3 * spec.cyl_r) <= 0.1 * spec.cyl_r
    out.append(img[:, ring].mean())
    return np.array(out)
