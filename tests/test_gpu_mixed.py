"""Mixed precision on the GPU: half-precision path lengths (FP16 / BF16) and DELTA16 voxel
indices, FP32 accumulation, FP64 TV and residual reductions.

* DELTA16 is lossless: with FP32 values it reproduces the CSR32 sweep to FP32 rounding, for
  every schedule that reads it, including rows with escaped (large) column jumps.
* Half-precision values: the GPU run matches the oracle on the *stored* (quantized) system
  to the FP32 bar; against the oracle on the FP64 system, the mean RSP in every insert ROI
  and in the background stays within 1e-3 (relative; absolute where |mean| < 0.05).
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu_util import ntvs_module, oracle_run, quantize, rel_l2, roi_means

pytestmark = pytest.mark.gpu


def _sweep(ntvs, shape, rp, col, val, b, nb, x0, lam, storage, schedule):
    r = ntvs.Reconstructor(0)
    try:
        r.load(shape, rp, col, val, b, n_blocks=nb, storage=storage, schedule=schedule)
        st = r.stats()
        r.set_params(lam=lam, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        return r.get_image(), st
    finally:
        r.close()


@pytest.mark.parametrize("schedule", ["plain", "window", "pipeline"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_delta16_is_lossless(schedule, dtype):
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_DELTA16, NTVS_SCHED_PIPELINE, NTVS_SCHED_PLAIN, NTVS_SCHED_WINDOW
    sched = {"plain": NTVS_SCHED_PLAIN, "window": NTVS_SCHED_WINDOW, "pipeline": NTVS_SCHED_PIPELINE}[schedule]
    s = synth.generate(synth.spec_scaled_3d(nx=40, ny=40, nz=6, n_hist=30_000, n_angles=36, n_blocks=4, seed=12))
    val, b = s.val.astype(dtype), s.b.astype(dtype)
    x0 = s.xstar * 0.9 + 0.05
    got, st = _sweep(ntvs, (40, 40, 6), s.row_ptr, s.col, val, b, 4, x0, 1.2, NTVS_DELTA16, sched)
    assert st["drop_schedule"] == sched
    want, _ = oracle.drop_sweep(s.row_ptr, s.col, val.astype(np.float64), b.astype(np.float64), s.block_ptr(), x0, 1.2)
    assert rel_l2(got, want) < (1e-12 if dtype == np.float64 else 1e-6)


def test_delta16_with_many_escaped_jumps():
    """Random rows: most column differences exceed int16 and go to the exception lists."""
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_DELTA16, NTVS_SCHED_PLAIN
    rng = np.random.default_rng(3)
    shape = (250, 250, 3)
    V = int(np.prod(shape))
    M = 4000
    lens = rng.integers(0, 90, size=M)
    rp = np.zeros(M + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    col = np.concatenate([rng.choice(V, size=n, replace=False) for n in lens]).astype(np.int32)
    val = rng.uniform(0.1, 1.0, size=col.size)
    b = rng.uniform(5, 40, size=M)
    x0 = rng.uniform(0.5, 1.5, size=V)
    got, _ = _sweep(ntvs, shape, rp, col, val, b, 3, x0, 0.9, NTVS_DELTA16, NTVS_SCHED_PLAIN)
    want, _ = oracle.drop_sweep(rp, col, val, b, synth.block_partition(M, 3), x0, 0.9)
    assert rel_l2(got, want) < 1e-12


@pytest.mark.parametrize("schedule", ["plain", "window", "pipeline"])
@pytest.mark.parametrize("kind", ["fp16", "bf16"])
def test_delta16_words_match_oracle_on_stored_system(schedule, kind):
    """DELTA16 with 16-bit values keeps each entry as one 32-bit word (offset in the low
    half, the value's bits in the high half).  Every schedule that reads the words, the TMA
    pipeline's single-array ring included, gives the oracle's sweep on the quantized system,
    and the projection of the stored rows equals the oracle's."""
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_DELTA16, NTVS_SCHED_PIPELINE, NTVS_SCHED_PLAIN, NTVS_SCHED_WINDOW
    sched = {"plain": NTVS_SCHED_PLAIN, "window": NTVS_SCHED_WINDOW, "pipeline": NTVS_SCHED_PIPELINE}[schedule]
    s = synth.generate(synth.spec_scaled_3d(nx=40, ny=40, nz=6, n_hist=30_000, n_angles=36, n_blocks=4, seed=12))
    vq, v64 = quantize(s.val, kind)
    b = s.b.astype(np.float32)
    x0 = s.xstar * 0.9 + 0.05
    r = ntvs.Reconstructor(0)
    try:
        r.load((40, 40, 6), s.row_ptr, s.col, vq, b, n_blocks=4, storage=NTVS_DELTA16, schedule=sched)
        st = r.stats()
        proj = r.forward_project(x0)
        r.set_params(lam=1.2, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        got = r.get_image()
    finally:
        r.close()
    assert st["drop_schedule"] == sched
    want, _ = oracle.drop_sweep(s.row_ptr, s.col, v64, b.astype(np.float64), s.block_ptr(), x0, 1.2)
    assert rel_l2(got, want) < 1e-6
    M = s.M
    ref = np.array([v64[s.row_ptr[i]:s.row_ptr[i + 1]] @ x0[s.col[s.row_ptr[i]:s.row_ptr[i + 1]]] for i in range(M)])
    np.testing.assert_allclose(proj, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


@pytest.mark.parametrize("schedule", ["plain", "window", "pipeline"])
def test_delta16_chunks_mix_packed_and_escaped(schedule):
    """Rows of slowly varying columns with rare far jumps: rows without a jump are narrow (one
    base), in the others most 32-entry chunks are stored as base + 16-bit offsets and the
    chunks holding a jump as full columns.  The count of escaped chunks follows the
    format's definition exactly, and every schedule gives the oracle's sweep."""
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_DELTA16, NTVS_SCHED_PIPELINE, NTVS_SCHED_PLAIN, NTVS_SCHED_WINDOW
    sched = {"plain": NTVS_SCHED_PLAIN, "window": NTVS_SCHED_WINDOW, "pipeline": NTVS_SCHED_PIPELINE}[schedule]
    rng = np.random.default_rng(11)
    shape = (120, 120, 8)   # V = 115200 > 65535; an FP64 slice window of 115 KB
    V = int(np.prod(shape))
    M = 3000
    lens = rng.integers(1, 140, size=M)
    rp = np.zeros(M + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    cols = []
    for i, n in enumerate(lens):   # a walk of small steps inside one slice, a far jump now and then
        z = (i * 8) // M
        c = z * 14400 + int(rng.integers(0, 9000)) + np.cumsum(rng.integers(1, 40, size=n))
        jump = rng.random(n) < 0.01
        c = np.where(jump, rng.integers(0, V, size=n), c % V)
        cols.append(c)
    col = np.concatenate(cols).astype(np.int32)
    val = rng.uniform(0.1, 1.0, size=col.size)
    b = rng.uniform(5, 40, size=M)
    x0 = rng.uniform(0.5, 1.5, size=V)
    # a row whose columns span at most 65535 is narrow (one base, no escape); in the other
    # rows, chunks of 32 entries from the row's first entry are escaped when their columns
    # span more than 65535
    spans = [np.ptp(c[k:k + 32]) for c in cols if np.ptp(c) > 65535 for k in range(0, len(c), 32)]
    want_esc = int(sum(sp > 65535 for sp in spans))
    n_chunks = sum((len(c) + 31) // 32 for c in cols)
    n_narrow = sum(np.ptp(c) <= 65535 for c in cols)
    assert 0 < n_narrow < M   # both kinds of rows occur
    r = ntvs.Reconstructor(0)
    try:
        r.set_voxel_tile(1, 1)
        r.load(shape, rp, col, val, b, n_blocks=3, storage=NTVS_DELTA16, schedule=sched)
        st = r.stats()
        r.set_params(lam=0.9, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        got = r.get_image()
    finally:
        r.close()
    assert st["drop_schedule"] == sched
    assert st["n_escaped"] == want_esc and 0 < want_esc < n_chunks // 2
    want, _ = oracle.drop_sweep(rp, col, val, b, synth.block_partition(M, 3), x0, 0.9)
    assert rel_l2(got, want) < 1e-12


@pytest.mark.parametrize("kind", ["fp16", "bf16"])
@pytest.mark.parametrize("storage", ["csr32", "delta16"])
def test_half_values_match_oracle_on_stored_system(kind, storage):
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_CSR32, NTVS_DELTA16
    spec = synth.spec_scaled_3d(nx=48, ny=48, nz=4, n_hist=60_000, n_angles=60, n_blocks=5)
    s = synth.generate(spec)
    vq, v64 = quantize(s.val, kind)
    b32 = s.b.astype(np.float32)
    prm = oracle.Params(lam=0.3, N=3, alpha=0.75, seed=2, eps_tv=1e-4)
    r = ntvs.Reconstructor(0)
    try:
        r.load((48, 48, 4), s.row_ptr, s.col, vq, b32, n_blocks=5,
               storage={"csr32": NTVS_CSR32, "delta16": NTVS_DELTA16}[storage])
        r.set_params(lam=prm.lam, N=prm.N, alpha=prm.alpha, seed=prm.seed, eps_tv=prm.eps_tv)
        r.set_image(s.xbar)
        r.run(6)
        x = r.get_image()
    finally:
        r.close()
    ref = oracle_run(s, v64, b32.astype(np.float64), prm, 6, s.xbar)
    assert rel_l2(x, ref.x) <= 1e-5


@pytest.mark.parametrize("kind", ["fp16", "bf16"])
def test_slice_2d_mixed_roi_error(kind):
    """The 2D 32x32 slice workload with half-precision lengths and DELTA16 indices: per-ROI
    mean RSP vs the FP64 oracle on the FP64 system, after 4 cycles (lambda = 1e-3) and after
    a strong run (lambda = 0.5)."""
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_DELTA16
    spec = synth.spec_slice_2d()
    s = synth.generate(spec)
    vq, _ = quantize(s.val, kind)
    b32 = s.b.astype(np.float32)
    for lam in (1e-3, 0.5):
        prm = oracle.Params(lam=lam, N=3, alpha=0.75, seed=1)
        r = ntvs.Reconstructor(0)
        try:
            r.load((32, 32, 1), s.row_ptr, s.col, vq, b32, n_blocks=10, storage=NTVS_DELTA16)
            r.set_params(lam=lam, N=3, alpha=0.75, seed=1)
            r.set_image(s.xbar)
            r.run(4)
            x = r.get_image()
        finally:
            r.close()
        ref = oracle_run(s, s.val, s.b, prm, 4, s.xbar)
        g, w = roi_means(x, spec), roi_means(ref.x, spec)
        err = np.where(np.abs(w) < 0.05, np.abs(g - w), np.abs(g - w) / np.abs(w))
        assert np.all(err <= 1e-3), f"ROI errors {err}"
