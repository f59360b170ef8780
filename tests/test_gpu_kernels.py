"""GPU parity of the single steps of the hot path against the FP64 oracle (through the C ABI).

Tolerances: the FP64 path differs from the oracle only in summation order (1e-12
relative); the FP32 path computes each voxel of the TV gradient with ~10 float
operations of O(1) terms (absolute error ~1e-6) and each DROP update with ~300-term
float dot products (relative 1e-6); the bounds below leave a factor of ~10.
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu_util import empty_system, load, ntvs_module, rel_l2

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (7, 1, 1), (1, 9, 1), (33, 17, 1), (40, 37, 5), (64, 48, 3), (200, 200, 16)]


def _image(shape, seed, kind):
    V = int(np.prod(shape))
    rng = np.random.default_rng(seed)
    if kind == "random":
        return rng.uniform(0.0, 2.0, size=V)
    xs, _, _ = synth.phantom(synth.spec_scaled_3d(nx=shape[0], ny=shape[1], nz=shape[2]))
    return xs + 0.01 * rng.normal(size=V)   # piecewise constant + noise


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["random", "phantom"])
def test_tv_gradient_and_value(dtype, shape, kind):
    ntvs = ntvs_module()
    if kind == "phantom" and shape[0] != shape[1]:
        pytest.skip("phantom needs a square slice")
    x = _image(shape, 11, kind).astype(dtype)
    x64 = x.astype(np.float64)
    eps = 1e-8
    r = empty_system(ntvs, shape) if dtype == np.float64 else _empty32(ntvs, shape)
    try:
        r.set_params(lam=1.0, N=1, alpha=0.5, eps_tv=eps)
        r.set_image(x)
        g, gn = r.tv_gradient(np.float64)
        tv = r.tv()
    finally:
        r.close()
    g_ref = oracle.tv_grad(x64, shape, eps)
    scale = max(np.abs(g_ref).max(), 1.0)
    if dtype == np.float64:
        np.testing.assert_allclose(g, g_ref, rtol=1e-11, atol=1e-11 * scale)
        assert gn == pytest.approx(np.linalg.norm(g_ref), rel=1e-12)
    else:
        np.testing.assert_allclose(g, g_ref, rtol=1e-4, atol=2e-5 * scale)
        assert gn == pytest.approx(np.linalg.norm(g_ref), rel=1e-5)
    assert tv == pytest.approx(oracle.tv(x64, shape), rel=1e-12, abs=1e-12)


def _empty32(ntvs, shape):
    r = ntvs.Reconstructor(0)
    r.load(shape, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(0, np.float32))
    return r


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_perturb_step_closed_form(dtype):
    ntvs = ntvs_module()
    shape = (31, 29, 3)
    x = _image(shape, 3, "random").astype(dtype)
    r = empty_system(ntvs, shape) if dtype == np.float64 else _empty32(ntvs, shape)
    try:
        r.set_params(lam=1.0, N=1, alpha=0.5, eps_tv=1e-8)
        r.set_image(x)
        r.perturb(0.37)
        got = r.get_image()
    finally:
        r.close()
    x64 = x.astype(np.float64)
    g = oracle.tv_grad(x64, shape, 1e-8)
    want = x64 - 0.37 * g / np.linalg.norm(g)
    tol = 1e-13 if dtype == np.float64 else 2e-7
    np.testing.assert_allclose(got, want, rtol=0, atol=tol * max(1.0, np.abs(want).max()))


def test_perturb_checked_decisions():
    ntvs = ntvs_module()
    shape = (5, 5, 1)
    x = np.zeros(25)
    x[12] = 0.05
    r = empty_system(ntvs, shape)
    try:
        r.set_params(lam=1.0, N=1, alpha=0.5, eps_tv=1e-8)
        r.set_image(x)
        acc, px, pz = r.perturb_checked(1.0)     # overshoots the spike: rejected
        assert not acc and pz > px
        np.testing.assert_array_equal(r.get_image(), x)
        acc2, px2, pz2 = r.perturb_checked(1e-3)   # small step lowers TV: accepted
        assert acc2 and pz2 <= px2
        g = oracle.tv_grad(x, shape, 1e-8)
        np.testing.assert_allclose(r.get_image(), x - 1e-3 * g / np.linalg.norm(g), atol=1e-15)
        assert px == pytest.approx(oracle.tv(x, shape), rel=1e-14)
    finally:
        r.close()


def _small_system(curved=True, n_hist=6000, nx=24, nz=3, blocks=3, seed=5):
    return synth.generate(synth.spec_scaled_3d(nx=nx, ny=nx, nz=nz, n_hist=n_hist, n_angles=30, n_blocks=blocks,
                                               seed=seed, curved=curved))


def test_gradient_follows_single_drop_blocks():
    """The FP32 gradient reads split FP32 copies of x that only the last block of a sweep
    writes; after any single block they are refreshed before the gradient."""
    ntvs = ntvs_module()
    s = _small_system(n_hist=4000)
    shape = (s.spec.nx, s.spec.ny, s.spec.nz)
    r, _, _ = load(ntvs, s, np.float32)
    try:
        r.set_params(lam=0.9, N=0, alpha=0.5, eps_tv=1e-6)
        r.set_image(s.xbar.astype(np.float32))
        for t in (0, 2, 1):
            r.drop_block(t)
            x = r.get_image()
            g, _ = r.tv_gradient(np.float64)
            g_ref = oracle.tv_grad(x, shape, 1e-6)
            scale = max(np.abs(g_ref).max(), 1.0)
            np.testing.assert_allclose(g, g_ref, rtol=1e-4, atol=2e-5 * scale)
    finally:
        r.close()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("curved", [False, True])
def test_drop_block_and_sweep(dtype, curved):
    ntvs = ntvs_module()
    s = _small_system(curved)
    r, val64, b64 = load(ntvs, s, dtype)
    bp = s.block_ptr()
    x0 = s.xbar.astype(dtype).astype(np.float64)
    try:
        r.set_params(lam=0.9, N=0, alpha=0.5)
        r.set_image(x0.astype(dtype))
        r.drop_block(1)
        got1 = r.get_image()
        res1 = r.block_resid()[1]
        r.set_image(x0.astype(dtype))
        r.drop_sweep()
        got = r.get_image()
        res = r.block_resid()
    finally:
        r.close()
    want1, ss1 = oracle.drop_block(s.row_ptr, s.col, val64, b64, bp[1], bp[2], x0, 0.9)
    want, ss = oracle.drop_sweep(s.row_ptr, s.col, val64, b64, bp, x0, 0.9)
    tol = 1e-12 if dtype == np.float64 else 1e-6
    assert rel_l2(got1, want1) < tol
    assert rel_l2(got, want) < tol
    assert res1 == pytest.approx(ss1, rel=1e-10 if dtype == np.float64 else 1e-4)
    np.testing.assert_allclose(res, ss, rtol=1e-10 if dtype == np.float64 else 1e-4)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("schedule", ["plain", "window", "pipeline", "auto"])
def test_drop_schedules_match_oracle(dtype, schedule):
    """Every DROP kernel schedule (stored-order rows with global reductions; rows grouped by
    home z-slice with a shared-memory window; the same fed by TMA bulk copies) gives the
    oracle's sweep."""
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import (NTVS_SCHED_AUTO, NTVS_SCHED_PIPELINE, NTVS_SCHED_PLAIN,
                                             NTVS_SCHED_WINDOW)
    code = {"plain": NTVS_SCHED_PLAIN, "window": NTVS_SCHED_WINDOW, "pipeline": NTVS_SCHED_PIPELINE,
            "auto": NTVS_SCHED_AUTO}[schedule]
    s = synth.generate(synth.spec_scaled_3d(nx=40, ny=40, nz=5, n_hist=30_000, n_angles=36, n_blocks=4, seed=8))
    val = s.val.astype(dtype)
    b = s.b.astype(dtype)
    x0 = s.xstar * 0.9 + 0.05
    r = ntvs.Reconstructor(0)
    try:
        r.load((40, 40, 5), s.row_ptr, s.col, val, b, n_blocks=4, schedule=code)
        st = r.stats()
        if schedule == "auto":
            assert st["drop_schedule"] == NTVS_SCHED_WINDOW   # rows come in runs of one slice
        else:
            assert st["drop_schedule"] == code
        r.set_params(lam=1.1, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        got = r.get_image()
        res = r.block_resid()
    finally:
        r.close()
    want, ss = oracle.drop_sweep(s.row_ptr, s.col, val.astype(np.float64), b.astype(np.float64), s.block_ptr(),
                                 x0, 1.1)
    assert rel_l2(got, want) < (1e-12 if dtype == np.float64 else 1e-6)
    np.testing.assert_allclose(res, ss, rtol=1e-10 if dtype == np.float64 else 1e-4)


@pytest.mark.parametrize("tile", [(4, 4), (1, 1)])
@pytest.mark.parametrize("parts", ["1", "2", "3", "7", "empty_blocks"])
def test_staged_load_matches_oracle(parts, tile):
    """FP32 values from host arrays reach the device through a ring of three block-sized
    slots, packed into {column, value} pairs block by block (the copy of block t + 3 waits
    for block t).  Every ring depth (1, 2 or 3 slots in use, and more blocks than slots),
    empty blocks (no copy into their slot), the tiled and the canonical voxel order: the
    sweep is the oracle's, and the loaded rows project like the oracle's."""
    ntvs = ntvs_module()
    s = synth.generate(synth.spec_scaled_3d(nx=40, ny=40, nz=5, n_hist=30_000, n_angles=36, n_blocks=4, seed=8))
    M = s.M
    if parts == "empty_blocks":
        bp = np.array([0, 0, M // 3, M // 3, M // 3 + 5, M, M], dtype=np.int64)
    else:
        nb = int(parts)
        bp = np.array([(M * t) // nb for t in range(nb + 1)], dtype=np.int64)
    val = s.val.astype(np.float32)
    b = s.b.astype(np.float32)
    x0 = s.xstar * 0.9 + 0.05
    r = ntvs.Reconstructor(0).set_voxel_tile(*tile)
    try:
        r.load((40, 40, 5), s.row_ptr, s.col, val, b, block_ptr=bp)
        r.set_params(lam=1.1, N=0, alpha=0.5)
        proj = r.forward_project(x0)
        r.set_image(x0)
        r.drop_sweep()
        got = r.get_image()
        res = r.block_resid()
    finally:
        r.close()
    val64, b64 = val.astype(np.float64), b.astype(np.float64)
    want, ss = oracle.drop_sweep(s.row_ptr, s.col, val64, b64, bp, x0, 1.1)
    assert rel_l2(got, want) < 1e-6
    np.testing.assert_allclose(res, ss, rtol=1e-4, atol=1e-12)
    ref = np.array([val64[s.row_ptr[i]:s.row_ptr[i + 1]] @ x0[s.col[s.row_ptr[i]:s.row_ptr[i + 1]]] for i in range(M)])
    np.testing.assert_allclose(proj, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def test_pipeline_stages_stay_inside_exact_sized_arrays():
    """The pipelined schedule copies stages of whole rows with 16-byte aligned bulk copies;
    with BF16 values and int32 columns (8-entry alignment) and nnz not a multiple of 8, the
    last rows must not be copied past the end of the caller's exact-sized device arrays
    (the library refuses a plan that would, and such rows are read from global memory);
    the sweep still equals the oracle's."""
    ntvs = ntvs_module()
    import torch
    from paper_1803_01112_gb300._ffi import NTVS_SCHED_PIPELINE
    s = synth.generate(synth.spec_scaled_3d(nx=40, ny=40, nz=5, n_hist=30_000, n_angles=36, n_blocks=4, seed=8))
    M = s.M
    while int(s.row_ptr[M]) % 8 == 0:   # drop rows from the end until nnz is not a multiple of 8
        M -= 1
    nnz = int(s.row_ptr[M])
    rp = torch.from_numpy(s.row_ptr[:M + 1].copy()).cuda()
    col = torch.from_numpy(s.col[:nnz].copy()).cuda()
    val = torch.from_numpy(s.val[:nnz].astype(np.float32)).to(torch.bfloat16).cuda()
    b = torch.from_numpy(s.b[:M].astype(np.float32)).cuda()
    assert col.numel() == nnz and nnz % 8 != 0
    x0 = s.xstar * 0.9 + 0.05
    r = ntvs.Reconstructor(0)
    try:
        r.load((40, 40, 5), rp, col, val, b, n_blocks=4, schedule=NTVS_SCHED_PIPELINE)
        assert r.stats()["drop_schedule"] == NTVS_SCHED_PIPELINE
        r.set_params(lam=1.1, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        got = r.get_image()
    finally:
        r.close()
    v64 = val.float().cpu().numpy().astype(np.float64)
    bp = synth.block_partition(M, 4)
    want, _ = oracle.drop_sweep(s.row_ptr[:M + 1], s.col[:nnz], v64, s.b[:M].astype(np.float32).astype(np.float64),
                                bp, x0, 1.1)
    assert rel_l2(got, want) < 1e-6


def test_fixed_point_window_follows_its_bound():
    """The FP32 windowed schedule accumulates its slice window in int32 fixed point with a
    per-block scale bounded by the previous sweep's largest |residual| / ||a||^2; rows above
    the bound (here: every row, after the image jumps tenfold) scatter with global
    reductions, and the next sweep's bound covers them again.  Every sweep equals the
    oracle's."""
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_SCHED_WINDOW
    s = synth.generate(synth.spec_scaled_3d(nx=40, ny=40, nz=5, n_hist=30_000, n_angles=36, n_blocks=4, seed=8))
    val, b = s.val.astype(np.float32), s.b.astype(np.float32)
    val64, b64 = val.astype(np.float64), b.astype(np.float64)
    r = ntvs.Reconstructor(0)
    try:
        r.load((40, 40, 5), s.row_ptr, s.col, val, b, n_blocks=4, schedule=NTVS_SCHED_WINDOW)
        assert r.stats()["drop_schedule"] == NTVS_SCHED_WINDOW
        r.set_params(lam=0.9, N=0, alpha=0.5)
        for x0 in (s.xbar, 10.0 * s.xbar, 10.0 * s.xbar, -3.0 * s.xstar):
            r.set_image(x0)
            r.drop_sweep()
            got = r.get_image()
            want, ss = oracle.drop_sweep(s.row_ptr, s.col, val64, b64, s.block_ptr(), x0, 0.9)
            assert rel_l2(got, want) < 1e-6
            np.testing.assert_allclose(r.block_resid(), ss, rtol=1e-4)
    finally:
        r.close()


def test_window_schedule_on_rows_without_slice_order():
    """Forcing the windowed schedule on rows in random order is slower but still exact."""
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_SCHED_AUTO, NTVS_SCHED_PIPELINE, NTVS_SCHED_WINDOW
    s = synth.generate(synth.spec_scaled_3d(nx=32, ny=32, nz=4, n_hist=8_000, n_angles=20, n_blocks=3, seed=4))
    perm = np.random.default_rng(0).permutation(s.M)
    lens = np.diff(s.row_ptr)[perm]
    rp = np.zeros(s.M + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    col = np.concatenate([s.col[s.row_ptr[i]:s.row_ptr[i + 1]] for i in perm]).astype(np.int32)
    val = np.concatenate([s.val[s.row_ptr[i]:s.row_ptr[i + 1]] for i in perm]).astype(np.float32)
    b = s.b[perm].astype(np.float32)
    x0 = s.xbar
    for code in (NTVS_SCHED_WINDOW, NTVS_SCHED_PIPELINE, NTVS_SCHED_AUTO):
        r = ntvs.Reconstructor(0)
        try:
            r.load((32, 32, 4), rp, col, val, b, n_blocks=3, schedule=code)
            if code == NTVS_SCHED_AUTO:
                assert r.stats()["drop_schedule"] not in (NTVS_SCHED_WINDOW, NTVS_SCHED_PIPELINE)   # plain
            r.set_params(lam=0.8, N=0, alpha=0.5)
            r.set_image(x0)
            r.drop_sweep()
            got = r.get_image()
        finally:
            r.close()
        want, _ = oracle.drop_sweep(rp, col, val.astype(np.float64), b.astype(np.float64),
                                    synth.block_partition(s.M, 3), x0, 0.8)
        assert rel_l2(got, want) < 1e-6


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_pipeline_rows_longer_than_a_ring_slot(dtype):
    """Rows with more entries than a shared-memory ring slot are read from global memory;
    short and long rows, empty rows and stored zeros mixed, several home slices."""
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_SCHED_PIPELINE
    rng = np.random.default_rng(21)
    nx, ny, nz = 64, 64, 3
    V = nx * ny * nz
    M = 3000
    lens = rng.integers(20, 300, size=M)
    lens[::50] = rng.integers(2100, 3900, size=lens[::50].size)   # longer than a slot
    lens[7::97] = 0
    rows = []
    for k, n in enumerate(lens):
        z = (k * 3) // M                                              # rows come slice by slice
        pool = np.arange(z * nx * ny, (z + 1) * nx * ny)
        rows.append(np.sort(rng.choice(pool, size=n, replace=False)))
    rp = np.zeros(M + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    col = np.concatenate(rows).astype(np.int32)
    val = rng.uniform(0.1, 1.2, size=col.size).astype(dtype)
    val[::31] = 0
    b = rng.uniform(5, 80, size=M).astype(dtype)
    x0 = rng.uniform(0.5, 1.5, size=V)
    r = ntvs.Reconstructor(0)
    try:
        r.load((nx, ny, nz), rp, col, val, b, n_blocks=4, schedule=NTVS_SCHED_PIPELINE)
        r.set_params(lam=0.9, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        got = r.get_image()
    finally:
        r.close()
    want, _ = oracle.drop_sweep(rp, col, val.astype(np.float64), b.astype(np.float64),
                                synth.block_partition(M, 4), x0, 0.9)
    assert rel_l2(got, want) < (1e-12 if dtype == np.float64 else 1e-6)


@pytest.mark.parametrize("lanes_case", ["short", "medium", "long"])
def test_drop_row_lengths_cover_every_lane_shape(lanes_case):
    # mean row length selects 4/8/16/32 lanes per row; rows beyond the register-held
    # chunks take the re-read tail path
    ntvs = ntvs_module()
    rng = np.random.default_rng(9)
    V = 5000
    per = {"short": (1, 20), "medium": (30, 110), "long": (200, 700)}[lanes_case]
    M = 3000
    lens = rng.integers(per[0], per[1], size=M)
    lens[::97] = 0                      # some empty rows
    rows = [np.sort(rng.choice(V, size=n, replace=False)) for n in lens]
    rp = np.zeros(M + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    col = np.concatenate(rows).astype(np.int32)
    val = rng.uniform(0.1, 1.2, size=col.size)
    val[::13] = 0.0                     # stored zeros do not count in s_j
    b = rng.uniform(5, 50, size=M)
    x0 = rng.uniform(0.5, 1.5, size=V)
    bp = np.array([0, 1000, 1001, 2500, 3000], np.int64)
    r = ntvs.Reconstructor(0)
    try:
        r.load((50, 100, 1), rp, col, val, b, block_ptr=bp)
        r.set_params(lam=1.3, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        got = r.get_image()
    finally:
        r.close()
    want, _ = oracle.drop_sweep(rp, col, val, b, bp, x0, 1.3)
    assert rel_l2(got, want) < 1e-12


def test_degenerate_systems():
    ntvs = ntvs_module()
    # more blocks than rows (empty blocks), a zero-norm row, a voxel hit by nothing, V = 1 grid
    rp = np.array([0, 1, 1, 3], np.int64)
    col = np.array([0, 1, 2], np.int32)
    val = np.array([1.0, 0.0, 2.0])
    b = np.array([3.0, 1.0, 4.0])
    x0 = np.array([0.0, 5.0, 0.0, -1.0])
    r = ntvs.Reconstructor(0)
    try:
        r.load((4, 1, 1), rp, col, val, b, n_blocks=7)
        r.set_params(lam=1.0, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        got = r.get_image()
    finally:
        r.close()
    want, _ = oracle.drop_sweep(rp, col, val, b, synth.block_partition(3, 7), x0, 1.0)
    np.testing.assert_allclose(got, want, atol=1e-15)
    r = ntvs.Reconstructor(0)
    try:
        r.load((1, 1, 1), np.array([0, 1], np.int64), np.array([0], np.int32), np.array([2.0]), np.array([3.0]))
        r.set_params(lam=1.0, N=2, alpha=0.5)
        r.set_image(np.array([0.25]))
        r.run(3)
        assert r.get_image()[0] == pytest.approx(1.5, abs=1e-15)   # exact projection, TV steps are zero
        assert r.tv() == 0.0
    finally:
        r.close()


def test_validation_errors():
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_ERR_ARG, NTVS_ERR_CSR, NTVS_ERR_STATE
    r = ntvs.Reconstructor(0)
    try:
        with pytest.raises(ntvs.NtvsError) as e:
            r.run(1)
        assert e.value.code == NTVS_ERR_STATE
        good = dict(row_ptr=np.array([0, 2, 3], np.int64), col=np.array([0, 1, 3], np.int32),
                    val=np.array([1.0, 1.0, 1.0]), b=np.array([1.0, 2.0]))
        bad_cases = [dict(row_ptr=np.array([0, 2, 1], np.int64), col=np.array([0, 1], np.int32),
                          val=np.array([1.0, 1.0]), b=np.array([1.0, 2.0])),
                     dict(good, col=np.array([0, 1, 4], np.int32)),
                     dict(good, col=np.array([0, -1, 3], np.int32)),
                     dict(good, val=np.array([1.0, np.nan, 1.0])),
                     dict(good, b=np.array([1.0, np.inf]))]
        for case in bad_cases:
            with pytest.raises(ntvs.NtvsError) as e:
                r.load((2, 2, 1), case["row_ptr"], case["col"], case["val"], case["b"])
            assert e.value.code == NTVS_ERR_CSR
        r.load((2, 2, 1), **good)
        for kw in (dict(alpha=1.0), dict(alpha=0.0), dict(N=-1), dict(beta0=-1.0), dict(tv_check=True, max_retries=0)):
            with pytest.raises(ntvs.NtvsError) as e:
                r.set_params(**dict(dict(lam=1.0, N=1, alpha=0.5), **kw))
            assert e.value.code == NTVS_ERR_ARG
        with pytest.raises(ntvs.NtvsError) as e:
            r.drop_block(5)
        assert e.value.code == NTVS_ERR_ARG
        with pytest.raises(ntvs.NtvsError) as e:
            r.load((2, 2, 1), **good, block_ptr=np.array([0, 3, 2], np.int64))
        assert e.value.code == NTVS_ERR_ARG
    finally:
        r.close()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_device_pointers_match_host(dtype):
    ntvs = ntvs_module()
    import torch
    s = _small_system(n_hist=3000)
    r_host, val64, b64 = load(ntvs, s, dtype)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    dev = dict(row_ptr=torch.from_numpy(s.row_ptr).cuda(), col=torch.from_numpy(s.col).cuda(),
               val=torch.from_numpy(s.val.astype(dtype)).cuda(), b=torch.from_numpy(s.b.astype(dtype)).cuda())
    r_dev = ntvs.Reconstructor(0, torch.cuda.current_stream().cuda_stream)
    try:
        r_dev.load((s.spec.nx, s.spec.ny, s.spec.nz), dev["row_ptr"], dev["col"], dev["val"], dev["b"],
                   n_blocks=s.spec.n_blocks)
        outs = []
        for r in (r_host, r_dev):
            r.set_params(lam=0.7, N=2, alpha=0.75, seed=3)
            r.set_image(torch.from_numpy(s.xbar.astype(dtype)).cuda() if r is r_dev else s.xbar.astype(dtype))
            r.run(2)
            out = torch.empty(s.spec.V, dtype=tdt, device="cuda")
            ntvs.ntvs_get_image(r.handle, out)
            r.sync()
            outs.append(out.cpu().numpy())
        # scatter atomics make the summation order (not the result class) run dependent
        tol = 1e-12 if dtype == np.float64 else 1e-6
        np.testing.assert_allclose(outs[0], outs[1], rtol=tol, atol=tol)
    finally:
        r_host.close()
        r_dev.close()


@pytest.mark.parametrize("storage", ["csr32", "delta16"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_forward_project_equals_the_stored_rows(storage, dtype):
    """ntvs_forward_project gives A x of the loaded rows (the dot products of the DROP sweep)."""
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_CSR32, NTVS_DELTA16
    s = synth.generate(synth.spec_scaled_3d(nx=40, ny=40, nz=5, n_hist=20_000, n_angles=36, n_blocks=4, seed=6))
    val = s.val.astype(dtype)
    x = s.xstar * 0.8 + 0.1
    r = ntvs.Reconstructor(0)
    try:
        r.load((40, 40, 5), s.row_ptr, s.col, val, s.b.astype(dtype), n_blocks=4,
               storage={"csr32": NTVS_CSR32, "delta16": NTVS_DELTA16}[storage])
        r.set_image(s.xbar)
        got = r.forward_project(x)
        got32 = r.forward_project(x.astype(np.float32), out=np.empty(s.M, np.float32))
        assert np.array_equal(r.get_image(), s.xbar)   # the current image is untouched
    finally:
        r.close()
    rows = np.repeat(np.arange(s.M), np.diff(s.row_ptr))
    want = np.bincount(rows, weights=val.astype(np.float64) * x[s.col], minlength=s.M)
    tol = 1e-13 if dtype == np.float64 else 2e-6
    np.testing.assert_allclose(got, want, rtol=tol, atol=tol * np.abs(want).max())
    np.testing.assert_allclose(got32, want, rtol=2e-6, atol=2e-6 * np.abs(want).max())
