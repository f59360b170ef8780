"""The FP32 path's internal voxel order (in-plane tiles of tx x ty voxels for the gather
copy, the DROP accumulator, the hit counts and the stored columns) against the FP64 oracle.

The order changes only which addresses the kernels touch, not what they sum: every bar
here is the FP32 bar of the canonical order (relative L2 1e-6 for one DROP sweep, 1e-5
for whole runs at eps 1e-4).  Grids are ragged (nx, ny not multiples of the tile) so the
padded tiles of the last tile row and column are exercised.  The stored systems' order also
permutes each slice's offsets inside aligned groups of 32 (the slice windows' bank
swizzle); at 37 x 29 the 1x1, 2x2 and 8x2 tiles give slices of 1073, 1140 and 1200 voxels,
so the padding of a slice to a multiple of 32 is exercised as well.
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu_util import ntvs_module, oracle_run, rel_l2

pytestmark = pytest.mark.gpu

TILES = [(1, 1), (2, 2), (4, 4), (8, 2), (16, 16)]


def _system(nx=37, ny=29, nz=3, n_hist=20_000, seed=11):
    return synth.generate(synth.spec_scaled_3d(nx=nx, ny=ny, nz=nz, n_hist=n_hist, n_angles=30, n_blocks=4,
                                               seed=seed))


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("schedule", ["plain", "window", "pipeline"])
def test_tiled_sweep_matches_oracle(tile, schedule):
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_SCHED_PIPELINE, NTVS_SCHED_PLAIN, NTVS_SCHED_WINDOW
    code = {"plain": NTVS_SCHED_PLAIN, "window": NTVS_SCHED_WINDOW, "pipeline": NTVS_SCHED_PIPELINE}[schedule]
    s = _system()
    val = s.val.astype(np.float32)
    b = s.b.astype(np.float32)
    x0 = s.xstar * 0.9 + 0.05
    r = ntvs.Reconstructor(0)
    try:
        r.set_voxel_tile(*tile)
        r.load((s.spec.nx, s.spec.ny, s.spec.nz), s.row_ptr, s.col, val, b, n_blocks=4, schedule=code)
        st = r.stats()
        assert (st["voxel_tile_x"], st["voxel_tile_y"]) == tile
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
    assert rel_l2(got, want) < 1e-6
    np.testing.assert_allclose(res, ss, rtol=1e-4)


@pytest.mark.parametrize("tile", [(1, 1), (4, 4), (8, 2)])
@pytest.mark.parametrize("check", [0, 1])
def test_tiled_ntvs_run_matches_oracle(tile, check):
    """Whole cycles: the TV steps write the gather copy through the same map as the DROP
    update, and set_image fills it through the map too."""
    ntvs = ntvs_module()
    s = _system(nx=41, ny=35, nz=3, n_hist=30_000, seed=12)
    val = s.val.astype(np.float32)
    b = s.b.astype(np.float32)
    prm = oracle.Params(lam=0.5, N=3, alpha=0.75, seed=5, eps_tv=1e-4, tv_check=check, max_retries=8)
    K = 3
    r = ntvs.Reconstructor(0)
    try:
        r.set_voxel_tile(*tile)
        r.load((s.spec.nx, s.spec.ny, s.spec.nz), s.row_ptr, s.col, val, b, n_blocks=4)
        r.set_params(lam=prm.lam, N=prm.N, alpha=prm.alpha, beta0=prm.beta0, tv_check=prm.tv_check,
                     seed=prm.seed, eps_tv=prm.eps_tv, max_retries=prm.max_retries)
        r.set_image(s.xbar.astype(np.float32))
        r.run(K)
        x = r.get_image()
        ell, tries, acc = r.trace()
    finally:
        r.close()
    ref = oracle_run(s, val.astype(np.float64), b.astype(np.float64), prm, K, s.xbar.astype(np.float32))
    assert rel_l2(x, ref.x) <= 1e-5
    np.testing.assert_array_equal(ell, ref.ell_k)
    if check:
        np.testing.assert_array_equal(acc, ref.accepted.reshape(-1))


def test_tiled_delta16_storage_matches_oracle():
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_DELTA16
    s = _system(nx=45, ny=30, nz=2, seed=13)
    val = s.val.astype(np.float32)
    b = s.b.astype(np.float32)
    x0 = s.xstar * 0.8 + 0.1
    r = ntvs.Reconstructor(0)
    try:
        r.set_voxel_tile(4, 4)
        r.load((s.spec.nx, s.spec.ny, s.spec.nz), s.row_ptr, s.col, val, b, n_blocks=4, storage=NTVS_DELTA16)
        r.set_params(lam=0.9, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        got = r.get_image()
    finally:
        r.close()
    want, _ = oracle.drop_sweep(s.row_ptr, s.col, val.astype(np.float64), b.astype(np.float64), s.block_ptr(),
                                x0, 0.9)
    assert rel_l2(got, want) < 1e-6


def test_device_columns_are_not_rewritten():
    """With device-resident columns the tiled order goes to a buffer of the context's own."""
    ntvs = ntvs_module()
    import torch
    s = _system(n_hist=5000, seed=14)
    col = torch.from_numpy(s.col).cuda()
    dev = dict(row_ptr=torch.from_numpy(s.row_ptr).cuda(), val=torch.from_numpy(s.val.astype(np.float32)).cuda(),
               b=torch.from_numpy(s.b.astype(np.float32)).cuda())
    x0 = s.xstar * 0.9
    r = ntvs.Reconstructor(0, torch.cuda.current_stream().cuda_stream)
    try:
        r.set_voxel_tile(4, 4)
        r.load((s.spec.nx, s.spec.ny, s.spec.nz), dev["row_ptr"], col, dev["val"], dev["b"], n_blocks=4)
        r.set_params(lam=1.0, N=0, alpha=0.5)
        r.set_image(x0.astype(np.float32))
        r.drop_sweep()
        got = r.get_image()
    finally:
        r.close()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(col.cpu().numpy(), s.col)
    want, _ = oracle.drop_sweep(s.row_ptr, s.col, s.val.astype(np.float32).astype(np.float64),
                                s.b.astype(np.float32).astype(np.float64), s.block_ptr(),
                                x0.astype(np.float32).astype(np.float64), 1.0)
    assert rel_l2(got, want) < 1e-6


def test_tile_settings_and_errors():
    ntvs = ntvs_module()
    s = _system(nx=20, ny=18, nz=2, n_hist=2000, seed=15)
    r = ntvs.Reconstructor(0)
    try:
        for bad in [(0, 4), (3, 4), (4, 32), (-1, 1)]:
            with pytest.raises(ntvs.NtvsError):
                r.set_voxel_tile(*bad)
        # the FP64 path keeps the canonical order whatever was requested
        r.set_voxel_tile(4, 4)
        r.load((20, 18, 2), s.row_ptr, s.col, s.val, s.b, n_blocks=2)
        st = r.stats()
        assert (st["voxel_tile_x"], st["voxel_tile_y"]) == (1, 1)
        # out-of-range columns are still reported in the tiled order
        col = s.col.copy()
        col[len(col) // 2] = 20 * 18 * 2
        with pytest.raises(ntvs.NtvsError, match="column index"):
            r.load((20, 18, 2), s.row_ptr, col, s.val.astype(np.float32), s.b.astype(np.float32), n_blocks=2)
        col[len(col) // 2] = -1
        with pytest.raises(ntvs.NtvsError, match="column index"):
            r.load((20, 18, 2), s.row_ptr, col, s.val.astype(np.float32), s.b.astype(np.float32), n_blocks=2)
    finally:
        r.close()


def test_tiled_onthefly_rows_equal_canonical():
    """On-the-fly rows trace their voxel indices into the tiled order directly; the sweep
    equals the canonical-order sweep (ragged grid)."""
    ntvs = ntvs_module()
    spec = synth.spec_scaled_3d(nx=38, ny=30, nz=3, n_hist=12_000, n_angles=24, n_blocks=3, seed=16)
    pr = synth.generate_paths(spec)
    x0 = 0.9 * pr.xstar + 0.05
    outs = []
    for tile in ((1, 1), (4, 4), (8, 2)):
        r = ntvs.Reconstructor(0)
        try:
            r.set_voxel_tile(*tile)
            r.load_paths((spec.nx, spec.ny, spec.nz), (spec.dx, spec.dy, spec.dz), pr.paths,
                         pr.b.astype(np.float32), n_blocks=3, n_seg=spec.n_seg, min_len=spec.min_len)
            st = r.stats()
            assert (st["voxel_tile_x"], st["voxel_tile_y"]) == tile
            r.set_params(lam=0.8, N=2, alpha=0.75, seed=3, eps_tv=1e-4)
            r.set_image(x0)
            r.run(2)
            outs.append(r.get_image())
        finally:
            r.close()
    for o in outs[1:]:
        assert rel_l2(o, outs[0]) <= 1e-6
