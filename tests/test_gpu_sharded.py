"""Row-sharded DROP through the C ABI (Sec. III-D: all rows of a block see the same x, so
a block's rows may be split over GPUs, their deltas summed and applied with the global hit
counts).  The paper runs on one GPU; the split is the library's.

On one GPU: two contexts each hold half of every block's rows; their partial deltas
(ntvs_drop_block_partial) are summed on the device and applied by both
(ntvs_apply_delta) with the summed hit counts; the image equals the oracle's sweep of the
whole system.  The all-reduce callback mode (ntvs_set_allreduce) runs with one rank, and
with two processes sharing the GPU whose collectives go through gloo on the host (no GPU
kernel waits on another process).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from _gpu_util import ntvs_module, rel_l2

pytestmark = pytest.mark.gpu


def _system(dtype, seed=8):
    s = synth.generate(synth.spec_scaled_3d(nx=32, ny=32, nz=4, n_hist=16_000, n_angles=32, n_blocks=4, seed=seed))
    return s, s.val.astype(dtype), s.b.astype(dtype)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_two_shards_partial_and_apply_match_oracle(dtype):
    ntvs = ntvs_module()
    import torch
    s, val, b = _system(dtype)
    bp = s.block_ptr()
    shape = (32, 32, 4)
    ctxs = []
    try:
        for rank in range(2):
            rp, c, v, bb, sbp = ntvs.shard_rows(s.row_ptr, s.col, val, b, bp, rank, 2)
            r = ntvs.Reconstructor(0)
            r.load(shape, rp, c, v, bb, n_blocks=len(sbp) - 1, block_ptr=sbp)
            ctxs.append(r)
        for t in range(len(bp) - 1):          # global hit counts of every block
            tot = sum(r.hit_counts(t).astype(np.int64) for r in ctxs).astype(np.int32)
            for r in ctxs:
                r.set_hit_counts(t, tot)
            assert np.array_equal(ctxs[0].hit_counts(t), tot)
        x0 = 0.9 * s.xstar + 0.05
        for r in ctxs:
            r.set_params(lam=1.2, N=0, alpha=0.5)
            r.set_image(x0)
        tdt = torch.float64 if dtype == np.float64 else torch.float32
        res = []
        for t in range(len(bp) - 1):
            parts = [torch.empty(32 * 32 * 4, dtype=tdt, device="cuda") for _ in ctxs]
            ss = sum(r.drop_block_partial(t, out=p)[1] for r, p in zip(ctxs, parts))
            tot = parts[0] + parts[1]
            torch.cuda.synchronize()
            for r in ctxs:
                r.apply_delta(t, tot)
            res.append(ss)
        x_a, x_b = ctxs[0].get_image(), ctxs[1].get_image()
    finally:
        for r in ctxs:
            r.close()
    want, ss_want = oracle.drop_sweep(s.row_ptr, s.col, val.astype(np.float64), b.astype(np.float64), bp, x0, 1.2)
    np.testing.assert_array_equal(x_a, x_b)
    assert rel_l2(x_a, want) < (1e-12 if dtype == np.float64 else 1e-6)
    np.testing.assert_allclose(res, ss_want, rtol=1e-10 if dtype == np.float64 else 1e-4)


def test_partial_of_row_ranges_adds_up_to_the_block():
    ntvs = ntvs_module()
    s, val, b = _system(np.float64, seed=3)
    bp = s.block_ptr()
    x0 = 0.8 * s.xstar + 0.1
    r = ntvs.Reconstructor(0)
    try:
        r.load((32, 32, 4), s.row_ptr, s.col, val, b, n_blocks=4)
        r.set_params(lam=0.7, N=0, alpha=0.5)
        r.set_image(x0)
        t = 2
        mid = (int(bp[t]) + int(bp[t + 1])) // 2 + 7
        d1, s1 = r.drop_block_partial(t, r0=int(bp[t]), r1=mid)
        d2, s2 = r.drop_block_partial(t, r0=mid, r1=int(bp[t + 1]))
        dw, sw = r.drop_block_partial(t)
        cnt = r.hit_counts(t)
        r.apply_delta(t, d1 + d2)
        got = r.get_image()
        with pytest.raises(ntvs.NtvsError):
            r.drop_block_partial(t, r0=int(bp[t]) - 1, r1=mid)
    finally:
        r.close()
    np.testing.assert_allclose(d1 + d2, dw, rtol=1e-12, atol=1e-15)
    assert s1 + s2 == pytest.approx(sw, rel=1e-12)
    want, _ = oracle.drop_block(s.row_ptr, s.col, val, b, int(bp[t]), int(bp[t + 1]), x0, 0.7)
    assert rel_l2(got, want) < 1e-12
    p0, p1 = int(s.row_ptr[bp[t]]), int(s.row_ptr[bp[t + 1]])
    ref_cnt = np.bincount(s.col[p0:p1][val[p0:p1] != 0], minlength=32 * 32 * 4)
    np.testing.assert_array_equal(cnt, ref_cnt)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_allreduce_callback_with_one_rank(dtype):
    """Sharded mode with a single rank (the sum over one rank is the identity): the NTVS
    run equals the oracle's and the callback sees the counts once, then every block's
    delta and residual."""
    ntvs = ntvs_module()
    from paper_1803_01112_gb300 import _ffi
    s, val, b = _system(dtype, seed=5)
    calls = []

    def cb(buf, n, dt, stream, user):
        calls.append((n, dt))
        return 0

    fn = _ffi.ALLREDUCE_FN(cb)
    prm = oracle.Params(lam=0.4, N=3, alpha=0.75, seed=4, eps_tv=1e-4)
    r = ntvs.Reconstructor(0)
    try:
        r.load((32, 32, 4), s.row_ptr, s.col, val, b, n_blocks=4)
        r.set_allreduce(fn)
        r.set_params(lam=prm.lam, N=prm.N, alpha=prm.alpha, seed=prm.seed, eps_tv=prm.eps_tv)
        r.set_image(s.xbar.astype(dtype))
        r.run(2)
        x = r.get_image()
        with pytest.raises(ntvs.NtvsError):   # counts are already global
            r.set_allreduce(fn)
    finally:
        r.close()
    ref = oracle.ntvs(s.row_ptr, s.col, val.astype(np.float64), b.astype(np.float64), s.block_ptr(), (32, 32, 4),
                      prm, 2, s.xbar)
    assert rel_l2(x, ref.x) < (1e-10 if dtype == np.float64 else 1e-5)
    assert calls[0][1] == _ffi.NTVS_I32 and len(calls) == 1 + 2 * 4 * 2
    assert all(dt == _ffi.NTVS_F64 and n == 1 for n, dt in calls[2::2])


_WORKER = r'''
import os, sys, numpy as np
sys.path.insert(0, os.environ["NTVS_ROOT"])
import torch, torch.distributed as dist
import synth, paper_1803_01112_gb300 as ntvs
rank, world = int(sys.argv[1]), int(sys.argv[2])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + sys.argv[3], rank=rank, world_size=world)
torch.cuda.set_device(0)
s = synth.generate(synth.spec_scaled_3d(nx=32, ny=32, nz=4, n_hist=16_000, n_angles=32, n_blocks=4, seed=5))
rp, c, v, bb, sbp = ntvs.shard_rows(s.row_ptr, s.col, s.val, s.b, s.block_ptr(), rank, world)
r = ntvs.Reconstructor(0)
r.load((32, 32, 4), rp, c, v, bb, n_blocks=len(sbp) - 1, block_ptr=sbp)
fn = ntvs.torch_allreduce(device=0)
r.set_allreduce(fn)
r.set_params(lam=0.4, N=3, alpha=0.75, seed=4, eps_tv=1e-4)
r.set_image(s.xbar)
r.run(2)
np.save(sys.argv[4] + f"_{rank}.npy", r.get_image())
r.close()
dist.destroy_process_group()
'''


def test_two_process_sharded_run_over_gloo(tmp_path):
    """Two processes, each with half of every block's rows, run 2 NTVS cycles with their
    deltas summed by gloo collectives; both end with the oracle's image of the whole
    system."""
    ntvs_module()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "worker.py"
    script.write_text(_WORKER)
    port = str(29500 + os.getpid() % 1000)
    env = dict(os.environ, NTVS_ROOT=root)
    out = str(tmp_path / "x")
    procs = [subprocess.Popen([sys.executable, str(script), str(k), "2", port, out], env=env) for k in range(2)]
    codes = [p.wait(timeout=300) for p in procs]
    assert codes == [0, 0]
    s, val, b = _system(np.float64, seed=5)
    prm = oracle.Params(lam=0.4, N=3, alpha=0.75, seed=4, eps_tv=1e-4)
    ref = oracle.ntvs(s.row_ptr, s.col, val, b, s.block_ptr(), (32, 32, 4), prm, 2, s.xbar)
    x0, x1 = np.load(out + "_0.npy"), np.load(out + "_1.npy")
    np.testing.assert_array_equal(x0, x1)
    assert rel_l2(x0, ref.x) < 1e-10
