"""Host logic of the multi-GPU benchmark path on CPU: torchrun-style ranks over gloo.

Reconstructions are independent, so N GPUs run N replicas; the only cross-rank steps are
the timing barrier and the MAX of the per-rank times, checked here with world size 2.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    bench.barrier(w)
    m = bench.max_over_ranks(10.0 * (rank + 1), w)
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((r, w, local, m))


def test_replica_timing_is_max_over_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 20.0 for o in out)


def test_single_rank_helpers_are_identity(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)


def _shard_main(rank, world, port, q):
    """One rank of the row-sharded DROP block design: rank p owns rows [r0 + p*h, ...) of the
    block, forms its partial numerator sum_i a_ij (b_i - <a_i, x>) / ||a_i||^2 over them, and
    an all-reduce (sum) of the partials over the ranks gives the block's numerator; every
    rank then applies x += lambda * num / s with the block's global hit counts s."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = synth.generate(synth.spec_scaled_3d(nx=20, ny=20, nz=2, n_hist=3000, n_angles=12, n_blocks=3, seed=71))
    bp = s.block_ptr()
    x = s.xstar * 0.9 + 0.05
    lam = 0.7
    t = 1
    r0, r1 = int(bp[t]), int(bp[t + 1])
    h = -(-(r1 - r0) // world)
    mine = range(r0 + rank * h, min(r1, r0 + (rank + 1) * h))
    num = np.zeros(s.spec.V)
    for i in mine:
        p0, p1 = s.row_ptr[i], s.row_ptr[i + 1]
        cols, vals = s.col[p0:p1], s.val[p0:p1]
        n2 = float(np.dot(vals, vals))
        if n2 > 0:
            num[cols] += vals * (s.b[i] - float(np.dot(vals, x[cols]))) / n2
    tn = torch.from_numpy(num)
    dist.all_reduce(tn, op=dist.ReduceOp.SUM)
    cnt = np.zeros(s.spec.V)
    for i in range(r0, r1):
        p0, p1 = s.row_ptr[i], s.row_ptr[i + 1]
        nz = s.val[p0:p1] != 0
        cnt[s.col[p0:p1][nz]] += 1
    x_new = x + np.where(cnt > 0, lam * tn.numpy() / np.where(cnt > 0, cnt, 1), 0.0)
    dist.destroy_process_group()
    q.put((rank, x_new, x, r0, r1, lam))


def test_row_sharded_drop_block_equals_unsharded_oracle():
    """Host emulation of the multi-GPU design (rows of a block split over ranks, one
    all-reduce of the partial delta per block): two gloo ranks give the oracle's block."""
    torch = pytest.importorskip("torch")
    import numpy as np
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=180) for _ in procs], key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    s = synth.generate(synth.spec_scaled_3d(nx=20, ny=20, nz=2, n_hist=3000, n_angles=12, n_blocks=3, seed=71))
    _, _, x, r0, r1, lam = out[0]
    want, _ = oracle.drop_block(s.row_ptr, s.col, s.val, s.b, r0, r1, x, lam)
    for o in out:
        np.testing.assert_allclose(o[1], want, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(out[0][1], out[1][1])
