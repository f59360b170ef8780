"""Batched reconstructions on the GPU: every member of a batch (different grids, systems,
block counts and (lambda, N, alpha, beta0) parameters) must match the oracle run on that
member alone, after several cycles, and the single-context GPU path."""
import numpy as np
import pytest

import oracle
import synth
from _gpu_util import ntvs_module, rel_l2

pytestmark = pytest.mark.gpu


def _members():
    out = []
    cfgs = [dict(nx=24, ny=24, nz=2, n_hist=6000, n_blocks=3, lam=0.4, N=3, alpha=0.75),
            dict(nx=40, ny=32, nz=3, n_hist=9000, n_blocks=5, lam=2e-4, N=6, alpha=0.6),
            dict(nx=16, ny=16, nz=1, n_hist=2000, n_blocks=1, lam=1.0, N=0, alpha=0.5),
            dict(nx=32, ny=32, nz=4, n_hist=12000, n_blocks=2, lam=0.05, N=1, alpha=0.9, beta0=0.5),
            dict(nx=20, ny=28, nz=2, n_hist=4000, n_blocks=7, lam=0.8, N=4, alpha=0.75)]
    for k, c in enumerate(cfgs):
        spec = synth.spec_scaled_3d(nx=c["nx"], ny=c["ny"], nz=c["nz"], n_hist=c["n_hist"], n_angles=24,
                                    n_blocks=c["n_blocks"], seed=30 + k)
        s = synth.generate(spec)
        prm = oracle.Params(lam=c["lam"], N=c["N"], alpha=c["alpha"], beta0=c.get("beta0", 1.0), seed=100 + k,
                            eps_tv=1e-4)
        out.append((s, prm))
    return out


def test_batch_members_match_oracle_and_single_path():
    ntvs = ntvs_module()
    members = _members()
    K = 5
    bt = ntvs.Batch(0)
    try:
        for s, prm in members:
            shape = (s.spec.nx, s.spec.ny, s.spec.nz)
            bt.add(shape, s.row_ptr, s.col, s.val.astype(np.float32), s.b.astype(np.float32), s.spec.n_blocks,
                   ntvs.Params(lam=prm.lam, N=prm.N, alpha=prm.alpha, beta0=prm.beta0, seed=prm.seed,
                               eps_tv=prm.eps_tv), s.xbar)
        bt.finalize(max_cycles=16)
        bt.run(K - 2)
        bt.run(2)   # runs chain: k continues
        bt.run(0)
        st = bt.stats()
        assert st["members"] == len(members) and st["cycles"] == K
        assert st["lanes_per_row"] in (8, 16, 32)
        imgs = [bt.get_image(i) for i in range(len(members))]
        tvs = [bt.tv(i) for i in range(len(members))]
    finally:
        bt.close()
    for i, (s, prm) in enumerate(members):
        shape = (s.spec.nx, s.spec.ny, s.spec.nz)
        v64, b64 = s.val.astype(np.float32).astype(np.float64), s.b.astype(np.float32).astype(np.float64)
        ref = oracle.ntvs(s.row_ptr, s.col, v64, b64, s.block_ptr(), shape, prm, K, s.xbar)
        assert rel_l2(imgs[i], ref.x) <= 1e-5, f"member {i}"
        assert tvs[i] == pytest.approx(oracle.tv(imgs[i], shape), rel=1e-12)
        # the single-context path gives the same image
        r = ntvs.Reconstructor(0)
        try:
            r.load(shape, s.row_ptr, s.col, s.val.astype(np.float32), s.b.astype(np.float32),
                   n_blocks=s.spec.n_blocks)
            r.set_params(lam=prm.lam, N=prm.N, alpha=prm.alpha, beta0=prm.beta0, seed=prm.seed, eps_tv=prm.eps_tv)
            r.set_image(s.xbar)
            r.run(K)
            assert rel_l2(imgs[i], r.get_image()) <= 1e-6
        finally:
            r.close()


def test_batch_rejects_what_it_does_not_run():
    ntvs = ntvs_module()
    s = synth.generate(synth.spec_scaled_3d(nx=16, ny=16, nz=1, n_hist=500, n_angles=8, n_blocks=1))
    bt = ntvs.Batch(0)
    try:
        with pytest.raises(ntvs.NtvsError):      # FP64 values
            bt.add((16, 16, 1), s.row_ptr, s.col, s.val, s.b, 1, ntvs.Params(lam=1.0, N=1, alpha=0.5), s.xbar)
        with pytest.raises(ntvs.NtvsError):      # TV check
            bt.add((16, 16, 1), s.row_ptr, s.col, s.val.astype(np.float32), s.b.astype(np.float32), 1,
                   ntvs.Params(lam=1.0, N=1, alpha=0.5, tv_check=True), s.xbar)
        with pytest.raises(ntvs.NtvsError):      # nothing added yet
            bt.finalize(4)
        bt.add((16, 16, 1), s.row_ptr, s.col, s.val.astype(np.float32), s.b.astype(np.float32), 1,
               ntvs.Params(lam=1.0, N=1, alpha=0.5), s.xbar)
        bt.finalize(2)
        with pytest.raises(ntvs.NtvsError):      # beyond max_cycles
            bt.run(3)
    finally:
        bt.close()


def _shuffle_rows_within_blocks(s, seed):
    """The same system with the rows of every block in random order (block-DROP does not
    depend on the order inside a block), so its rows no longer come in runs of one slice."""
    rng = np.random.default_rng(seed)
    bp = s.block_ptr()
    order = np.concatenate([bp[t] + rng.permutation(bp[t + 1] - bp[t]) for t in range(len(bp) - 1)])
    lens = np.diff(s.row_ptr)[order]
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    idx = np.concatenate([np.arange(s.row_ptr[i], s.row_ptr[i + 1]) for i in order]).astype(np.int64)
    return rp, s.col[idx], s.val[idx], s.b[order], bp


def test_batch_row_order_and_large_slices_match_oracle():
    """Members with rows that run slice by slice, with rows in random order inside each
    block, and with a 160x160 slice, in one batch: every member equals its oracle run."""
    ntvs = ntvs_module()
    K = 3
    a = synth.generate(synth.spec_scaled_3d(nx=40, ny=40, nz=3, n_hist=12_000, n_angles=24, n_blocks=3, seed=50))
    b = synth.generate(synth.spec_scaled_3d(nx=36, ny=32, nz=2, n_hist=9_000, n_angles=24, n_blocks=2, seed=51))
    c = synth.generate(synth.spec_scaled_3d(nx=160, ny=160, nz=1, n_hist=6_000, n_angles=12, n_blocks=2, seed=52))
    rp_b, col_b, val_b, b_b, bp_b = _shuffle_rows_within_blocks(b, 3)
    cases = [((40, 40, 3), a.row_ptr, a.col, a.val, a.b, a.block_ptr(), a.xbar),
             ((36, 32, 2), rp_b, col_b, val_b, b_b, bp_b, b.xbar),
             ((160, 160, 1), c.row_ptr, c.col, c.val, c.b, c.block_ptr(), c.xbar)]
    prms = [oracle.Params(lam=0.5, N=2, alpha=0.75, seed=60 + k, eps_tv=1e-4) for k in range(3)]
    bt = ntvs.Batch(0)
    try:
        for (shape, rp, col, val, bb, bp, x0), prm in zip(cases, prms):
            bt.add(shape, rp, col, val.astype(np.float32), bb.astype(np.float32), len(bp) - 1,
                   ntvs.Params(lam=prm.lam, N=prm.N, alpha=prm.alpha, seed=prm.seed, eps_tv=prm.eps_tv), x0,
                   block_ptr=bp)
        bt.finalize(max_cycles=4)
        bt.run(K)
        imgs = [bt.get_image(i) for i in range(3)]
        # per cycle: 2 steps x (grad, apply) + phi + k, and per block step reset, DROP, apply
        assert bt.stats()["kernels_per_cycle"] == 2 * 2 + 2 + 3 * 3
    finally:
        bt.close()
    for (shape, rp, col, val, bb, bp, x0), prm, img in zip(cases, prms, imgs):
        v64, b64 = val.astype(np.float32).astype(np.float64), bb.astype(np.float32).astype(np.float64)
        ref = oracle.ntvs(rp, col, v64, b64, bp, shape, prm, K, x0)
        assert rel_l2(img, ref.x) <= 1e-5
