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
