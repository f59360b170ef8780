"""Batched reconstructions on the GPU: every member of a batch (different grids, systems,
block counts, (lambda, N, alpha, beta0) parameters, with and without the TV check) must
match the oracle run on that member alone, after several cycles, and the single-context
GPU path; one cycle is two launches (setup + the persistent kernel) whatever the schedule."""
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
        assert st["kernels_per_cycle"] == 2 and st["n_launches"] == 2 * K
        # the finalize-time tuning timed 3 x 4 x 2 schedules, then 3 rows-per-warp settings
        tun = bt.tuning()
        assert len(tun) == 27 and all(ms > 0 for *_, ms in tun)
        assert st["lanes_per_row_all"] in (0, 8, 16, 32)
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
        with pytest.raises(ntvs.NtvsError):      # the decoupled rule has no TV check
            bt.add((16, 16, 1), s.row_ptr, s.col, s.val.astype(np.float32), s.b.astype(np.float32), 1,
                   ntvs.Params(lam=1.0, N=1, alpha=0.5, tv_check=True, step_rule=2), s.xbar)
        with pytest.raises(ntvs.NtvsError):      # a column outside the grid
            bad = s.col.copy()
            bad[3] = 16 * 16
            bt.add((16, 16, 1), s.row_ptr, bad, s.val.astype(np.float32), s.b.astype(np.float32), 1,
                   ntvs.Params(lam=1.0, N=1, alpha=0.5), s.xbar)
        with pytest.raises(ntvs.NtvsError):      # a non-finite right-hand side
            bb = s.b.astype(np.float32)
            bb[0] = np.nan
            bt.add((16, 16, 1), s.row_ptr, s.col, s.val.astype(np.float32), bb, 1,
                   ntvs.Params(lam=1.0, N=1, alpha=0.5), s.xbar)
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
        assert bt.stats()["kernels_per_cycle"] == 2
    finally:
        bt.close()
    for (shape, rp, col, val, bb, bp, x0), prm, img in zip(cases, prms, imgs):
        v64, b64 = val.astype(np.float32).astype(np.float64), bb.astype(np.float32).astype(np.float64)
        ref = oracle.ntvs(rp, col, v64, b64, bp, shape, prm, K, x0)
        assert rel_l2(img, ref.x) <= 1e-5


def _check_case(seed):
    return synth.generate(synth.spec_scaled_3d(nx=32, ny=32, nz=3, n_hist=20_000, n_angles=40, n_blocks=4,
                                               seed=seed))


def test_batch_tv_check_members_match_oracle():
    """Checked and unchecked members side by side; the checked ones take their decisions
    on the device (speculative passes of four tries) and must reproduce the oracle's
    tries, acceptances and ell schedule."""
    ntvs = ntvs_module()
    K = 4
    cases = [(_check_case(3), oracle.Params(lam=0.3, N=4, alpha=0.75, seed=5, tv_check=True)),
             (_check_case(3), oracle.Params(lam=0.3, N=6, alpha=0.75, seed=9, tv_check=True)),
             (_check_case(4), oracle.Params(lam=0.3, N=3, alpha=0.75, seed=2)),
             (_check_case(5), oracle.Params.otvs(0.3, seed=1))]
    bt = ntvs.Batch(0)
    try:
        for s, prm in cases:
            bt.add((32, 32, 3), s.row_ptr, s.col, s.val.astype(np.float32), s.b.astype(np.float32), 4,
                   ntvs.Params(lam=prm.lam, N=prm.N, alpha=prm.alpha, beta0=prm.beta0, seed=prm.seed,
                               tv_check=prm.tv_check, step_rule=prm.step_rule), s.xbar)
        bt.finalize(max_cycles=K)
        bt.run(K)
        imgs = [bt.get_image(i) for i in range(len(cases))]
        mems = [bt.member(i) for i in range(len(cases))]
    finally:
        bt.close()
    rejections = 0
    for (s, prm), img, mem in zip(cases, imgs, mems):
        v64, b64 = s.val.astype(np.float32).astype(np.float64), s.b.astype(np.float32).astype(np.float64)
        ref = oracle.ntvs(s.row_ptr, s.col, v64, b64, s.block_ptr(), (32, 32, 3), prm, K, s.xbar)
        assert rel_l2(img, ref.x) <= 1e-5
        assert mem["k"] == K and mem["n_steps"] == K * prm.N
        if prm.tv_check:
            assert mem["n_tries"] == ref.tries.sum() and mem["n_accepted"] == ref.accepted.sum()
            assert mem["ell_prev"] == ref.ell_prev
            rejections += ref.tries.sum() - ref.tries.size
    assert rejections > 0


def test_batch_tv_check_skips_a_step_after_max_retries():
    """beta0 so large that every try raises phi: each step makes max_retries = 6 tries
    (a pass of four, then one of two) and is skipped; ell advances by 6 per step."""
    ntvs = ntvs_module()
    s = _check_case(6)
    prm = oracle.Params(lam=0.3, N=2, alpha=0.99, beta0=1e6, seed=4, tv_check=True, max_retries=6)
    K = 2
    bt = ntvs.Batch(0)
    try:
        bt.add((32, 32, 3), s.row_ptr, s.col, s.val.astype(np.float32), s.b.astype(np.float32), 4,
               ntvs.Params(lam=prm.lam, N=prm.N, alpha=prm.alpha, beta0=prm.beta0, seed=prm.seed, tv_check=True,
                           max_retries=6), s.xbar)
        bt.set_schedule(rows_per_item=256, window_floats=0)
        bt.finalize(max_cycles=K)
        bt.run(K)
        img = bt.get_image(0)
        mem = bt.member(0)
    finally:
        bt.close()
    v64, b64 = s.val.astype(np.float32).astype(np.float64), s.b.astype(np.float32).astype(np.float64)
    ref = oracle.ntvs(s.row_ptr, s.col, v64, b64, s.block_ptr(), (32, 32, 3), prm, K, s.xbar)
    assert ref.accepted.sum() == 0 and np.all(ref.tries == 6)
    assert mem["n_tries"] == 6 * K * prm.N and mem["n_accepted"] == 0 and mem["ell_prev"] == ref.ell_prev
    assert rel_l2(img, ref.x) <= 1e-5


@pytest.mark.parametrize("rows,window", [(64, 1024), (512, 0), (128, 16384)])
def test_batch_schedules_agree(rows, window):
    """Every fixed schedule (rows per item; a shared scatter window holding whole items,
    one too small for them, so that only the entries near the item's mean column are
    staged, or none) gives the oracle's images; only the order of FP32 summation differs."""
    ntvs = ntvs_module()
    K = 3
    members = _members()[:3]
    bt = ntvs.Batch(0)
    try:
        for s, prm in members:
            bt.add((s.spec.nx, s.spec.ny, s.spec.nz), s.row_ptr, s.col, s.val.astype(np.float32),
                   s.b.astype(np.float32), s.spec.n_blocks,
                   ntvs.Params(lam=prm.lam, N=prm.N, alpha=prm.alpha, beta0=prm.beta0, seed=prm.seed,
                               eps_tv=prm.eps_tv), s.xbar)
        bt.set_schedule(rows_per_item=rows, window_floats=window)
        bt.finalize(max_cycles=K)
        bt.run(K)
        st = bt.stats()
        assert st["rows_per_item"] == rows and st["window_floats"] == window
        imgs = [bt.get_image(i) for i in range(len(members))]
    finally:
        bt.close()
    for (s, prm), img in zip(members, imgs):
        shape = (s.spec.nx, s.spec.ny, s.spec.nz)
        v64, b64 = s.val.astype(np.float32).astype(np.float64), s.b.astype(np.float32).astype(np.float64)
        ref = oracle.ntvs(s.row_ptr, s.col, v64, b64, s.block_ptr(), shape, prm, K, s.xbar)
        assert rel_l2(img, ref.x) <= 1e-5


def test_batch_window_rows_above_the_bound_go_global():
    """The shared window holds int32 multiples of a quantum scaled by a bound on |r_i/lambda|
    (seeded with max_i |b_i| / ||a_i||^2, the residual at x = 0, then twice the previous
    sweep's largest).  Starting from x0 = -5 xbar every residual of the first sweep is about
    six times the seed, so those rows must scatter to global memory; later sweeps take the
    bound from what they saw.  The images stay the oracle's."""
    ntvs = ntvs_module()
    K = 3
    members = _members()[:3]
    bt = ntvs.Batch(0)
    x0s = []
    try:
        for s, prm in members:
            x0 = -5.0 * s.xbar
            x0s.append(x0)
            bt.add((s.spec.nx, s.spec.ny, s.spec.nz), s.row_ptr, s.col, s.val.astype(np.float32),
                   s.b.astype(np.float32), s.spec.n_blocks,
                   ntvs.Params(lam=prm.lam, N=prm.N, alpha=prm.alpha, beta0=prm.beta0, seed=prm.seed,
                               eps_tv=prm.eps_tv), x0)
        bt.set_schedule(rows_per_item=128, window_floats=8192)
        bt.finalize(max_cycles=K)
        bt.run(K)
        imgs = [bt.get_image(i) for i in range(len(members))]
    finally:
        bt.close()
    for (s, prm), img, x0 in zip(members, imgs, x0s):
        shape = (s.spec.nx, s.spec.ny, s.spec.nz)
        v64, b64 = s.val.astype(np.float32).astype(np.float64), s.b.astype(np.float32).astype(np.float64)
        ref = oracle.ntvs(s.row_ptr, s.col, v64, b64, s.block_ptr(), shape, prm, K, x0)
        assert rel_l2(img, ref.x) <= 1e-5


def test_batch_members_from_paths_match_oracle():
    """Members traced on the device from path records: their stored rows (read back) are
    valid intersection-length rows, and each member equals the oracle run on those rows."""
    ntvs = ntvs_module()
    K = 3
    specs = [synth.spec_scaled_3d(nx=40, ny=40, nz=3, n_hist=12_000, n_angles=24, n_blocks=3, seed=70),
             synth.spec_scaled_3d(nx=24, ny=32, nz=2, n_hist=7_001, n_angles=24, n_blocks=2, seed=71,
                                  curved=False)]
    paths = [synth.generate_paths(sp) for sp in specs]
    prms = [oracle.Params(lam=0.5, N=2, alpha=0.75, seed=80 + k, eps_tv=1e-4) for k in range(2)]
    bt = ntvs.Batch(0)
    try:
        for sp, P, prm in zip(specs, paths, prms):
            bt.add_paths((sp.nx, sp.ny, sp.nz), (sp.dx, sp.dy, sp.dz), P.paths, P.b.astype(np.float32),
                         sp.n_blocks, ntvs.Params(lam=prm.lam, N=prm.N, alpha=prm.alpha, seed=prm.seed,
                                                  eps_tv=prm.eps_tv), P.xbar, n_seg=sp.n_seg, min_len=sp.min_len)
        bt.finalize(max_cycles=K)
        bt.run(K)
        imgs = [bt.get_image(i) for i in range(2)]
        rows = [bt.rows(i) for i in range(2)]
    finally:
        bt.close()
    for sp, P, prm, img, (rp, col, val) in zip(specs, paths, prms, imgs, rows):
        V = sp.nx * sp.ny * sp.nz
        assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == col.size
        assert col.min() >= 0 and col.max() < V and np.all(val >= sp.min_len)
        # the stored rows and the generator's (FP64 trace of the same paths) agree closely
        s = synth.generate(sp)
        assert abs(val.astype(np.float64).sum() / s.val.sum() - 1.0) < 1e-3
        shape = (sp.nx, sp.ny, sp.nz)
        bp = synth.block_partition(P.M, sp.n_blocks)
        b32 = P.b.astype(np.float32).astype(np.float64)
        ref = oracle.ntvs(rp, col, val.astype(np.float64), b32, bp, shape, prm, K, P.xbar)
        assert rel_l2(img, ref.x) <= 1e-5


def test_batch_bounded_wait_reports_a_stalled_member():
    """The starve hook keeps member 0 in its first phase: the other members finish, every
    CTA runs out of work, the bounded wait (50 ms) ends the cycle and the host gets
    NTVS_ERR_TIMEOUT instead of a hang."""
    ntvs = ntvs_module()
    members = _members()[:3]
    bt = ntvs.Batch(0)
    try:
        for s, prm in members:
            bt.add((s.spec.nx, s.spec.ny, s.spec.nz), s.row_ptr, s.col, s.val.astype(np.float32),
                   s.b.astype(np.float32), s.spec.n_blocks, ntvs.Params(lam=prm.lam, N=prm.N, alpha=prm.alpha),
                   s.xbar)
        bt.set_fault_hook(wait_ns=50_000_000, flags=ntvs._ffi.NTVS_HOOK_STARVE_BATCH)
        bt.finalize(max_cycles=2)
        bt.run(1)
        with pytest.raises(ntvs.NtvsError) as e:
            bt.sync()
        assert e.value.code == ntvs._ffi.NTVS_ERR_TIMEOUT
        assert "member 0" in str(e.value)
    finally:
        bt.close()
