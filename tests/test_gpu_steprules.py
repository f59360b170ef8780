"""The OTVS (Appendix B) and decoupled (Sec. VI) step-size rules on the GPU against the
FP64 oracle, through the C ABI, in the single-context and the batched drivers.

Bars as for NTVS: FP64 relative L2 <= 1e-10, FP32 <= 1e-5 (eps 1e-4); ell traces and
check decisions identical.  The two-voxel cases are checked against the values worked by
hand for the oracle's own pins (no rows: P_T is the identity).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from _gpu_util import ntvs_module, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def _gpu_params(ntvs, prm):
    return ntvs.Params(lam=prm.lam, N=prm.N, alpha=prm.alpha, beta0=prm.beta0, tv_check=prm.tv_check,
                       seed=prm.seed, eps_tv=prm.eps_tv, max_retries=prm.max_retries, step_rule=prm.step_rule,
                       gamma=prm.gamma)


def _run(ntvs, s, dtype, prm, K, x0):
    r = ntvs.Reconstructor(0)
    try:
        r.load((s.spec.nx, s.spec.ny, s.spec.nz), s.row_ptr, s.col, s.val.astype(dtype), s.b.astype(dtype),
               n_blocks=s.spec.n_blocks)
        r.set_params(_gpu_params(ntvs, prm))
        r.set_image(np.asarray(x0, dtype))
        r.run(K)
        x = r.get_image()
        ell, tries, acc = r.trace()
        st = r.stats()
    finally:
        r.close()
    return x, ell, tries, acc, st


def _system():
    return synth.generate(synth.spec_scaled_3d(nx=40, ny=36, nz=3, n_hist=30_000, n_angles=30, n_blocks=4,
                                               seed=21))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_otvs_matches_oracle(dtype):
    ntvs = ntvs_module()
    s = _system()
    K = 8
    prm = oracle.Params.otvs(0.5, eps_tv=1e-8 if dtype == np.float64 else 1e-4)
    x, ell, tries, acc, st = _run(ntvs, s, dtype, prm, K, s.xbar)
    v64, b64 = s.val.astype(dtype).astype(np.float64), s.b.astype(dtype).astype(np.float64)
    ref = oracle_run(s, v64, b64, prm, K, np.asarray(s.xbar, dtype))
    np.testing.assert_array_equal(ell, ref.ell_k)
    np.testing.assert_array_equal(tries, ref.tries.reshape(-1))
    np.testing.assert_array_equal(acc, ref.accepted.reshape(-1))
    assert st["ell_prev"] == ref.ell_prev
    assert rel_l2(x, ref.x) <= (1e-10 if dtype == np.float64 else 1e-5)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("gamma", [0.5, 0.95])
def test_decoupled_matches_oracle(dtype, gamma):
    ntvs = ntvs_module()
    s = _system()
    K = 6
    prm = oracle.Params(lam=0.5, N=4, alpha=0.8, beta0=0.7, step_rule=oracle.STEP_DECOUPLED, gamma=gamma,
                        eps_tv=1e-8 if dtype == np.float64 else 1e-4)
    x, ell, tries, acc, st = _run(ntvs, s, dtype, prm, K, s.xbar)
    v64, b64 = s.val.astype(dtype).astype(np.float64), s.b.astype(dtype).astype(np.float64)
    ref = oracle_run(s, v64, b64, prm, K, np.asarray(s.xbar, dtype))
    np.testing.assert_array_equal(ell, np.arange(K))
    assert st["ell_prev"] == 0
    assert rel_l2(x, ref.x) <= (1e-10 if dtype == np.float64 else 1e-5)


def _two_voxel_context(ntvs):
    r = ntvs.Reconstructor(0)
    r.load((2, 1, 1), np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros(0))
    return r


def test_two_voxel_otvs_worked_by_hand():
    ntvs = ntvs_module()
    r = _two_voxel_context(ntvs)
    try:
        r.set_params(ntvs.Params.otvs(1.0, eps_tv=1e-12))
        r.set_image(np.array([0.0, 0.5]))
        r.run(4)
        x = r.get_image()
        ell, tries, acc = r.trace()
    finally:
        r.close()
    np.testing.assert_array_equal(ell, [0, 2, 3, 4])
    np.testing.assert_array_equal(tries, [2, 1, 1, 2])
    d = 0.5 - 11.0 * math.sqrt(2.0) / 32.0
    np.testing.assert_allclose(x, [0.25 - d / 2, 0.25 + d / 2], rtol=1e-12, atol=1e-12)


def test_two_voxel_decoupled_closed_form():
    ntvs = ntvs_module()
    alpha, gamma, N, K, beta0 = 0.5, 0.8, 3, 5, 1.5
    r = _two_voxel_context(ntvs)
    try:
        r.set_params(lam=1.0, N=N, alpha=alpha, beta0=beta0, eps_tv=1e-12, step_rule=ntvs.NTVS_STEP_DECOUPLED,
                     gamma=gamma)
        r.set_image(np.array([0.0, 100.0]))
        r.run(K)
        x = r.get_image()
    finally:
        r.close()
    total = beta0 * (1 - alpha ** N) / (1 - alpha) * (1 - gamma ** K) / (1 - gamma)
    np.testing.assert_allclose(x, [total / math.sqrt(2.0), 100.0 - total / math.sqrt(2.0)], rtol=1e-12)


def test_batched_step_rules_match_oracle():
    """Batched members under the three rules (the batch runs without the TV check, so its
    OTVS-rule member carries ell with unchecked steps)."""
    ntvs = ntvs_module()
    members = []
    rules = [dict(step_rule=oracle.STEP_NTVS), dict(step_rule=oracle.STEP_OTVS, alpha=0.5),
             dict(step_rule=oracle.STEP_DECOUPLED, gamma=0.6), dict(step_rule=oracle.STEP_DECOUPLED, gamma=0.9)]
    for i, rk in enumerate(rules):
        s = synth.generate(synth.spec_scaled_3d(nx=24 + 4 * i, ny=24, nz=2, n_hist=5000, n_angles=20, n_blocks=2,
                                                seed=40 + i))
        kw = dict(lam=0.5, N=3, alpha=0.75, seed=7 + i, eps_tv=1e-4)
        kw.update(rk)
        members.append((s, oracle.Params(**kw)))
    K = 5
    bt = ntvs.Batch(0)
    try:
        for s, prm in members:
            bt.add((s.spec.nx, s.spec.ny, s.spec.nz), s.row_ptr, s.col, s.val.astype(np.float32),
                   s.b.astype(np.float32), s.spec.n_blocks, _gpu_params(ntvs, prm), s.xbar)
        bt.finalize(max_cycles=8)
        bt.run(K)
        imgs = [bt.get_image(i) for i in range(len(members))]
    finally:
        bt.close()
    for i, (s, prm) in enumerate(members):
        v64, b64 = s.val.astype(np.float32).astype(np.float64), s.b.astype(np.float32).astype(np.float64)
        ref = oracle.ntvs(s.row_ptr, s.col, v64, b64, s.block_ptr(), (s.spec.nx, s.spec.ny, s.spec.nz), prm, K,
                          s.xbar)
        assert rel_l2(imgs[i], ref.x) <= 1e-5, f"member {i}"


def test_step_rule_argument_errors():
    ntvs = ntvs_module()
    r = ntvs.Reconstructor(0)
    try:
        with pytest.raises(ntvs.NtvsError, match="step_rule"):
            r.set_params(lam=1.0, N=1, alpha=0.5, step_rule=3)
        with pytest.raises(ntvs.NtvsError, match="gamma"):
            r.set_params(lam=1.0, N=1, alpha=0.5, step_rule=ntvs.NTVS_STEP_DECOUPLED, gamma=1.0)
        with pytest.raises(ntvs.NtvsError, match="TV check"):
            r.set_params(lam=1.0, N=1, alpha=0.5, step_rule=ntvs.NTVS_STEP_DECOUPLED, gamma=0.5, tv_check=True)
        r.set_params(ntvs.Params.otvs(1e-4))
    finally:
        r.close()
