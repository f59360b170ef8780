"""Pins of the oracle's other step-size rules: OTVS (Appendix B: ell never reset, beta =
(1/2)^ell, one checked step per cycle) and the decoupled rule beta_{k,n} = alpha^n gamma^k
(Sec. VI).

The closed forms use a two-voxel image (nx = 2) with no rows, so P_T is the identity:
phi = |x1 - x0|, the normalized perturbation direction is (+1, -1)/sqrt(2) towards the
mean, and every accepted step of size beta moves the difference d = x1 - x0 by
sqrt(2) * beta towards (and possibly past) zero, while the mean stays put.
"""
import math

import numpy as np
import pytest

import oracle
import synth

R2 = math.sqrt(2.0)


def _two_voxels(prm, K, x0):
    return oracle.ntvs(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros(0),
                       np.array([0, 0], np.int64), (2, 1, 1), prm, K, np.asarray(x0, np.float64))


@pytest.mark.parametrize("alpha,gamma,N,K", [(0.5, 0.8, 3, 5), (0.75, 0.3, 1, 7), (0.9, 0.9, 4, 3)])
def test_decoupled_total_shift_closed_form(alpha, gamma, N, K):
    """With d large no step crosses the mean: x0 moves up by the sum of all steps over
    sqrt(2), and that sum over k < K, n < N of beta0 alpha^n gamma^k is
    beta0 (1 - alpha^N)/(1 - alpha) (1 - gamma^K)/(1 - gamma)."""
    beta0 = 1.5
    prm = oracle.Params(lam=1.0, N=N, alpha=alpha, beta0=beta0, eps_tv=1e-12, step_rule=oracle.STEP_DECOUPLED,
                        gamma=gamma)
    res = _two_voxels(prm, K, [0.0, 100.0])
    total = beta0 * (1 - alpha ** N) / (1 - alpha) * (1 - gamma ** K) / (1 - gamma)
    np.testing.assert_allclose(res.x, [total / R2, 100.0 - total / R2], rtol=1e-12, atol=1e-12)
    # the first step of cycle k is beta0 gamma^k, and the ratio within a cycle is alpha
    np.testing.assert_allclose(res.beta_step[:, 0], beta0 * gamma ** np.arange(K), rtol=1e-15)
    np.testing.assert_allclose(res.beta_step[:, 1:] / res.beta_step[:, :-1], alpha, rtol=1e-14)
    assert res.ell_prev == 0


def test_otvs_without_rejections_closed_form():
    """Far from the mean every try is accepted: ell advances by one per cycle, beta_k = 2^-k,
    and x0 moves by (2 - 2^(1-K))/sqrt(2)."""
    K = 9
    res = _two_voxels(oracle.Params.otvs(1.0, eps_tv=1e-12), K, [0.0, 100.0])
    np.testing.assert_array_equal(res.ell_k, np.arange(K))
    np.testing.assert_array_equal(res.tries.reshape(-1), np.ones(K))
    shift = (2.0 - 2.0 ** (1 - K)) / R2
    np.testing.assert_allclose(res.x, [shift, 100.0 - shift], rtol=1e-13)
    assert res.ell_prev == K


def test_otvs_with_rejections_worked_by_hand():
    """d0 = 1/2.  Cycle 0: beta 1 overshoots to |1/2 - sqrt2| > 1/2 (reject), beta 1/2 gives
    |1/2 - sqrt2/2| = 0.207 (accept).  Cycle 1: beta 1/4 -> 0.146 (accept).  Cycle 2: beta
    1/8 -> 0.030 (accept).  Cycle 3: beta 1/16 -> 0.058 > 0.030 (reject), beta 1/32 -> 0.0139
    (accept).  So ell_k = 0, 2, 3, 4; tries 2, 1, 1, 2; d = 1/2 - 11 sqrt2 / 32."""
    res = _two_voxels(oracle.Params.otvs(1.0, eps_tv=1e-12), 4, [0.0, 0.5])
    np.testing.assert_array_equal(res.ell_k, [0, 2, 3, 4])
    np.testing.assert_array_equal(res.tries.reshape(-1), [2, 1, 1, 2])
    np.testing.assert_array_equal(res.accepted.reshape(-1), [1, 1, 1, 1])
    np.testing.assert_allclose(res.beta_step.reshape(-1), [0.5, 0.25, 0.125, 1 / 32], rtol=0)
    d = 0.5 - 11.0 * R2 / 32.0
    np.testing.assert_allclose(res.x, [0.25 - d / 2, 0.25 + d / 2], rtol=1e-12, atol=1e-12)
    assert res.ell_prev == 6


def _small():
    return synth.generate(synth.spec_slice_2d().replace(n_hist=3000, n_blocks=3, nx=24, ny=24))


def test_otvs_ell_is_the_running_count_of_tries():
    s = _small()
    prm = oracle.Params.otvs(0.5, eps_tv=1e-8)
    K = 6
    res = oracle.ntvs(s.row_ptr, s.col, s.val, s.b, s.block_ptr(), (24, 24, 1), prm, K, s.xbar)
    counts = np.concatenate([[0], np.cumsum(res.tries.reshape(-1))])
    np.testing.assert_array_equal(res.ell_k, counts[:K])
    assert res.ell_prev == counts[K]
    np.testing.assert_allclose(res.beta_step.reshape(-1), 0.5 ** (res.ell_step.reshape(-1)), rtol=0)


def test_otvs_equals_checked_ntvs_on_the_same_schedule():
    """OTVS is the checked NTVS loop with N = 1, alpha = 1/2 and ell carried over: replaying
    the OTVS ell_k through the NTVS rule gives the same image and traces."""
    s = _small()
    K = 5
    a = oracle.ntvs(s.row_ptr, s.col, s.val, s.b, s.block_ptr(), (24, 24, 1), oracle.Params.otvs(0.5, eps_tv=1e-8),
                    K, s.xbar)
    ntvs = oracle.Params(lam=0.5, N=1, alpha=0.5, tv_check=True, eps_tv=1e-8)
    b = oracle.ntvs(s.row_ptr, s.col, s.val, s.b, s.block_ptr(), (24, 24, 1), ntvs, K, s.xbar,
                    ell_override=a.ell_k)
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.tries, b.tries)


def test_decoupled_with_gamma_alpha_equals_ntvs_with_ell_k_equal_k():
    """alpha^n alpha^k = alpha^(k + n): the decoupled rule with gamma = alpha is NTVS with
    ell_k = k replayed."""
    s = _small()
    K, N, alpha = 4, 3, 0.7
    dec = oracle.Params(lam=0.5, N=N, alpha=alpha, gamma=alpha, step_rule=oracle.STEP_DECOUPLED, eps_tv=1e-6)
    a = oracle.ntvs(s.row_ptr, s.col, s.val, s.b, s.block_ptr(), (24, 24, 1), dec, K, s.xbar)
    ntvs = oracle.Params(lam=0.5, N=N, alpha=alpha, eps_tv=1e-6)
    b = oracle.ntvs(s.row_ptr, s.col, s.val, s.b, s.block_ptr(), (24, 24, 1), ntvs, K, s.xbar,
                    ell_override=np.arange(K))
    np.testing.assert_allclose(a.x, b.x, rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal(a.ell_k, np.arange(K))


def test_rule_arguments():
    s = _small()
    with pytest.raises(ValueError):
        oracle.ntvs(s.row_ptr, s.col, s.val, s.b, s.block_ptr(), (24, 24, 1),
                    oracle.Params(lam=0.5, N=1, alpha=0.5, tv_check=True, step_rule=oracle.STEP_DECOUPLED), 1,
                    s.xbar)
    with pytest.raises(ValueError):
        oracle.ntvs(s.row_ptr, s.col, s.val, s.b, s.block_ptr(), (24, 24, 1),
                    oracle.Params(lam=0.5, N=1, alpha=0.5, step_rule=7), 1, s.xbar)
