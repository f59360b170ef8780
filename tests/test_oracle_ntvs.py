"""Pins of the oracle's NTVS loop (Appendix C) and its ell schedule (Sec. III-B, item 4).

* SplitMix64: published first outputs of the stream seeded with 0 and an independent
  stateful Python SplitMix64.
* ell_k = rand(k, ell_{k-1}): bounds, and ell_k = k for N = 1 without the check (Sec. III-B).
* N = 0 is plain DROP; the check variant with no rejection equals the variant without it;
  accepted perturbations never raise phi; a budget of one rejected try leaves x unchanged.
"""
import numpy as np
import pytest

import oracle
import synth

MASK = (1 << 64) - 1


def splitmix64_stateful(seed, count):
    """SplitMix64 as published: state += golden gamma, then the two xor-shift-multiply rounds."""
    state, out = seed & MASK, []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_published_values():
    assert [oracle.splitmix64(0, n) for n in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("seed", [0, 1, 12345, 0xDEADBEEFCAFEF00D])
def test_splitmix64_matches_stateful_definition(seed):
    ref = splitmix64_stateful(seed, 300)
    assert [oracle.splitmix64(seed, n) for n in range(300)] == ref
    # the input generator's own copy agrees too
    assert [synth.splitmix64_at(seed, n) for n in range(300)] == ref


def test_rand_ell_bounds_and_spread():
    seen = set()
    for k in range(2000):
        prev = (k * 7919) % 97
        e = oracle.rand_ell(42, k, prev)
        assert min(k, prev) <= e <= max(k, prev)
        if prev == 50 and k > 50:
            seen.add(e - 50)
    # degenerate interval
    assert oracle.rand_ell(3, 10, 10) == 10
    # uniform draw on [lo, hi] = lo + (draw k) mod (hi - lo + 1)
    k, prev = 5, 17
    assert oracle.rand_ell(9, k, prev) == 5 + splitmix64_stateful(9, k + 1)[k] % 13


def _tiny_problem(seed=0, V_shape=(6, 5, 2), M=80, per_row=6):
    rng = np.random.default_rng(seed)
    nx, ny, nz = V_shape
    V = nx * ny * nz
    rows = [np.sort(rng.choice(V, size=per_row, replace=False)) for _ in range(M)]
    rp = np.zeros(M + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    val = rng.uniform(0.2, 1.4, size=col.size)
    xs = rng.uniform(0.5, 1.5, size=V)
    b = np.add.reduceat(val * xs[col], rp[:-1]) * (1 + 0.01 * rng.normal(size=M))
    x0 = rng.uniform(0.8, 1.2, size=V)
    return rp, col, val, b, V_shape, x0


def test_N1_without_check_has_ell_k_equal_k():
    rp, col, val, b, shape, x0 = _tiny_problem()
    bp = synth.block_partition(len(b), 4)
    res = oracle.ntvs(rp, col, val, b, bp, shape, oracle.Params(lam=0.1, N=1, alpha=0.75, seed=77), 12, x0)
    np.testing.assert_array_equal(res.ell_k, np.arange(12))
    np.testing.assert_array_equal(res.ell_step[:, 0], np.arange(12))


@pytest.mark.parametrize("N,check", [(3, False), (6, False), (2, True), (5, True)])
def test_ell_k_at_least_k_and_steps_increment(N, check):
    rp, col, val, b, shape, x0 = _tiny_problem(1)
    bp = synth.block_partition(len(b), 3)
    res = oracle.ntvs(rp, col, val, b, bp, shape,
                      oracle.Params(lam=0.2, N=N, alpha=0.6, seed=5, tv_check=check), 10, x0)
    assert np.all(res.ell_k >= np.arange(10))
    if not check:
        np.testing.assert_array_equal(res.ell_step, res.ell_k[:, None] + np.arange(N)[None, :])
    else:   # every try bumps ell by one
        for k in range(10):
            ell = res.ell_k[k]
            for n in range(N):
                ell += res.tries[k, n]
                assert res.ell_step[k, n] == ell - 1
    # rand(k, ell_{k-1}) never exceeds the previous cycle's final ell
    finals = res.ell_step[:, -1] + 1
    assert np.all(res.ell_k[1:] <= np.maximum(finals[:-1], np.arange(1, 10)))


def test_N0_is_plain_drop():
    rp, col, val, b, shape, x0 = _tiny_problem(2)
    bp = synth.block_partition(len(b), 5)
    res = oracle.ntvs(rp, col, val, b, bp, shape, oracle.Params(lam=0.5, N=0, alpha=0.75), 6, x0)
    x = x0.copy()
    for _ in range(6):
        x, _ = oracle.drop_sweep(rp, col, val, b, bp, x, 0.5)
    np.testing.assert_array_equal(res.x, x)


def test_check_without_rejections_equals_no_check():
    # tiny steps along -grad phi always lower phi, so every first try is accepted
    rp, col, val, b, shape, x0 = _tiny_problem(3)
    bp = synth.block_partition(len(b), 4)
    p = dict(lam=0.3, N=3, alpha=0.75, beta0=1e-4, seed=11)
    a = oracle.ntvs(rp, col, val, b, bp, shape, oracle.Params(**p, tv_check=False), 5, x0)
    c = oracle.ntvs(rp, col, val, b, bp, shape, oracle.Params(**p, tv_check=True), 5, x0)
    assert np.all(c.tries == 1) and np.all(c.accepted == 1)
    np.testing.assert_array_equal(a.x, c.x)
    np.testing.assert_array_equal(a.ell_k, c.ell_k)


def test_accepted_steps_never_raise_tv():
    # no rows: P_T is the identity, so phi must not increase over a cycle in check mode
    shape = (8, 7, 3)
    V = 168
    x = np.random.default_rng(4).uniform(0, 2, size=V)
    empty = (np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros(0))
    ell_prev = 0
    for k in range(8):
        before = oracle.tv(x, shape)
        res = oracle.ntvs(*empty, [0], shape, oracle.Params(lam=1.0, N=4, alpha=0.75, tv_check=True, seed=2),
                          1, x, k0=k, ell_prev=ell_prev)
        assert oracle.tv(res.x, shape) <= before
        x, ell_prev = res.x, res.ell_prev


def test_rejected_budget_leaves_image_unchanged():
    # a lone spike: the unit-length first step overshoots and raises phi
    shape = (5, 5, 1)
    x = np.zeros(25)
    x[12] = 0.05
    empty = (np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros(0))
    res = oracle.ntvs(*empty, [0], shape, oracle.Params(lam=1.0, N=1, alpha=0.5, tv_check=True, max_retries=1),
                      1, x)
    assert res.tries[0, 0] == 1 and res.accepted[0, 0] == 0
    np.testing.assert_array_equal(res.x, x)
    # with a larger budget a step is eventually accepted, after ell has grown
    res2 = oracle.ntvs(*empty, [0], shape, oracle.Params(lam=1.0, N=1, alpha=0.5, tv_check=True), 1, x)
    assert res2.accepted[0, 0] == 1 and res2.tries[0, 0] > 1
    assert oracle.tv(res2.x, shape) <= oracle.tv(x, shape)


def test_flat_image_has_zero_perturbation():
    shape = (4, 4, 2)
    x = np.full(32, 0.9)
    empty = (np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros(0))
    res = oracle.ntvs(*empty, [0], shape, oracle.Params(lam=1.0, N=3, alpha=0.75), 2, x)
    np.testing.assert_array_equal(res.x, x)


def test_resume_equals_one_run():
    rp, col, val, b, shape, x0 = _tiny_problem(5)
    bp = synth.block_partition(len(b), 4)
    p = oracle.Params(lam=0.2, N=4, alpha=0.75, seed=99)
    whole = oracle.ntvs(rp, col, val, b, bp, shape, p, 6, x0)
    first = oracle.ntvs(rp, col, val, b, bp, shape, p, 3, x0)
    second = oracle.ntvs(rp, col, val, b, bp, shape, p, 3, first.x, k0=3, ell_prev=first.ell_prev)
    np.testing.assert_array_equal(whole.x, second.x)
    np.testing.assert_array_equal(whole.ell_k, np.concatenate([first.ell_k, second.ell_k]))


def test_ell_override_replays_schedule():
    rp, col, val, b, shape, x0 = _tiny_problem(6)
    bp = synth.block_partition(len(b), 2)
    p = oracle.Params(lam=0.2, N=3, alpha=0.75, seed=1234)
    a = oracle.ntvs(rp, col, val, b, bp, shape, p, 4, x0)
    c = oracle.ntvs(rp, col, val, b, bp, shape, oracle.Params(lam=0.2, N=3, alpha=0.75, seed=1),
                    4, x0, ell_override=a.ell_k)
    np.testing.assert_array_equal(a.x, c.x)


def test_perturbation_step_closed_form():
    # no rows (P_T = identity), N = 1, no check: cycle k moves x by -beta0*alpha^k * g/||g||
    shape = (6, 4, 2)
    x0 = np.random.default_rng(8).uniform(0, 2, size=48)
    empty = (np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros(0))
    eps, a, b0 = 1e-8, 0.6, 0.8
    res = oracle.ntvs(*empty, [0], shape, oracle.Params(lam=1.0, N=1, alpha=a, beta0=b0, eps_tv=eps), 2, x0)
    x = x0.copy()
    for k in range(2):
        g = oracle.tv_grad(x, shape, eps)
        x = x - b0 * a ** k * g / np.linalg.norm(g)
    np.testing.assert_allclose(res.x, x, rtol=1e-14, atol=1e-15)
