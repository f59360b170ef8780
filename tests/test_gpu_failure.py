"""Failure detection on the GPU without a fault: every bounded device wait gives up after
its budget, records an error code and lets its CTA leave; the host reports
NTVS_ERR_TIMEOUT and the context stays usable.

A test hook (ntvs_set_fault_hook) shortens the budget to 20 ms and makes one wait run out
on purpose -- a flag that nothing sets: the pipelined DROP producer withholds every CTA's
first stage, or the first CTA of the TV-check loop withholds its first arrival at the grid
barrier.  Afterwards the hook is cleared and a normal run must match the oracle again.
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu_util import load, ntvs_module, oracle_run, rel_l2

pytestmark = pytest.mark.gpu

WAIT_NS = 20_000_000


def test_pipelined_drop_wait_runs_out_and_context_recovers():
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_ERR_TIMEOUT, NTVS_HOOK_STARVE_PIPE, NTVS_SCHED_PIPELINE
    s = synth.generate(synth.spec_scaled_3d(nx=24, ny=24, nz=3, n_hist=6_000, n_angles=12, n_blocks=2, seed=9))
    val, b = s.val.astype(np.float32), s.b.astype(np.float32)
    x0 = s.xstar * 0.9 + 0.05
    r = ntvs.Reconstructor(0)
    try:
        r.load((24, 24, 3), s.row_ptr, s.col, val, b, n_blocks=2, schedule=NTVS_SCHED_PIPELINE)
        assert r.stats()["drop_schedule"] == NTVS_SCHED_PIPELINE
        r.set_params(lam=1.1, N=0, alpha=0.5)
        r.set_image(x0)
        r.set_fault_hook(WAIT_NS, NTVS_HOOK_STARVE_PIPE)
        r.drop_block(0)
        with pytest.raises(ntvs.NtvsError) as ei:
            r.sync()
        assert ei.value.code == NTVS_ERR_TIMEOUT and "pipelined DROP" in str(ei.value)
        r.sync()                          # the error was reported once and cleared
        r.set_fault_hook(0, 0)
        r.set_image(x0)
        r.drop_sweep()
        got = r.get_image()
    finally:
        r.close()
    want, _ = oracle.drop_sweep(s.row_ptr, s.col, val.astype(np.float64), b.astype(np.float64), s.block_ptr(),
                                x0, 1.1)
    assert rel_l2(got, want) < 1e-6


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_check_loop_barrier_runs_out_and_context_recovers(dtype):
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_ERR_TIMEOUT, NTVS_HOOK_STARVE_CHECK
    s = synth.generate(synth.spec_scaled_3d(nx=32, ny=32, nz=3, n_hist=20_000, n_angles=40, n_blocks=4))
    r, val64, b64 = load(ntvs, s, dtype)
    prm = oracle.Params(lam=0.3, N=4, alpha=0.75, seed=5, tv_check=True)
    kw = dict(lam=prm.lam, N=prm.N, alpha=prm.alpha, seed=prm.seed, tv_check=True)
    try:
        r.set_params(**kw)
        r.set_image(s.xbar.astype(dtype))
        r.set_fault_hook(WAIT_NS, NTVS_HOOK_STARVE_CHECK)
        r.run(1)
        with pytest.raises(ntvs.NtvsError) as ei:
            r.stats()
        assert ei.value.code == NTVS_ERR_TIMEOUT and "TV-check loop" in str(ei.value)
        # clear the hook, rewind the state and run the same cycles normally
        r.set_fault_hook(0, 0)
        r.set_state(0, 0)
        r.set_image(s.xbar.astype(dtype))
        r.run(3)
        x = r.get_image()
        st = r.stats()
    finally:
        r.close()
    ref = oracle_run(s, val64, b64, prm, 3, s.xbar)
    assert rel_l2(x, ref.x) <= (1e-10 if dtype == np.float64 else 1e-5)
    assert st["k"] == 3


def test_fault_hook_argument_errors():
    ntvs = ntvs_module()
    from paper_1803_01112_gb300._ffi import NTVS_ERR_ARG
    r = ntvs.Reconstructor(0)
    try:
        with pytest.raises(ntvs.NtvsError) as ei:
            r.set_fault_hook(0, 64)
        assert ei.value.code == NTVS_ERR_ARG
    finally:
        r.close()
