"""On-the-fly rows on the GPU: the system is given as path records and traced in every DROP
sweep (FP32 geometry).  The oracle runs on the generator's stored rows (the same paths,
traced in FP64 on the host), so the bar accounts for FP32 path geometry: coordinates of
~100 mm carry ~1e-5 mm of rounding, i.e. ~1e-5 relative per intersection length; the
images are held to 3e-5 relative L2 (10x the dot-product error this implies)."""
import numpy as np
import pytest

import oracle
import synth
from _gpu_util import ntvs_module, rel_l2

pytestmark = pytest.mark.gpu


def _load(ntvs, spec, pr):
    r = ntvs.Reconstructor(0)
    r.load_paths((spec.nx, spec.ny, spec.nz), (spec.dx, spec.dy, spec.dz), pr.paths, pr.b.astype(np.float32),
                 n_blocks=spec.n_blocks, n_seg=spec.n_seg, min_len=spec.min_len)
    return r


@pytest.mark.parametrize("curved", [False, True])
def test_onthefly_sweep_matches_oracle_on_stored_rows(curved):
    ntvs = ntvs_module()
    spec = synth.spec_scaled_3d(nx=40, ny=36, nz=4, n_hist=20_000, n_angles=40, n_blocks=5, seed=41, curved=curved)
    s = synth.generate(spec)
    pr = synth.generate_paths(spec)
    b32 = pr.b.astype(np.float32).astype(np.float64)
    r = _load(ntvs, spec, pr)
    try:
        assert r.stats()["drop_schedule"] == 4   # NTVS_SCHED_ONTHEFLY
        for x0 in (s.xbar, 0.9 * s.xstar + 0.05):
            r.set_params(lam=0.8, N=0, alpha=0.5)
            r.set_image(x0)
            r.drop_sweep()
            got = r.get_image()
            want, ss = oracle.drop_sweep(s.row_ptr, s.col, s.val, b32, s.block_ptr(), x0, 0.8)
            assert rel_l2(got, want) <= 3e-5
            np.testing.assert_allclose(r.block_resid(), ss, rtol=1e-3)
    finally:
        r.close()


def test_onthefly_ntvs_run_matches_oracle():
    ntvs = ntvs_module()
    spec = synth.spec_scaled_3d(nx=32, ny=32, nz=3, n_hist=15_000, n_angles=30, n_blocks=4, seed=42)
    s = synth.generate(spec)
    pr = synth.generate_paths(spec)
    b32 = pr.b.astype(np.float32).astype(np.float64)
    prm = oracle.Params(lam=0.4, N=3, alpha=0.75, seed=6, eps_tv=1e-4)
    r = _load(ntvs, spec, pr)
    try:
        r.set_params(lam=prm.lam, N=prm.N, alpha=prm.alpha, seed=prm.seed, eps_tv=prm.eps_tv)
        r.set_image(s.xbar)
        r.run(3)
        got = r.get_image()
    finally:
        r.close()
    ref = oracle.ntvs(s.row_ptr, s.col, s.val, b32, s.block_ptr(), (32, 32, 3), prm, 3, s.xbar)
    assert rel_l2(got, ref.x) <= 3e-5


def test_onthefly_equals_stored_fp32_rows_on_gpu():
    """The traced rows and the generator's rows stored as FP32 CSR give the same sweep."""
    ntvs = ntvs_module()
    spec = synth.spec_scaled_3d(nx=48, ny=48, nz=5, n_hist=30_000, n_angles=36, n_blocks=3, seed=43)
    s = synth.generate(spec)
    pr = synth.generate_paths(spec)
    x0 = 0.8 * s.xstar + 0.1
    outs = []
    r = _load(ntvs, spec, pr)
    try:
        r.set_params(lam=1.0, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        outs.append(r.get_image())
    finally:
        r.close()
    r = ntvs.Reconstructor(0)
    try:
        r.load((48, 48, 5), s.row_ptr, s.col, s.val.astype(np.float32), pr.b.astype(np.float32), n_blocks=3)
        r.set_params(lam=1.0, N=0, alpha=0.5)
        r.set_image(x0)
        r.drop_sweep()
        outs.append(r.get_image())
    finally:
        r.close()
    assert rel_l2(outs[0], outs[1]) <= 3e-5


def test_onthefly_rejects_bad_paths():
    ntvs = ntvs_module()
    spec = synth.spec_scaled_3d(nx=16, ny=16, nz=2, n_hist=200, n_angles=8, n_blocks=1)
    pr = synth.generate_paths(spec)
    bad = pr.paths.copy()
    bad[7, 3] = np.nan
    r = ntvs.Reconstructor(0)
    try:
        with pytest.raises(ntvs.NtvsError):
            r.load_paths((16, 16, 2), (spec.dx, spec.dy, spec.dz), bad, pr.b.astype(np.float32))
        with pytest.raises(ntvs.NtvsError):
            r.load_paths((16, 16, 2), (spec.dx, spec.dy, spec.dz), pr.paths, pr.b.astype(np.float32), n_seg=0)
    finally:
        r.close()
