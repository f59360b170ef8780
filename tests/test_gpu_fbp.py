"""Parity of the initial-iterate kernels (include/ntvs_fbp.h) with the FP64 oracle.

Integer work (bin indices, counts, median selection, hull decisions away from tau) is
compared exactly; floating point within bounds derived from the arithmetic:
  * bin means: the same values summed in another order (atomics) -> 1e-14 relative;
  * filter: n_t products summed with and without fused multiply-add -> 1e-13 of the
    row's largest |q|;
  * back-projection: cos/sin within an ulp and a multiply by 1/dt instead of a divide move
    each interpolation weight by ~1e-16; over n_theta terms -> 1e-12 of max |f|;
  * median: a 1-Lipschitz function of its inputs in the max norm, so its error is the
    input's error; the chain inherits the back-projection bound.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from _gpu_util import ntvs_module

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ntvs():
    return ntvs_module()


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def _geoms(ntvs, **kw):
    keys = ("nx", "ny", "nz", "dx", "dy", "dz", "n_theta", "n_t", "dt")
    args = [kw[k] for k in keys]
    return oracle.fbp_geom(*args, theta0=kw.get("theta0", 0.0)), ntvs.fbp_geom(*args, theta0=kw.get("theta0", 0.0))


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _gpu_bin(ntvs, torch, gd, paths, wepl):
    S = gd.nz * gd.n_theta * gd.n_t
    sino = torch.empty(S, dtype=torch.float64, device="cuda")
    cnt = torch.empty(S, dtype=torch.int32, device="cuda")
    ntvs.ntvs_fbp_bin(gd, _dev(torch, paths, torch.float32), _dev(torch, wepl, torch.float64), sino, cnt)
    torch.cuda.synchronize()
    shape = (gd.nz, gd.n_theta, gd.n_t)
    return sino.cpu().numpy().reshape(shape), cnt.cpu().numpy().reshape(shape)


def _rec(p, q):
    return np.array([p[0], p[1], p[2], q[0], q[1], q[2], 0, 0, 0, 0], np.float32)


def test_bin_hand_records(ntvs, torch):
    go, gd = _geoms(ntvs, nx=8, ny=8, nz=2, dx=1.0, dy=1.0, dz=2.5, n_theta=5, n_t=10, dt=2.0)
    d = (math.cos(math.radians(80)), math.sin(math.radians(80)))
    n = (math.cos(math.radians(170)), math.sin(math.radians(170)))
    p0 = (4.6 * n[0] - 60 * d[0], 4.6 * n[1] - 60 * d[1], 4.0)
    p1 = (4.6 * n[0] + 60 * d[0], 4.6 * n[1] + 60 * d[1], 4.0)
    recs = np.stack([_rec((-100, 5, 1.0), (100, 5, 1.0)), _rec((100, 5.5, 1.2), (-100, 5.5, 1.2)),
                     _rec((3, -100, 3.0), (3, 100, 3.0)), _rec((-50, -40, 0.5), (50, 60, 0.5)),
                     _rec(p0, p1), _rec(p1, p0), _rec((100, -10, 1.0), (-100, -10, 1.0)),
                     _rec((-100, 10, 1.0), (100, 10, 1.0)), _rec((-100, 0, 6.0), (100, 0, 6.0)),
                     np.zeros(10, np.float32)])
    wepl = np.arange(1.0, len(recs) + 1.0)
    so, co = oracle.fbp_bin(recs, wepl, go)
    sg, cg = _gpu_bin(ntvs, torch, gd, recs, wepl)
    assert np.array_equal(cg, co)
    assert np.array_equal(sg, so)
    assert co.sum() == 7


@pytest.mark.parametrize("theta0", [0.0, 0.05])
def test_bin_near_angle_edges(ntvs, torch, theta0):
    # normals 2e-7 .. 8e-6 rad either side of every angle-bin edge (the fold at pi included),
    # both chord directions: the FP32 angle alone would misplace some of them
    n_theta = 12
    go, gd = _geoms(ntvs, nx=8, ny=8, nz=2, dx=1.0, dy=1.0, dz=2.5, n_theta=n_theta, n_t=40, dt=1.0, theta0=theta0)
    rng = np.random.default_rng(5)
    recs = []
    for e in range(2 * n_theta):
        edge = theta0 + e * math.pi / n_theta
        for d in (2e-7, -2e-7, 5e-7, -5e-7, 2e-6, -2e-6, 8e-6, -8e-6):
            th = edge + d
            n = np.array([math.cos(th), math.sin(th)])
            u = np.array([-n[1], n[0]])
            t = rng.uniform(-15, 15)
            z = rng.uniform(0.1, 4.9)
            p0, p1 = t * n - 80 * u, t * n + 80 * u
            recs.append(_rec((p0[0], p0[1], z), (p1[0], p1[1], z)))
            recs.append(_rec((p1[0], p1[1], z), (p0[0], p0[1], z)))
    recs = np.stack(recs)
    wepl = rng.uniform(1, 2, len(recs))
    so, co = oracle.fbp_bin(recs, wepl, go)
    sg, cg = _gpu_bin(ntvs, torch, gd, recs, wepl)
    assert co.sum() == len(recs)
    assert np.array_equal(cg, co)
    assert np.allclose(sg, so, rtol=1e-14, atol=0.0)


def _synthetic(n_hist, seed=11, nx=48, nz=3, n_angles=60, curved=True):
    sp = synth.spec_scaled_3d(nx=nx, ny=nx, nz=nz, n_hist=n_hist, n_angles=n_angles, n_blocks=5, seed=seed,
                              curved=curved)
    return sp, synth.generate_paths(sp)


def _matched_geom(ntvs, sp, dt=0.75, n_t=56):
    # projection angles a * 360/n_angles fold onto multiples of 360/n_angles degrees: put
    # the angle-bin centres there (theta0 = minus half a bin)
    n_theta = sp.n_angles // 2
    th0 = -0.5 * math.pi / n_theta
    return _geoms(ntvs, nx=sp.nx, ny=sp.ny, nz=sp.nz, dx=sp.dx, dy=sp.dy, dz=sp.dz, n_theta=n_theta, n_t=n_t, dt=dt,
                  theta0=th0)


def test_bin_synthetic_with_ragged_tail(ntvs, torch):
    sp, P = _synthetic(60_001)
    go, gd = _matched_geom(ntvs, sp)
    so, co = oracle.fbp_bin(P.paths, P.b, go)
    sg, cg = _gpu_bin(ntvs, torch, gd, P.paths, P.b)
    assert np.array_equal(cg, co)
    assert co.sum() > 0.9 * P.M
    assert np.allclose(sg, so, rtol=1e-14, atol=0.0)


def test_bin_no_histories(ntvs, torch):
    _, gd = _geoms(ntvs, nx=4, ny=4, nz=1, dx=1.0, dy=1.0, dz=1.0, n_theta=3, n_t=5, dt=1.0)
    sino = torch.full((15,), 7.0, dtype=torch.float64, device="cuda")
    cnt = torch.full((15,), 7, dtype=torch.int32, device="cuda")
    ntvs.ntvs_fbp_bin(gd, torch.empty((0, 10), dtype=torch.float32, device="cuda"),
                      torch.empty(0, dtype=torch.float64, device="cuda"), sino, cnt)
    torch.cuda.synchronize()
    assert torch.all(sino == 0).item() and torch.all(cnt == 0).item()


@pytest.mark.parametrize("nz,n_theta,n_t", [(2, 7, 333), (1, 2, 8192), (3, 5, 1)])
def test_filter_parity(ntvs, torch, nz, n_theta, n_t):
    go, gd = _geoms(ntvs, nx=4, ny=4, nz=nz, dx=1.0, dy=1.0, dz=1.0, n_theta=n_theta, n_t=n_t, dt=0.7)
    p = np.random.default_rng(n_t).standard_normal((nz, n_theta, n_t)) + 3.0
    qo = oracle.fbp_filter(p, go)
    q = torch.empty(p.size, dtype=torch.float64, device="cuda")
    ntvs.ntvs_fbp_filter(gd, _dev(torch, p.reshape(-1), torch.float64), q)
    torch.cuda.synchronize()
    qg = q.cpu().numpy().reshape(p.shape)
    scale = np.abs(qo).max(axis=-1, keepdims=True)
    assert np.all(np.abs(qg - qo) <= 1e-13 * scale)


@pytest.mark.parametrize("n_theta,theta0", [(45, 0.3), (4096, -0.01)])
def test_backproject_parity(ntvs, torch, n_theta, theta0):
    nx, ny, nz = (37, 29, 3) if n_theta < 1000 else (20, 12, 1)
    go, gd = _geoms(ntvs, nx=nx, ny=ny, nz=nz, dx=0.8, dy=1.1, dz=2.0, n_theta=n_theta, n_t=64, dt=0.9,
                    theta0=theta0)
    q = np.random.default_rng(n_theta).standard_normal((nz, n_theta, 64))
    fo = oracle.fbp_backproject(q, go)
    img = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
    ntvs.ntvs_fbp_backproject(gd, _dev(torch, q.reshape(-1), torch.float64), img)
    torch.cuda.synchronize()
    fg = img.cpu().numpy()
    assert np.abs(fg - fo).max() <= 1e-12 * np.abs(fo).max()


@pytest.mark.parametrize("radius", [0, 1, 2, 3])
@pytest.mark.parametrize("ball", [False, True])
@pytest.mark.parametrize("hull", [False, True])
def test_median_parity_exact(ntvs, torch, radius, ball, hull):
    nx, ny, nz = 23, 17, 6
    rng = np.random.default_rng(100 * radius + 10 * ball + hull)
    x = np.round(rng.standard_normal(nx * ny * nz) * 4.0) / 4.0      # many ties
    x[rng.integers(0, x.size, 40)] = -0.0
    ref = oracle.median(x, (nx, ny, nz), radius, ball=ball) if radius > 0 else x.copy()
    if hull:
        ref = oracle.hull(ref, 0.25)
    out = torch.empty(x.size, dtype=torch.float64, device="cuda")
    ntvs.ntvs_median_filter(_dev(torch, x, torch.float64), out, (nx, ny, nz), radius, ball=ball, use_hull=hull,
                            tau=0.25)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_median_single_voxel_and_line(ntvs, torch):
    for shape in ((1, 1, 1), (9, 1, 1), (1, 1, 7)):
        x = np.random.default_rng(sum(shape)).standard_normal(int(np.prod(shape)))
        for ball in (False, True):
            out = torch.empty(x.size, dtype=torch.float64, device="cuda")
            ntvs.ntvs_median_filter(_dev(torch, x, torch.float64), out, shape, 2, ball=ball)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), oracle.median(x, shape, 2, ball=ball))


def test_hull_parity(ntvs, torch):
    x = np.random.default_rng(3).standard_normal(10_001)
    t = _dev(torch, x, torch.float64)
    ntvs.ntvs_hull(t, 0.1)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), oracle.hull(x, 0.1))


def _chain_compare(ntvs, torch, go, gd, paths, wepl, r, ball, tau):
    raw = oracle.initial_iterate(paths, wepl, go, median_r=r, median_ball=ball, use_hull=False)
    ref = oracle.hull(raw, tau)
    V = gd.nx * gd.ny * gd.nz
    out = torch.empty(V, dtype=torch.float64, device="cuda")
    ntvs.ntvs_initial_iterate(gd, _dev(torch, paths, torch.float32), _dev(torch, wepl, torch.float64), out,
                              median_radius=r, median_ball=ball, use_hull=True, tau=tau)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    tol = 1e-12 * np.abs(raw).max()
    away = np.abs(raw - tau) > 10 * tol      # hull decisions within rounding of tau may differ
    assert np.all(np.abs(got[away] - ref[away]) <= tol)
    assert np.all((got[~away] == 0.0) | (np.abs(got[~away] - tau) <= 10 * tol))
    return got, ref


@pytest.mark.parametrize("r,ball", [(2, False), (2, True), (0, False)])
def test_initial_iterate_chain(ntvs, torch, r, ball):
    sp, P = _synthetic(80_000, seed=12, nx=40, nz=4)
    go, gd = _matched_geom(ntvs, sp, dt=1.0, n_t=40)
    got, ref = _chain_compare(ntvs, torch, go, gd, P.paths, P.b, r, ball, 0.5)
    assert np.count_nonzero(ref) > 0.3 * ref.size


def test_initial_iterate_rejects_a_small_workspace(ntvs, torch):
    _, gd = _geoms(ntvs, nx=8, ny=8, nz=1, dx=1.0, dy=1.0, dz=1.0, n_theta=4, n_t=8, dt=1.0)
    need = ntvs.ntvs_fbp_workspace_bytes(gd)
    ws = torch.empty(need - 1, dtype=torch.uint8, device="cuda")
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    with pytest.raises(ntvs.NtvsError) as e:
        ntvs.ntvs_initial_iterate(gd, torch.zeros((1, 10), dtype=torch.float32, device="cuda"),
                                  torch.zeros(1, dtype=torch.float64, device="cuda"), out, workspace=ws)
    assert e.value.code == ntvs._ffi.NTVS_ERR_ARG


def test_initial_iterate_full_ctp404_size(ntvs, torch):
    """The CTP404 workload: 10M bent histories over 360 angles, 200x200x16 voxels of
    1x1x2.5 mm, 180 angle bins centred on whole degrees, 160 lateral bins of 1 mm."""
    sp = synth.spec_ctp404_3d()
    P = synth.generate_paths(sp)
    go, gd = _geoms(ntvs, nx=sp.nx, ny=sp.ny, nz=sp.nz, dx=sp.dx, dy=sp.dy, dz=sp.dz, n_theta=180, n_t=160, dt=1.0,
                    theta0=-math.pi / 360)
    so, co = oracle.fbp_bin(P.paths, P.b, go)
    sg, cg = _gpu_bin(ntvs, torch, gd, P.paths, P.b)
    assert np.array_equal(cg, co)
    assert np.allclose(sg, so, rtol=1e-14, atol=0.0)
    got, ref = _chain_compare(ntvs, torch, go, gd, P.paths, P.b, 2, False, 0.3)
    # the phantom's background (RSP 1) comes back near 1 inside the cylinder
    L = P.label.reshape(sp.nz, sp.ny, sp.nx)
    inner = L == len(sp.inserts)
    assert abs(np.median(got.reshape(L.shape)[inner]) - 1.0) < 0.05
