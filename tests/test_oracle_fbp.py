"""Pins of the initial-iterate oracle (FBP, median filter, hull), fixed by what the
mathematics and hand computation give rather than by the oracle itself.

  * Analytic projections of discs (the Radon transform of a disc of radius R is
    2 rho sqrt(R^2 - (t - c . n_theta)^2)) reconstruct to the disc: the interior level,
    the exterior, the centroid of an off-centre disc (a transposed or sign-flipped
    coordinate moves it), the level scale (a dropped dt or pi/n_theta changes it).
  * The discrete Ram-Lak kernel sums to zero over all lags (its DC gain is 0).
  * Hand-placed chords fall into bins worked out by hand, reversed chords (the fold by
    pi) included, and the bin mean and count of shared bins.
  * Median filter: constants, a lone outlier, a linear ramp (point-symmetric window),
    a corner pixel worked by hand, and scipy's median filter on interior voxels.
  * End to end: noise-free straight histories through the synthetic phantom reconstruct
    to its RSPs.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def disc_sinogram(g, discs):
    """Point samples of the Radon transform of discs (cx, cy, R, rho) at the bin centres."""
    th = g.theta0 + (np.arange(g.n_theta) + 0.5) * math.pi / g.n_theta
    t = (np.arange(g.n_t) + 0.5 - g.n_t / 2) * g.dt
    p = np.zeros((g.nz, g.n_theta, g.n_t))
    for cx, cy, R, rho in discs:
        s = t[None, :] - (cx * np.cos(th)[:, None] + cy * np.sin(th)[:, None])
        p[:] += 2.0 * rho * np.sqrt(np.clip(R * R - s * s, 0.0, None))
    return p


def _grid(g):
    x = (np.arange(g.nx) + 0.5) * g.dx - 0.5 * g.nx * g.dx
    y = (np.arange(g.ny) + 0.5) * g.dy - 0.5 * g.ny * g.dy
    return np.meshgrid(x, y)


@pytest.mark.parametrize("disc", [(0.0, 0.0, 30.0, 1.0), (20.0, -10.0, 15.0, 1.0), (-12.0, 25.0, 10.0, 2.5)])
def test_disc_reconstructs_to_the_disc(disc):
    g = oracle.fbp_geom(128, 128, 1, 1.0, 1.0, 1.0, 180, 400, 0.5)
    img = oracle.fbp_backproject(oracle.fbp_filter(disc_sinogram(g, [disc]), g), g).reshape(g.ny, g.nx)
    X, Y = _grid(g)
    cx, cy, R, rho = disc
    r = np.hypot(X - cx, Y - cy)
    inside = img[r < R - 3]
    outside = img[(r > R + 3) & (np.hypot(X, Y) < 60)]
    assert abs(inside.mean() / rho - 1.0) < 2e-3
    assert np.abs(inside / rho - 1.0).max() < 5e-3
    assert np.abs(outside / rho).max() < 0.1
    m = img > 0.5 * rho
    w = img * m
    assert abs((w * X).sum() / w.sum() - cx) < 0.03
    assert abs((w * Y).sum() / w.sum() - cy) < 0.03


def test_disc_level_does_not_depend_on_the_bin_width():
    # a dropped dt in the filter or in the interpolation changes the level with dt
    levels = []
    for dt, nt in ((0.5, 400), (1.0, 200), (2.0, 100)):
        g = oracle.fbp_geom(96, 96, 1, 1.0, 1.0, 1.0, 90, nt, dt)
        img = oracle.fbp_backproject(oracle.fbp_filter(disc_sinogram(g, [(0.0, 0.0, 35.0, 1.0)]), g), g)
        X, Y = _grid(g)
        levels.append(img.reshape(g.ny, g.nx)[np.hypot(X, Y) < 20].mean())
    assert np.allclose(levels, 1.0, atol=6e-3), levels


def test_disc_with_a_shifted_angle_origin():
    # theta0 shifts where the angle bins sit; the sinogram sampled there still reconstructs
    g = oracle.fbp_geom(96, 96, 1, 1.0, 1.0, 1.0, 120, 300, 0.5, theta0=-0.3)
    img = oracle.fbp_backproject(oracle.fbp_filter(disc_sinogram(g, [(15.0, 5.0, 12.0, 1.0)]), g), g)
    X, Y = _grid(g)
    img = img.reshape(g.ny, g.nx)
    assert abs(img[np.hypot(X - 15, Y - 5) < 9].mean() - 1.0) < 3e-3
    w = img * (img > 0.5)
    assert abs((w * X).sum() / w.sum() - 15.0) < 0.03 and abs((w * Y).sum() / w.sum() - 5.0) < 0.03


def test_two_slices_are_reconstructed_independently():
    g = oracle.fbp_geom(64, 64, 2, 1.0, 1.0, 2.5, 90, 200, 0.5)
    p = disc_sinogram(g, [(0.0, 0.0, 20.0, 1.0)])
    p[1] *= 0.0
    img = oracle.fbp_backproject(oracle.fbp_filter(p, g), g).reshape(2, 64, 64)
    assert np.all(img[1] == 0.0)
    X, Y = _grid(g)
    assert abs(img[0][np.hypot(X, Y) < 15].mean() - 1.0) < 3e-3


def test_ramlak_kernel_has_zero_dc_gain():
    # 1/4 - (2/pi^2) sum_{odd m > 0} 1/m^2 = 1/4 - (2/pi^2)(pi^2/8) = 0 (per dt^2)
    dt = 0.7
    s = sum(oracle.ramlak(m, dt) for m in range(-200001, 200002))
    assert abs(s) * dt * dt < 2e-6
    assert oracle.ramlak(0, dt) == pytest.approx(1.0 / (4 * dt * dt))
    assert oracle.ramlak(2, dt) == 0.0 and oracle.ramlak(-4, dt) == 0.0
    assert oracle.ramlak(3, dt) == pytest.approx(-1.0 / (9 * math.pi ** 2 * dt * dt))
    assert oracle.ramlak(-3, dt) == oracle.ramlak(3, dt)


def _rec(p, q):
    return np.array([p[0], p[1], p[2], q[0], q[1], q[2], 0, 0, 0, 0], np.float32)


# 5 angle bins of 36 degrees, 10 lateral bins of 2 mm (t in [-10, 10)), 2 slices of 2.5 mm
G = oracle.fbp_geom(8, 8, 2, 1.0, 1.0, 2.5, 5, 10, 2.0)


def test_chord_lines_worked_by_hand():
    # horizontal chord y = 5 left to right: normal (0, 1), theta = pi/2, t = 5
    th, t, z = oracle.fbp_line(_rec((-100, 5, 1.0), (100, 5, 1.0)))
    assert th == pytest.approx(math.pi / 2) and t == pytest.approx(5.0) and z == pytest.approx(1.0)
    # the same line right to left: normal (0, -1) at 3pi/2, folded to pi/2 with t negated
    th, t, _ = oracle.fbp_line(_rec((100, 5, 1.0), (-100, 5, 1.0)))
    assert th == pytest.approx(math.pi / 2) and t == pytest.approx(5.0)
    # vertical chord x = 3 upwards: normal (-1, 0) at pi, folded to 0 with t = 3
    th, t, _ = oracle.fbp_line(_rec((3, -100, 3.0), (3, 100, 3.0)))
    assert th == pytest.approx(0.0, abs=1e-15) and t == pytest.approx(3.0)
    # y = x + 10: normal at 3pi/4, distance 10/sqrt(2) from the origin
    th, t, _ = oracle.fbp_line(_rec((-50, -40, 0.5), (50, 60, 0.5)))
    assert th == pytest.approx(3 * math.pi / 4) and t == pytest.approx(10 / math.sqrt(2))
    # entry and exit at different heights: z is their mean
    assert oracle.fbp_line(_rec((-10, 0, 1.0), (10, 0, 2.0)))[2] == pytest.approx(1.5)
    assert oracle.fbp_line(np.zeros(10, np.float32)) is None


def test_bins_worked_by_hand():
    assert oracle.fbp_bin_of(_rec((-100, 5, 1.0), (100, 5, 1.0)), G) == (0, 2, 7)   # 90 deg, u = 7.5
    assert oracle.fbp_bin_of(_rec((100, 5, 1.0), (-100, 5, 1.0)), G) == (0, 2, 7)
    assert oracle.fbp_bin_of(_rec((3, -100, 3.0), (3, 100, 3.0)), G) == (1, 0, 6)   # 0 deg, u = 6.5
    assert oracle.fbp_bin_of(_rec((-50, -40, 0.5), (50, 60, 0.5)), G) == (0, 3, 8)  # 135 deg, u = 8.54
    # normal at 170 degrees and its reverse (normal at -10 degrees): last bin, same t
    d = (math.cos(math.radians(80)), math.sin(math.radians(80)))
    n = (math.cos(math.radians(170)), math.sin(math.radians(170)))
    p0 = (4.6 * n[0] - 60 * d[0], 4.6 * n[1] - 60 * d[1], 4.0)
    p1 = (4.6 * n[0] + 60 * d[0], 4.6 * n[1] + 60 * d[1], 4.0)
    assert oracle.fbp_bin_of(_rec(p0, p1), G) == (1, 4, 7)   # t = 4.6: u = 7.3
    assert oracle.fbp_bin_of(_rec(p1, p0), G) == (1, 4, 7)
    # the lateral range is half open: t = -10 (u = 0) is in bin 0, t = +10 (u = 10) is out
    assert oracle.fbp_bin_of(_rec((100, -10, 1.0), (-100, -10, 1.0)), G) == (0, 2, 0)
    assert oracle.fbp_bin_of(_rec((-100, 10, 1.0), (100, 10, 1.0)), G) is None
    # outside: |t| beyond the bins, z above the slices, empty record
    assert oracle.fbp_bin_of(_rec((-100, 50, 1.0), (100, 50, 1.0)), G) is None
    assert oracle.fbp_bin_of(_rec((-100, 0, 6.0), (100, 0, 6.0)), G) is None
    assert oracle.fbp_bin_of(_rec((-100, 0, -0.5), (100, 0, -0.5)), G) is None
    assert oracle.fbp_bin_of(np.zeros(10, np.float32), G) is None


def test_angle_origin_moves_the_bins():
    # theta0 = -18 deg: bin a covers [-18 + 36a, 18 + 36a) deg; a normal at 170 deg is
    # 188 deg past theta0, i.e. 8 deg with t negated: bin 0
    g = oracle.fbp_geom(8, 8, 2, 1.0, 1.0, 2.5, 5, 10, 2.0, theta0=-math.radians(18))
    d = (math.cos(math.radians(80)), math.sin(math.radians(80)))
    n = (math.cos(math.radians(170)), math.sin(math.radians(170)))
    p0 = (4.6 * n[0] - 60 * d[0], 4.6 * n[1] - 60 * d[1], 1.0)
    p1 = (4.6 * n[0] + 60 * d[0], 4.6 * n[1] + 60 * d[1], 1.0)
    assert oracle.fbp_bin_of(_rec(p0, p1), g) == (0, 0, 2)    # rebased to 8 deg, t = -4.6: u = 2.7
    assert oracle.fbp_bin_of(_rec((-100, 5, 1.0), (100, 5, 1.0)), g) == (0, 3, 7)   # 90 deg: [90, 126)
    # theta0 = +18 deg: a normal at 10 deg is 8 deg before theta0, i.e. 172 deg past it with t
    # negated (bin 4 covers [162, 198) deg); t = 4.6 becomes -4.6: u = 2.7
    g = oracle.fbp_geom(8, 8, 2, 1.0, 1.0, 2.5, 5, 10, 2.0, theta0=math.radians(18))
    d = (math.cos(math.radians(100)), math.sin(math.radians(100)))
    n = (math.cos(math.radians(10)), math.sin(math.radians(10)))
    p0 = (4.6 * n[0] - 60 * d[0], 4.6 * n[1] - 60 * d[1], 1.0)
    p1 = (4.6 * n[0] + 60 * d[0], 4.6 * n[1] + 60 * d[1], 1.0)
    assert oracle.fbp_bin_of(_rec(p0, p1), g) == (0, 4, 2)
    assert oracle.fbp_bin_of(_rec(p1, p0), g) == (0, 4, 2)


def test_bin_means_and_counts():
    recs = np.stack([_rec((-100, 5, 1.0), (100, 5, 1.0)), _rec((100, 5.5, 1.2), (-100, 5.5, 1.2)),
                     _rec((3, -100, 3.0), (3, 100, 3.0)), _rec((-100, 50, 1.0), (100, 50, 1.0)),
                     np.zeros(10, np.float32)])
    wepl = np.array([2.0, 4.0, 7.0, 100.0, 100.0])
    sino, cnt = oracle.fbp_bin(recs, wepl, G)
    assert cnt.sum() == 3
    assert cnt[0, 2, 7] == 2 and sino[0, 2, 7] == 3.0
    assert cnt[1, 0, 6] == 1 and sino[1, 0, 6] == 7.0
    others = np.ones_like(cnt, bool)
    others[0, 2, 7] = others[1, 0, 6] = False
    assert np.all(sino[others] == 0.0) and np.all(cnt[others] == 0)


# ------------------------------------------------------------------ median filter
def test_median_windows():
    w2 = oracle.median_window(2, False)
    assert len(w2) == 21 and np.all(w2[:, 2] == 0)
    assert len(oracle.median_window(1, False)) == 9     # r^2 + 1 = 2: the 3x3 square
    assert len(oracle.median_window(2, True)) == 57
    assert len(oracle.median_window(0, False)) == 1


def test_median_constant_and_outlier():
    x = np.full((1, 7, 7), 3.0)
    assert np.all(oracle.median(x, (7, 7, 1), 2) == 3.0)
    x[0, 3, 3] = 100.0
    assert np.all(oracle.median(x, (7, 7, 1), 2) == 3.0)
    x[0, 0, 0] = -50.0   # a corner outlier too: its window holds 8 values, 7 of them 3
    assert np.all(oracle.median(x, (7, 7, 1), 2) == 3.0)


def test_median_keeps_a_linear_ramp_inside():
    ix, iy = np.meshgrid(np.arange(9.0), np.arange(9.0))
    x = (ix + 2.0 * iy)[None]
    out = oracle.median(x, (9, 9, 1), 2).reshape(9, 9)
    assert np.array_equal(out[2:-2, 2:-2], x[0, 2:-2, 2:-2])


def test_median_corner_worked_by_hand():
    # 5x5 values ix + 5 iy: the corner's in-image window is (0,0),(1,0),(2,0),(0,1),(1,1),
    # (2,1),(0,2),(1,2) -> 0,1,2,5,6,7,10,11; element 8//2 = 4 of the sorted list is 6
    ix, iy = np.meshgrid(np.arange(5.0), np.arange(5.0))
    out = oracle.median((ix + 5 * iy)[None], (5, 5, 1), 2).reshape(5, 5)
    assert out[0, 0] == 6.0
    # (4, 0): window (0,0),(-1,0),(-2,0),(0,1),(-1,1),(-2,1),(0,2),(-1,2)
    # -> 4,3,2,9,8,7,14,13 sorted 2,3,4,7,8,9,13,14 -> 8
    assert out[0, 4] == 8.0


def test_median_slices_do_not_mix_in_2d_but_do_in_3d():
    x = np.zeros((3, 6, 6))
    x[1] = 1.0
    assert np.array_equal(oracle.median(x, (6, 6, 3), 2).reshape(3, 6, 6), x)
    # 3D: a voxel of the middle slice sees 21 ones and 36 zeros
    assert np.all(oracle.median(x, (6, 6, 3), 2, ball=True).reshape(3, 6, 6)[1, 2:4, 2:4] == 0.0)


@pytest.mark.parametrize("ball", [False, True])
def test_median_matches_scipy_inside(ball):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(4)
    nx, ny, nz = 17, 13, 7
    x = rng.standard_normal((nz, ny, nx))
    out = oracle.median(x, (nx, ny, nz), 2, ball=ball).reshape(nz, ny, nx)
    o = np.arange(-2, 3)
    OZ, OY, OX = np.meshgrid(o if ball else np.zeros(1, int), o, o, indexing="ij")
    fp = (OX ** 2 + OY ** 2 + OZ ** 2 <= 5)
    ref = ndimage.median_filter(x, footprint=fp, mode="constant")
    zs = slice(2, -2) if ball else slice(None)
    assert np.array_equal(out[zs, 2:-2, 2:-2], ref[zs, 2:-2, 2:-2])


def test_hull():
    x = np.array([-1.0, 0.0, 0.05, 0.1, 0.2, 1.0])
    assert np.array_equal(oracle.hull(x, 0.1), [0.0, 0.0, 0.0, 0.0, 0.2, 1.0])
    assert np.array_equal(oracle.hull(x, -5.0), x)


# ------------------------------------------------------------------ end to end
def test_noise_free_phantom_reconstructs_to_its_rsps():
    ndimage = pytest.importorskip("scipy.ndimage")
    sp = synth.spec_scaled_3d(nx=64, ny=64, nz=2, n_hist=100_000, n_angles=90, n_blocks=5, seed=7,
                              curved=False).replace(noise_sigma=0.0)
    P = synth.generate_paths(sp)
    # 90 angles over a full turn fold onto 45 line directions at 2 + 4a degrees: the bin centres
    g = oracle.fbp_geom(sp.nx, sp.ny, sp.nz, sp.dx, sp.dy, sp.dz, 45, 64, 1.0)
    sino, cnt = oracle.fbp_bin(P.paths, P.b, g)
    assert cnt.sum() == P.M and (cnt[:, :, 8:56] == 0).sum() == 0
    img = oracle.initial_iterate(P.paths, P.b, g, median_r=0).reshape(sp.nz, sp.ny, sp.nx)
    L = P.label.reshape(sp.nz, sp.ny, sp.nx)
    nins = len(sp.inserts)
    bg = np.stack([ndimage.binary_erosion(L[z] == nins, iterations=2) for z in range(sp.nz)])
    assert abs(img[bg].mean() - 1.0) < 0.01
    for i, ins in enumerate(sp.inserts):
        m = np.stack([ndimage.binary_erosion(L[z] == i, iterations=1) for z in range(sp.nz)])
        assert abs(img[m].mean() - ins.rsp) < 0.1, (i, ins.rsp, img[m].mean())
    # the median filter and the hull keep the interior level and clear the air around it
    img2 = oracle.initial_iterate(P.paths, P.b, g, median_r=2, use_hull=True, tau=0.5)
    img2 = img2.reshape(sp.nz, sp.ny, sp.nx)
    assert abs(img2[bg].mean() - 1.0) < 0.01
    far = np.stack([ndimage.binary_erosion(L[z] == -1, iterations=3) for z in range(sp.nz)])
    assert np.all(img2[far] == 0.0)
