"""The seeded input generator: geometry, determinism and consistency of the synthetic systems."""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _chord(t, theta, hx, hy):
    """length of the line {t n + s u} inside the square [-hx,hx] x [-hy,hy]"""
    u = np.array([math.cos(theta), math.sin(theta)])
    n = np.array([-math.sin(theta), math.cos(theta)])
    p = t * n
    lo, hi = -np.inf, np.inf
    for a, h in ((0, hx), (1, hy)):
        if abs(u[a]) < 1e-15:
            if abs(p[a]) > h:
                return 0.0
            continue
        s0, s1 = sorted(((-h - p[a]) / u[a], (h - p[a]) / u[a]))
        lo, hi = max(lo, s0), min(hi, s1)
    return max(0.0, hi - lo)


def test_straight_rows_sum_to_chord_length():
    s = synth.generate(synth.spec_slice_2d())
    rl = np.add.reduceat(s.val, s.row_ptr[:-1])
    hx = hy = 16.0
    for r in range(0, s.M, 113):
        th = math.radians(360.0 * s.angle[r] / s.spec.n_angles)
        assert rl[r] == pytest.approx(_chord(s.t[r], th, hx, hy), abs=1e-9 + 40 * s.spec.min_len)


def test_rows_are_valid_csr():
    s = synth.generate(synth.spec_scaled_3d(n_hist=5000))
    assert s.row_ptr[0] == 0 and np.all(np.diff(s.row_ptr) >= 0)
    assert s.col.min() >= 0 and s.col.max() < s.spec.V
    assert s.val.min() >= s.spec.min_len
    for r in range(0, s.M, 7):
        c = s.col[s.row_ptr[r]:s.row_ptr[r + 1]]
        assert np.unique(c).size == c.size


def test_noise_free_wepl_is_line_integral():
    sp = synth.spec_scaled_3d(n_hist=3000).replace(noise_sigma=0.0)
    s = synth.generate(sp)
    np.testing.assert_allclose(np.add.reduceat(s.val * s.xstar[s.col], s.row_ptr[:-1]), s.b, rtol=1e-12)


def test_bent_paths_stay_near_the_chord():
    sp = synth.spec_scaled_3d(nx=60, ny=60, nz=6, n_hist=2000)
    s = synth.generate(sp)
    hw = 0.5 * math.sqrt(sp.dx ** 2 + sp.dy ** 2)
    for r in range(0, s.M, 37):
        th = math.radians(360.0 * s.angle[r] / sp.n_angles)
        c = s.col[s.row_ptr[r]:s.row_ptr[r + 1]]
        ix, iy = c % sp.nx, (c // sp.nx) % sp.ny
        xc = -0.5 * sp.nx * sp.dx + (ix + 0.5) * sp.dx
        yc = -0.5 * sp.ny * sp.dy + (iy + 0.5) * sp.dy
        lat = -math.sin(th) * xc + math.cos(th) * yc - s.t[r]
        assert np.max(np.abs(lat)) <= sp.dev_max + hw + 1e-9
        iz = c // (sp.nx * sp.ny)
        zc = (iz + 0.5) * sp.dz
        assert np.max(np.abs(zc - s.z[r])) <= sp.dev_max + 0.5 * sp.dz + 1e-9


def test_rows_in_angle_then_slice_then_lateral_order():
    s = synth.generate(synth.spec_scaled_3d(n_hist=4000))
    assert np.all(np.diff(s.angle) >= 0)
    key = s.angle.astype(np.int64) * 10**6 + np.floor(s.z / s.spec.dz).astype(np.int64)
    assert np.all(np.diff(key) >= 0)


def test_generator_does_not_depend_on_thread_count():
    code = ("import synth, hashlib; s = synth.generate(synth.spec_scaled_3d(n_hist=3000)); "
            "print(hashlib.sha256(s.col.tobytes() + s.val.tobytes() + s.b.tobytes()).hexdigest())")
    out = []
    for th in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=th)
        out.append(subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, check=True,
                                  capture_output=True, text=True).stdout.strip())
    assert out[0] == out[1]


def test_phantom_values_and_labels():
    sp = synth.spec_slice_2d()
    xs, xb, lab = synth.phantom(sp)
    assert set(np.unique(lab)) == {-1, 0, 1, 2, 3, 4}
    assert np.all(xb[lab >= 0] == 1.0) and np.all(xb[lab < 0] == 0.0)
    iy, ix = np.meshgrid(np.arange(sp.ny), np.arange(sp.nx), indexing="ij")
    xc = (-0.5 * sp.nx + ix.reshape(-1) + 0.5) * sp.dx
    yc = (-0.5 * sp.ny + iy.reshape(-1) + 0.5) * sp.dy
    for i, ins in enumerate(sp.inserts):   # the voxel at an insert's centre lies wholly inside it
        j = np.argmin((xc - ins.cx) ** 2 + (yc - ins.cy) ** 2)
        assert lab[j] == i
        assert xs[j] == pytest.approx(ins.rsp, abs=1e-12)


def test_row_range_equals_slice_of_whole_system():
    sp = synth.spec_scaled_3d(n_hist=5000)
    whole = synth.generate(sp)
    part = synth.generate(sp, rows=(1200, 3100))
    p0, p1 = whole.row_ptr[1200], whole.row_ptr[3100]
    np.testing.assert_array_equal(part.row_ptr, whole.row_ptr[1200:3101] - p0)
    np.testing.assert_array_equal(part.col, whole.col[p0:p1])
    np.testing.assert_array_equal(part.val, whole.val[p0:p1])
    np.testing.assert_array_equal(part.b, whole.b[1200:3100])


def test_path_records_match_the_traced_rows():
    """A path record re-traced on the CPU (a plain polyline walk) gives the generator's row."""
    sp = synth.spec_scaled_3d(nx=30, ny=26, nz=4, n_hist=400)
    s = synth.generate(sp)
    pr = synth.generate_paths(sp)
    np.testing.assert_allclose(pr.b, s.b, rtol=1e-12)
    o = np.array([-0.5 * sp.nx * sp.dx, -0.5 * sp.ny * sp.dy, 0.0])
    h = np.array([sp.dx, sp.dy, sp.dz])
    n = np.array([sp.nx, sp.ny, sp.nz])
    for r in range(0, s.M, 23):
        p = pr.paths[r].astype(np.float64)
        P, Q, A = p[0:3], p[3:6], p[6:10]
        u = (Q[:2] - P[:2]) / np.linalg.norm(Q[:2] - P[:2])
        nv = np.array([-u[1], u[0], 0.0])
        sg = np.linspace(0.0, 1.0, sp.n_seg + 1)
        h10, h11 = sg ** 3 - 2 * sg ** 2 + sg, sg ** 3 - sg ** 2
        pts = P[None] + sg[:, None] * (Q - P)[None] + (A[0] * h10 + A[1] * h11)[:, None] * nv[None]
        pts[:, 2] += A[2] * h10 + A[3] * h11
        acc = {}
        for a, bq in zip(pts[:-1], pts[1:]):   # fine sampling of each segment
            ts = np.linspace(0.0, 1.0, 4001)
            mid = a[None] + ((ts[:-1] + ts[1:]) / 2)[:, None] * (bq - a)[None]
            idx = np.floor((mid - o) / h).astype(int)
            ok = np.all((idx >= 0) & (idx < n), axis=1)
            seg_len = np.linalg.norm(bq - a) / 4000
            for j in ((idx[ok, 2] * sp.ny + idx[ok, 1]) * sp.nx + idx[ok, 0]):
                acc[j] = acc.get(j, 0.0) + seg_len
        cols = s.col[s.row_ptr[r]:s.row_ptr[r + 1]]
        vals = s.val[s.row_ptr[r]:s.row_ptr[r + 1]]
        assert np.sum(vals) == pytest.approx(sum(acc.values()), rel=2e-3, abs=2e-3)
        big = {j for j, v in acc.items() if v > 0.05}
        assert big <= set(cols.tolist())
