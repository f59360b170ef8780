"""Pins of the oracle's TV value and gradient (phi = TV, Sec. II; v = -grad/||grad||, Appendix A).

Nothing here re-types the oracle's stencil: each check is a closed form, an invariant,
a hand expansion (tests/golden/tv_2x2.json) or a finite-difference derivative.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_constant_image_has_zero_tv():
    for shape in [(1, 1, 1), (7, 1, 1), (5, 4, 1), (4, 3, 5)]:
        x = np.full(int(np.prod(shape)), 1.37)
        assert oracle.tv(x, shape) == 0.0


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_step_edge_closed_form(axis):
    # a plane step of height h: one nonzero forward difference per line crossing the plane
    nx, ny, nz = 6, 5, 4
    n = (nx, ny, nz)
    h = -0.73
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = (ix, iy, iz)[axis]
    x = np.where(idx >= 3, h, 0.0).reshape(-1)
    lines = n[0] * n[1] * n[2] // n[axis]
    assert oracle.tv(x, n) == pytest.approx(abs(h) * lines, rel=1e-15)


def test_one_dimensional_tv_is_sum_of_absolute_jumps():
    rng = np.random.default_rng(0)
    x = rng.normal(size=17)
    assert oracle.tv(x, (17, 1, 1)) == pytest.approx(np.abs(np.diff(x)).sum(), rel=1e-14)
    # the same signal along y and along z
    assert oracle.tv(x, (1, 17, 1)) == pytest.approx(np.abs(np.diff(x)).sum(), rel=1e-14)
    assert oracle.tv(x, (1, 1, 17)) == pytest.approx(np.abs(np.diff(x)).sum(), rel=1e-14)


def test_homogeneity_and_shift_invariance():
    rng = np.random.default_rng(1)
    shape = (5, 4, 3)
    x = rng.uniform(0, 2, size=60)
    t = oracle.tv(x, shape)
    assert oracle.tv(-2.5 * x, shape) == pytest.approx(2.5 * t, rel=1e-14)
    assert oracle.tv(x + 11.0, shape) == pytest.approx(t, rel=1e-12)


def test_isotropic_not_anisotropic():
    # a diagonal ramp x = ix + iy: interior voxels have d = (1,1) -> sqrt(2), not 2
    nx = ny = 4
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = (ix + iy).astype(float).reshape(-1)
    # interior (ix<3, iy<3): sqrt2 each (9 voxels); ix=3, iy<3: d=(0,1) -> 1 (3 voxels);
    # iy=3, ix<3: d=(1,0) -> 1 (3 voxels); corner: 0
    assert oracle.tv(x, (nx, ny, 1)) == pytest.approx(9 * math.sqrt(2) + 6, rel=1e-14)


def test_hand_expanded_2x2():
    g = json.load(open(os.path.join(GOLD, "tv_2x2.json")))
    shape = tuple(g["shape"])
    x = np.array(g["x"])
    ev = lambda s: eval(s, {"sqrt": math.sqrt})
    assert oracle.tv(x, shape) == pytest.approx(ev(g["phi"]), rel=1e-15)
    grad = oracle.tv_grad(x, shape, 0.0)
    np.testing.assert_allclose(grad, [ev(s) for s in g["grad_eps0"]], rtol=1e-14, atol=1e-15)


def test_tv_eps_closed_form_on_constant():
    shape = (3, 2, 2)
    x = np.full(12, 4.0)
    eps = 1e-4
    assert oracle.tv(x, shape, eps) == pytest.approx(12 * math.sqrt(eps), rel=1e-14)


@pytest.mark.parametrize("shape", [(5, 4, 3), (6, 5, 1), (1, 1, 9), (3, 1, 4)])
def test_gradient_matches_central_differences(shape):
    rng = np.random.default_rng(sum(shape))
    V = int(np.prod(shape))
    x = rng.uniform(0, 2, size=V)
    eps = 1e-2
    g = oracle.tv_grad(x, shape, eps)
    h = 1e-6
    fd = np.empty(V)
    for q in range(V):
        xp = x.copy(); xp[q] += h
        xm = x.copy(); xm[q] -= h
        fd[q] = (oracle.tv(xp, shape, eps) - oracle.tv(xm, shape, eps)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7)


def test_gradient_of_constant_is_zero_and_sums_to_zero():
    shape = (4, 4, 2)
    assert np.all(oracle.tv_grad(np.full(32, 0.5), shape, 1e-8) == 0.0)
    x = np.random.default_rng(5).normal(size=32)
    # phi_eps(x + c) = phi_eps(x)  =>  sum_q g_q = 0
    assert abs(oracle.tv_grad(x, shape, 1e-8).sum()) < 1e-12


def test_gradient_2d_equals_3d_with_one_slice():
    # nz = 1 is the per-slice 2D form; a 3D volume of identical slices has the same
    # in-plane gradient per slice (z differences vanish)
    rng = np.random.default_rng(7)
    s = rng.uniform(size=20)
    g2 = oracle.tv_grad(s, (5, 4, 1), 1e-3)
    g3 = oracle.tv_grad(np.tile(s, 3), (5, 4, 3), 1e-3)
    for k in range(3):   # z differences are 0, so D and the in-plane terms are those of 2D
        np.testing.assert_allclose(g3[20 * k:20 * (k + 1)], g2, rtol=1e-13, atol=1e-15)
