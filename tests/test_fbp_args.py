"""Host-side checks of the initial-iterate entry points (include/ntvs_fbp.h): every invalid
argument is refused before any GPU work, so these run without a GPU."""
import ctypes

import pytest

from paper_1803_01112_gb300 import _build


@pytest.fixture(scope="module")
def L():
    _build.build()
    from paper_1803_01112_gb300 import _ffi
    return _ffi.lib()


def _g(**kw):
    from paper_1803_01112_gb300 import fbp_geom
    a = dict(nx=200, ny=200, nz=16, dx=1.0, dy=1.0, dz=2.5, n_theta=180, n_t=160, dt=1.0, theta0=0.0)
    a.update(kw)
    return fbp_geom(**a)


def test_workspace_bytes(L):
    S, V = 16 * 180 * 160, 200 * 200 * 16
    al = lambda b: (b + 255) // 256 * 256
    assert L.ntvs_fbp_workspace_bytes(ctypes.byref(_g())) == al(8 * S) + al(4 * S) + al(8 * S) + al(8 * V)
    assert L.ntvs_fbp_workspace_bytes(ctypes.byref(_g(nx=1, ny=1, nz=1, n_theta=1, n_t=1))) == 4 * 256


@pytest.mark.parametrize("bad", [dict(nx=0), dict(nz=-1), dict(n_theta=0), dict(n_t=0), dict(n_t=8193),
                                 dict(n_theta=4097), dict(nz=65536, nx=1, ny=1), dict(dx=0.0), dict(dt=-1.0),
                                 dict(dz=float("nan")), dict(theta0=float("inf")), dict(theta0=60.0),
                                 dict(nx=50000, ny=50000, nz=2)])
def test_invalid_geometry_is_refused(L, bad):
    from paper_1803_01112_gb300 import _ffi
    g = _g(**bad)
    assert L.ntvs_fbp_workspace_bytes(ctypes.byref(g)) == _ffi.NTVS_ERR_ARG
    assert L.ntvs_fbp_filter(ctypes.byref(g), 16, 4096, None) == _ffi.NTVS_ERR_ARG
    assert L.ntvs_fbp_backproject(ctypes.byref(g), 16, 4096, None) == _ffi.NTVS_ERR_ARG
    assert "ntvs_fbp_backproject" in L.ntvs_last_error().decode()


def test_reserved_field_must_be_zero(L):
    from paper_1803_01112_gb300 import _ffi
    g = _g()
    g.reserved = 1
    assert L.ntvs_fbp_workspace_bytes(ctypes.byref(g)) == _ffi.NTVS_ERR_ARG


def test_null_and_overlap_are_refused(L):
    from paper_1803_01112_gb300 import _ffi
    g = _g()
    ARG = _ffi.NTVS_ERR_ARG
    assert L.ntvs_fbp_workspace_bytes(None) == ARG
    assert L.ntvs_fbp_bin(ctypes.byref(g), None, None, 5, 256, 512, None) == ARG
    assert L.ntvs_fbp_bin(ctypes.byref(g), 256, 256, -1, 256, 512, None) == ARG
    assert L.ntvs_fbp_bin(ctypes.byref(g), 256, 256, 5, None, 512, None) == ARG
    assert L.ntvs_fbp_filter(ctypes.byref(g), None, 256, None) == ARG
    assert L.ntvs_fbp_filter(ctypes.byref(g), 4096, 4096 + 8, None) == ARG          # overlapping
    assert L.ntvs_median_filter(4096, 4096 + 8, 10, 10, 1, 2, 0, 0, 0.0, None) == ARG  # overlapping
    assert L.ntvs_median_filter(4096, 1 << 30, 10, 10, 1, 4, 0, 0, 0.0, None) == ARG   # radius 4
    assert L.ntvs_median_filter(4096, 1 << 30, 10, 10, 1, -1, 0, 0, 0.0, None) == ARG
    assert L.ntvs_median_filter(4096, 1 << 30, 0, 10, 1, 2, 0, 0, 0.0, None) == ARG
    assert L.ntvs_median_filter(4096, 1 << 30, 10, 10, 1, 2, 0, 1, float("nan"), None) == ARG
    assert L.ntvs_hull(None, 10, 0.0, None) == ARG
    assert L.ntvs_hull(4096, 0, 0.0, None) == ARG
    need = L.ntvs_fbp_workspace_bytes(ctypes.byref(g))
    assert L.ntvs_initial_iterate(ctypes.byref(g), 256, 256, 5, 2, 0, 0, 0.0, 4096, need - 1, 1 << 30, None) == ARG
    assert L.ntvs_initial_iterate(ctypes.byref(g), 256, 256, 5, 2, 0, 0, 0.0, 4096 + 16, need, 1 << 30, None) == ARG
    assert L.ntvs_initial_iterate(ctypes.byref(g), 256, 256, 5, 5, 0, 0, 0.0, 4096, need, 1 << 30, None) == ARG
    assert L.ntvs_initial_iterate(ctypes.byref(g), 256, 256, 5, 2, 0, 0, 0.0, None, need, 1 << 30, None) == ARG
