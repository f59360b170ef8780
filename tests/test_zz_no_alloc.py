"""The allocation-free TV entry point (ntvs_tv_value_static).

For callers that cannot allocate device memory -- code inside host callbacks or framework
hooks where allocation is forbidden, or under an allocator that must own every device
allocation -- the library offers phi(x) on caller-owned device buffers, with its reduction
scratch in a static device array.  This file checks it through the C ABI against the
context-based ntvs_get_tv, on two calls in a row (the second call sees the scratch the
first one left behind), and that images beyond the scratch limit are rejected.  It is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from _gpu_util import empty_system, ntvs_module

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(200, 200, 16), (33, 17, 5), (1, 1, 1), (256, 256, 256)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_static_scratch_tv_matches_context_tv(shape, dtype):
    ntvs = ntvs_module()
    import torch
    from paper_1803_01112_gb300 import _ffi
    V = int(np.prod(shape))
    x = np.random.default_rng(V).uniform(0.0, 2.0, size=V).astype(dtype)
    r = empty_system(ntvs, shape)
    try:
        r.set_image(x)
        want = r.tv()
    finally:
        r.close()
    xd = torch.from_numpy(x).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = _ffi.NTVS_F64 if dtype == np.float64 else _ffi.NTVS_F32
    for _ in range(2):
        out.fill_(-1.0)
        torch.cuda.synchronize()
        rc = ntvs.lib().ntvs_tv_value_static(ctypes.c_void_p(xd.data_ptr()), code, shape[0], shape[1], shape[2],
                                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == _ffi.NTVS_OK, ntvs.ntvs_last_error()
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_static_scratch_rejects_images_beyond_its_limit():
    ntvs = ntvs_module()
    import torch
    from paper_1803_01112_gb300 import _ffi
    xd = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 257 x 256 x 256 voxels is one slice past the 16,777,216-voxel limit; nothing is read
    rc = ntvs.lib().ntvs_tv_value_static(ctypes.c_void_p(xd.data_ptr()), _ffi.NTVS_F64, 256, 256, 257,
                                         ctypes.c_void_p(out.data_ptr()), None)
    assert rc == _ffi.NTVS_ERR_ARG
    assert "exceeds the static scratch limit" in ntvs.ntvs_last_error()
