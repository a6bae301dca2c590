"""hm_matvec_host_noalloc: the allocation-free host-buffer product.

Callers that cannot let the library allocate device memory (a fully
pre-budgeted serving process; code that must not trigger cudaFree's device-wide
synchronisation) use this entry point; it stages x and y through libhm's fixed
device array instead of buffers it would allocate.  The test checks, through
the C ABI, that two calls in a row give the same result as the existing
hm_matvec entry point (within the 4*eps tolerance of the parity tests), and
that a request larger than the fixed array is refused.  The file is named to
be collected last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def hm():
    from paper_2405_03456_gb300 import build, hm as _hm
    build.build()
    _hm.load()
    return _hm


def _device_product(M, x, y0, alpha, beta):
    xd = torch.from_numpy(np.asfortranarray(x)).cuda()
    yd = torch.from_numpy(np.asfortranarray(y0.copy())).cuda()
    if xd.dim() == 2:
        xd = xd.t().contiguous().t()
        yd = yd.t().contiguous().t()
    M.matvec(alpha, xd, beta, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def test_noalloc_matches_matvec_twice(hm):
    n, eps = 2048, 1e-6
    pts = synth.sphere_points(n)
    M = hm.HMatrix(pts, "laplace", 32, 2.0, "h", eps)
    try:
        M.compress(eps, "aflp", True)
        cases = [(synth.rhs(n, 1, seed=11)[:, 0], synth.rhs(n, 1, seed=12)[:, 0], 1.0, 1.0),
                 (synth.rhs(n, 3, seed=13), synth.rhs(n, 3, seed=14), 0.5, -2.0)]
        for x, y0, alpha, beta in cases:          # two calls in a row, different data
            want = _device_product(M, x, y0, alpha, beta)
            got = np.asfortranarray(y0.copy())
            hm.hm_matvec_host_noalloc(M.h, alpha, np.asfortranarray(x), beta, got)
            assert np.linalg.norm(got - want) <= 4 * eps * np.linalg.norm(want)
            assert M.sync_status() == 0
    finally:
        M.close()


def test_noalloc_rejects_oversize(hm):
    n = hm.HM_NOALLOC_MAX_ENTRIES // 64 + 1
    pts = synth.cube_points(n)
    M = hm.HMatrix(pts, "matern", 64, 2.0, "h", 1e-4)
    try:
        M.compress(1e-4, "fpx", True)
        x = np.asfortranarray(np.zeros((n, 64)))
        y = np.asfortranarray(np.zeros((n, 64)))
        with pytest.raises(hm.HMError, match="fixed limit"):
            hm.hm_matvec_host_noalloc(M.h, 1.0, x, 0.0, y)
    finally:
        M.close()
