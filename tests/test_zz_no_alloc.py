"""hm_matvec_host_noalloc: the allocation-free host-buffer product.

Callers that cannot let the library allocate device memory (a serving process
that reserved its whole HBM budget up front; code that must not trigger
cudaFree's device-wide synchronisation while other streams run) use this entry
point.  It stages x and y through libhm's fixed device array instead of buffers
it would allocate.  Through the C ABI the test checks:

* two calls in a row with different data give, bit for bit, what the existing
  hm_matvec entry point gives on device buffers (the same kernels run on the same
  inputs, so the results must be identical, not merely close);
* beta = 0 right after a call that left other data in the array: the product
  reads no y (the host y holds NaN) and no leftover scratch;
* a panel of 12 right-hand sides (the multi-RHS tensor-core path, ld = n in the
  array);
* device free memory is the same before and after every call (the array is part
  of the loaded library, so the calls themselves allocate nothing);
* a request larger than the array is refused.

The file is named to be collected last, so that a run stopping at the first
failure has run every other test before it.
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
    """hm_matvec on device buffers (column-major, ld = n)."""
    xd = torch.from_numpy(np.asfortranarray(x)).cuda()
    yd = torch.from_numpy(np.asfortranarray(y0.copy())).cuda()
    if xd.dim() == 2:
        xd = xd.t().contiguous().t()
        yd = yd.t().contiguous().t()
    M.matvec(alpha, xd, beta, yd)
    torch.cuda.synchronize()
    out = yd.cpu().numpy()
    return np.asfortranarray(out)


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def test_noalloc_matches_matvec_bitwise(hm):
    n, eps = 2048, 1e-6
    pts = synth.sphere_points(n)
    M = hm.HMatrix(pts, "laplace", 32, 2.0, "h", eps)
    try:
        M.compress(eps, "aflp", True)
        nan_y = np.full(n, np.nan)
        cases = [(synth.rhs(n, 1, seed=11)[:, 0], synth.rhs(n, 1, seed=12)[:, 0], 1.0, 1.0),
                 (synth.rhs(n, 3, seed=13), synth.rhs(n, 3, seed=14), 0.5, -2.0),
                 (synth.rhs(n, 1, seed=15)[:, 0], nan_y, 1.25, 0.0),           # leftover scratch, y unread
                 (synth.rhs(n, 12, seed=16), synth.rhs(n, 12, seed=17), -0.75, 0.5)]   # multi-RHS panel
        wants = [_device_product(M, x, np.nan_to_num(y0, nan=0.0) if beta == 0.0 else y0, a, beta)
                 for x, y0, a, beta in cases]
        xs = [np.asfortranarray(x) for x, _, _, _ in cases]
        gots = [np.asfortranarray(y0.copy()) for _, y0, _, _ in cases]
        hm.hm_matvec_host_noalloc(M.h, 1.0, xs[0], 1.0, np.asfortranarray(cases[0][1].copy()))  # first call: set-up
        torch.cuda.synchronize()
        for (x, y0, alpha, beta), xf, got, want in zip(cases, xs, gots, wants):
            free0 = torch.cuda.mem_get_info()[0]
            hm.hm_matvec_host_noalloc(M.h, alpha, xf, beta, got)
            free1 = torch.cuda.mem_get_info()[0]
            assert free1 == free0, "device free memory changed across the call"
            assert np.all(np.isfinite(got))
            assert np.array_equal(_bits(got), _bits(want)), (alpha, beta, x.shape)
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
