"""Full-size parity: every configuration the benchmark times, at its own size.

The benchmark's workloads (N = 131072 Laplace sphere, leaf 64) are far beyond
the oracle's dense product, so the check uses outputs the oracle computes one
by one: sampled rows of the EXACT dense product, y_i = sum_j a_ij x_j (the
oracle's kernel entries, ``oracle.kernels``), and, for decompression, the
oracle's decoder applied to a random sample of the resident packed units
(``hm_decompress_debug``, both tiers, bit for bit as in
``test_gpu_decode_resident.py``).

The H approximation differs from the exact matrix by about eps relative per
block (eqn. epsilon) and compression adds at most eps (Sec. 4.2), so sampled
rows must lie within 4 eps of the exact rows (the relative 2-norm over the
sample).  Covered here: H with AFLP and FPX at eps = 1e-4, 1e-6 (FP32 tier) and
1e-8 (float-float tier), the separate-coupling UH format, a 32-wide multi-RHS
panel (tensor-core path), the adjoint of a non-symmetric matrix (row-weighted
Laplace kernel), and the Matern cube at N = 262144.  Full-size payloads are where
large offsets, chunks shared by several warps and deep trees appear.
"""
import numpy as np
import pytest

import synth
from oracle import kernels

from decode_check import aflp_f, f32_tier_head, fields, oracle_values

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

N = 131072
NROWS = 192


@pytest.fixture(scope="module")
def hm():
    from paper_2405_03456_gb300 import build, hm as _hm
    build.build()
    _hm.load()
    return _hm


@pytest.fixture(scope="module")
def sphere():
    return synth.sphere_points(N)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def exact_rows(kind, pts, x, rows, param=None, transpose=False):
    """Rows of the exact dense product A x (or A^T x), one by one."""
    n = pts.shape[0]
    param = kernels.default_param(kind, n) if param is None else param
    cols = np.arange(n)
    out = []
    for i in rows:
        if transpose:   # row i of A^T is column i of A
            a = kernels.entries(kind, pts, cols, np.array([i]), param)[:, 0]
        else:
            a = kernels.entries(kind, pts, np.array([i]), cols, param)[0]
        out.append(a @ x)
    return np.array(out).reshape(len(rows), *x.shape[1:])


def device_product(M, x, alpha=1.0, adjoint=False):
    xd = torch.from_numpy(np.asfortranarray(x)).cuda()
    if xd.dim() == 2:
        xd = xd.t().contiguous().t()
    yd = torch.zeros_like(xd)
    M.matvec(alpha, xd, 0.0, yd, adjoint=adjoint)
    torch.cuda.synchronize()
    assert M.sync_status() == 0
    return yd.cpu().numpy()


def check_decode_sample(hm, M, nsample=1200, seed=0):
    """Bit-exact decode of a random sample of the resident units (both tiers)."""
    nu = M.info()["nunits"]
    rng = np.random.default_rng(seed)
    starts = np.sort(rng.choice(nu, size=min(nsample, nu), replace=False))
    for u in starts[:: max(1, len(starts) // 60)]:   # 60 runs of 20 consecutive units
        d_ff = hm.hm_decompress_debug(M.h, 1, int(u), int(u) + 20)
        d_32 = hm.hm_decompress_debug(M.h, 0, int(u), int(u) + 20)
        code, fmt = d_ff["code"], d_ff["fmt"]
        if code.size == 0:
            continue
        v = oracle_values(code, fmt)
        B, F, E, Mb = fields(fmt)
        f = aflp_f(code, fmt)
        wide = (F == 3) | ((F == 1) & (B == 8)) | ((F == 2) & ((Mb >= 48) | (f > 46)))
        ok = ~wide & (np.abs(v) >= 2.0 ** -74)
        got = d_ff["head"].astype(np.float64) + d_ff["tail"].astype(np.float64)
        assert np.array_equal(got[ok].view(np.uint64), v[ok].view(np.uint64)), int(u)
        ok32 = np.abs(v) >= 2.0 ** -126
        want32 = f32_tier_head(code, fmt, v)
        assert np.array_equal(d_32["head"][ok32].view(np.uint32), want32[ok32].view(np.uint32)), int(u)
        assert not np.any(d_32["tail"])
    assert M.sync_status() == 0


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_h_full_size_codecs(hm, sphere, eps):
    """H at the benchmark's size, AFLP and FPX (VALR): sampled exact rows and resident decode."""
    x = synth.rhs(N)[:, 0]
    rows = np.random.default_rng(11).choice(N, NROWS, replace=False)
    ye = exact_rows("laplace", sphere, x, rows)
    M = hm.HMatrix(sphere, "laplace", 64, 2.0, "h", eps)
    try:
        for codec in ("aflp", "fpx"):
            M.compress(eps, codec, True)
            y = device_product(M, x)
            assert rel(y[rows], ye) <= 4 * eps, (eps, codec)
            check_decode_sample(hm, M, seed=int(-np.log10(eps)))
    finally:
        M.close()


def test_uh_sep_full_size(hm, sphere):
    eps = 1e-6
    x = synth.rhs(N)[:, 0]
    rows = np.random.default_rng(12).choice(N, NROWS, replace=False)
    ye = exact_rows("laplace", sphere, x, rows)
    M = hm.HMatrix(sphere, "laplace", 64, 2.0, "uh_sep", eps)
    try:
        M.compress(eps, "aflp", True)
        assert rel(device_product(M, x)[rows], ye) <= 4 * eps
        check_decode_sample(hm, M, seed=5)
    finally:
        M.close()


def test_multi_rhs_panel_full_size(hm, sphere):
    """A 32-wide panel on the headline matrix, on both multi-RHS engines (the
    FP32 pipes; tcgen05 with BF16 limbs): every column within 4 eps of the exact
    rows, and the two engines within 1e-6 of each other."""
    eps = 1e-6
    X = synth.rhs(N, 32, seed=21)
    rows = np.random.default_rng(13).choice(N, 64, replace=False)
    ye = exact_rows("laplace", sphere, X, rows)
    M = hm.HMatrix(sphere, "laplace", 64, 2.0, "h", eps)
    try:
        M.compress(eps, "aflp", True)
        Ys = []
        for engine in (1, 0):
            assert M.multi_rhs_engine(engine) == engine
            Y = device_product(M, X)
            assert M.sync_status() == 0
            for k in range(32):
                assert rel(Y[rows, k], ye[:, k]) <= 4 * eps, (engine, k)
            Ys.append(Y)
        for k in range(32):
            assert rel(Ys[1][:, k], Ys[0][:, k]) <= 1e-6, k
    finally:
        M.close()


def test_adjoint_non_symmetric_full_size(hm, sphere):
    """M^T x of the row-weighted Laplace matrix diag(w) A (w_i = 1 + x_i / 2 of
    point i): M^T differs from M by far more than 4 eps, so the check pins the
    adjoint product itself."""
    eps = 1e-6
    x = synth.rhs(N)[:, 0]
    rows = np.random.default_rng(14).choice(N, 128, replace=False)
    yt = exact_rows("laplace_w", sphere, x, rows, transpose=True)
    yf = exact_rows("laplace_w", sphere, x, rows)
    assert rel(yf, yt) > 100 * eps            # the matrix is far from symmetric
    M = hm.HMatrix(sphere, "laplace_w", 64, 2.0, "h", eps)
    try:
        M.compress(eps, "aflp", True)
        assert rel(device_product(M, x, adjoint=True)[rows], yt) <= 4 * eps
        assert rel(device_product(M, x)[rows], yf) <= 4 * eps
    finally:
        M.close()


def test_matern_cube_large(hm):
    """Matern nu = 1.5 on N = 262144 uniform points of the unit cube (the
    covariance workload, half the benchmark leg's size so that the host build
    fits the test's time): sampled exact rows and resident decode."""
    n, eps = 262144, 1e-6
    pts = synth.cube_points(n)
    x = synth.rhs(n)[:, 0]
    rows = np.random.default_rng(15).choice(n, 128, replace=False)
    ye = exact_rows("matern", pts, x, rows)
    M = hm.HMatrix(pts, "matern", 64, 2.0, "h", eps)
    try:
        M.compress(eps, "aflp", True)
        assert rel(device_product(M, x)[rows], ye) <= 4 * eps
        check_decode_sample(hm, M, seed=7)
    finally:
        M.close()
