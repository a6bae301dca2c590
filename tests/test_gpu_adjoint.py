"""Adjoint products y := alpha*M^H*x + beta*y on the GPU (hm_matvec_adjoint)
against the oracle's adjoint of the uncompressed FP64 matrix (the remark after
Alg. 3), through the C ABI.

* every format, eps 1e-6 (FP32 tier) and 1e-8 (float-float tier): within 4 eps;
* several right-hand sides (the multi-RHS panels for r >= 9): within 4 eps per
  column;
* the adjoint identity <y, M x> = <M^H y, x> between the GPU's own forward and
  adjoint products in the float-float tier, where the products are accurate to
  about 1e-13: the Laplace matrix is symmetric up to its approximation error, so
  only this identity tells M^T x from M x there;
* the row-weighted Laplace matrix diag(w) A (far from symmetric: M^T x and M x
  differ by far more than 4 eps), every format and both tiers: within 4 eps of
  the oracle's adjoint, which pins the adjoint product itself in the FP32 tier
  as well.
"""
import numpy as np
import pytest

import synth
from oracle import hmatrix, matvec, nested

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

N = 2048


@pytest.fixture(scope="module")
def hm():
    from paper_2405_03456_gb300 import build, hm as _hm
    build.build()
    _hm.load()
    return _hm


_cache = {}


def oracle_adj(pts, fmt, eps, x, alpha, y0, beta):
    if (fmt, eps) not in _cache:
        h = hmatrix.build_h(pts, "laplace", 32, 2.0, eps)
        _cache[(fmt, eps)] = h if fmt == "h" else (nested.build_uniform(h) if fmt == "uh" else nested.build_h2(h))
    f = {"h": matvec.h_mvm_adjoint, "uh": matvec.uh_mvm_adjoint, "h2": matvec.h2_mvm_adjoint}[fmt]
    return f(_cache[(fmt, eps)], alpha, x, beta, y0)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cols(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda().t().contiguous().t()


@pytest.mark.parametrize("fmt", ["h", "uh", "h2"])
@pytest.mark.parametrize("eps", [1e-6, 1e-8])
def test_adjoint_within_4eps(hm, fmt, eps):
    pts = synth.sphere_points(N)
    x = synth.rhs(N, 1, seed=41)[:, 0]
    y0 = synth.rhs(N, 1, seed=42)[:, 0]
    ref = oracle_adj(pts, fmt, eps, x, 0.75, y0, -0.5)
    M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, eps)
    try:
        M.compress(eps, "aflp")
        xd = torch.from_numpy(x.copy()).cuda()
        outs = []
        for _ in range(2):
            yd = torch.from_numpy(y0.copy()).cuda()
            M.matvec(0.75, xd, -0.5, yd, adjoint=True)
            torch.cuda.synchronize()
            outs.append(yd.cpu().numpy())
        assert M.sync_status() == 0
        assert rel(outs[0], ref) <= 4 * eps
        assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
    finally:
        M.close()


@pytest.mark.parametrize("fmt", ["h", "h2"])
def test_adjoint_multi_rhs(hm, fmt):
    pts = synth.sphere_points(N)
    eps = 1e-6
    r = 19
    x = synth.rhs(N, r, seed=51)
    ref = oracle_adj(pts, fmt, eps, x, 1.0, np.zeros_like(x), 0.0)
    M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, eps)
    try:
        M.compress(eps, "aflp")
        yd = cols(np.zeros_like(x))
        M.matvec(1.0, cols(x), 0.0, yd, adjoint=True)
        got = yd.cpu().numpy()
        assert M.sync_status() == 0
        for k in range(r):
            assert rel(got[:, k], ref[:, k]) <= 4 * eps, k
    finally:
        M.close()


@pytest.mark.parametrize("fmt", ["h", "uh", "h2"])
@pytest.mark.parametrize("codec,eps", [("none", 1e-6), ("aflp", 1e-8)])
def test_adjoint_identity_on_gpu(hm, fmt, codec, eps):
    pts = synth.sphere_points(N)
    x = synth.rhs(N, 1, seed=61)[:, 0]
    y = synth.rhs(N, 1, seed=62)[:, 0]
    M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, eps)
    try:
        M.compress(eps, codec)
        mx = torch.zeros(N, dtype=torch.float64, device="cuda")
        mty = torch.zeros(N, dtype=torch.float64, device="cuda")
        M.matvec(1.0, torch.from_numpy(x.copy()).cuda(), 0.0, mx)
        M.matvec(1.0, torch.from_numpy(y.copy()).cuda(), 0.0, mty, adjoint=True)
        mx, mty = mx.cpu().numpy(), mty.cpu().numpy()
        assert M.sync_status() == 0
        lhs, rhs = float(y @ mx), float(mty @ x)
        assert abs(lhs - rhs) <= 1e-11 * np.linalg.norm(y) * np.linalg.norm(mx)
        # and the adjoint is not the forward product: M^T - M is of the order of eps
        mty_fwd = torch.zeros(N, dtype=torch.float64, device="cuda")
        M.matvec(1.0, torch.from_numpy(y.copy()).cuda(), 0.0, mty_fwd)
        assert rel(mty_fwd.cpu().numpy(), mty) > 1e-11
    finally:
        M.close()


def test_recompress_rebuilds_the_adjoint(hm):
    """hm_compress discards the transposed matrix: the adjoint after a second
    compression equals, bit for bit, that of a matrix compressed only that way."""
    pts = synth.sphere_points(N)
    x = torch.from_numpy(synth.rhs(N, 1, seed=71)[:, 0].copy()).cuda()
    outs = []
    for steps in ((("aflp", 1e-6), ("fpx", 1e-8)), (("fpx", 1e-8),)):
        M = hm.HMatrix(pts, "laplace", 32, 2.0, "h", 1e-6)
        try:
            for codec, eps in steps:
                M.compress(eps, codec)
                yd = torch.zeros(N, dtype=torch.float64, device="cuda")
                M.matvec(1.0, x, 0.0, yd, adjoint=True)
            outs.append(yd.cpu().numpy())
            assert M.sync_status() == 0
        finally:
            M.close()
    assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
    ref = oracle_adj(pts, "h", 1e-6, x.cpu().numpy(), 1.0, np.zeros(N), 0.0)
    assert rel(outs[0], ref) <= 4 * 1e-6


_wcache = {}


@pytest.mark.parametrize("fmt", ["h", "uh", "h2", "uh_sep"])
@pytest.mark.parametrize("eps", [1e-6, 1e-8])
def test_adjoint_non_symmetric(hm, fmt, eps):
    pts = synth.sphere_points(N)
    if eps not in _wcache:
        h = hmatrix.build_h(pts, "laplace_w", 32, 2.0, eps)
        _wcache[eps] = {"h": h, "uh": nested.build_uniform(h), "h2": nested.build_h2(h)}
    om = _wcache[eps]["uh" if fmt == "uh_sep" else fmt]
    fa = {"h": matvec.h_mvm_adjoint, "uh": matvec.uh_mvm_adjoint, "h2": matvec.h2_mvm_adjoint,
          "uh_sep": matvec.uh_mvm_adjoint}[fmt]
    fw = {"h": matvec.h_mvm, "uh": matvec.uh_mvm, "h2": matvec.h2_mvm, "uh_sep": matvec.uh_mvm}[fmt]
    x = synth.rhs(N, 1, seed=61)[:, 0]
    y0 = synth.rhs(N, 1, seed=62)[:, 0]
    ref = fa(om, 0.75, x, -0.5, y0)
    fwd = fw(om, 0.75, x, -0.5, y0)
    assert rel(fwd, ref) > 100 * eps                     # the check tells M^T x from M x
    M = hm.HMatrix(pts, "laplace_w", 32, 2.0, fmt, eps)
    try:
        M.compress(eps, "aflp", True)
        xd = torch.from_numpy(x.copy()).cuda()
        yd = torch.from_numpy(y0.copy()).cuda()
        M.matvec(0.75, xd, -0.5, yd, adjoint=True)
        torch.cuda.synchronize()
        assert M.sync_status() == 0
        assert rel(yd.cpu().numpy(), ref) <= 4 * eps
        yf = torch.from_numpy(y0.copy()).cuda()
        M.matvec(0.75, xd, -0.5, yf)
        torch.cuda.synchronize()
        assert rel(yf.cpu().numpy(), fwd) <= 4 * eps
    finally:
        M.close()
