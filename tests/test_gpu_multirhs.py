"""Multi-RHS products (panels of 32 right-hand sides through the tensor-core
kernels, FP32 tier) against the CPU oracle, through the C ABI.

Each column of Y := alpha*M*X + beta*Y must be within 4*eps of the oracle's
uncompressed FP64 product of that column, for RHS counts that give partial
panels (2, 19), a full panel (32) and a full plus a ragged panel (45); the
result must not depend on how many other right-hand sides share the panel
beyond summation order, and repeated products must be bitwise equal.
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
EPS = 1e-6


@pytest.fixture(scope="module")
def hm():
    from paper_2405_03456_gb300 import build, hm as _hm
    build.build()
    _hm.load()
    return _hm


@pytest.fixture(scope="module")
def oracle_mats():
    pts = synth.sphere_points(N)
    h = hmatrix.build_h(pts, "laplace", 32, 2.0, EPS)
    return pts, {"h": h, "uh": nested.build_uniform(h), "h2": nested.build_h2(h)}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def device_cols(a):
    t = torch.from_numpy(np.asfortranarray(a)).cuda()
    return t.t().contiguous().t()


@pytest.mark.parametrize("fmt", ["h", "uh", "h2"])
@pytest.mark.parametrize("r", [2, 19, 32, 45])
def test_multi_rhs_columns_within_4eps(hm, oracle_mats, fmt, r):
    pts, mats = oracle_mats
    x = synth.rhs(N, r, seed=100 + r)
    y0 = synth.rhs(N, r, seed=200 + r)
    f = {"h": matvec.h_mvm, "uh": matvec.uh_mvm, "h2": matvec.h2_mvm}[fmt]
    ref = f(mats[fmt], 0.5, x, -1.5, y0)
    M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, EPS)
    try:
        M.compress(EPS, "aflp")
        xd = device_cols(x)
        outs = []
        for _ in range(2):
            yd = device_cols(y0)
            M.matvec(0.5, xd, -1.5, yd)
            torch.cuda.synchronize()
            outs.append(yd.cpu().numpy())
        assert M.sync_status() == 0
        assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
        for k in range(r):
            assert rel(outs[0][:, k], ref[:, k]) <= 4 * EPS, k
    finally:
        M.close()


def test_multi_rhs_matches_single_rhs(hm, oracle_mats):
    """Column k of a 37-column product equals the single-RHS product of column k
    to well within the compression tolerance (only summation order differs)."""
    pts, _ = oracle_mats
    r = 37
    x = synth.rhs(N, r, seed=7)
    M = hm.HMatrix(pts, "laplace", 32, 2.0, "h", EPS)
    try:
        M.compress(EPS, "aflp")
        yd = torch.zeros((N, r), dtype=torch.float64, device="cuda").t().contiguous().t()
        M.matvec(1.0, device_cols(x), 0.0, yd)
        ym = yd.cpu().numpy()
        for k in (0, 31, 32, 36):
            ys = torch.zeros(N, dtype=torch.float64, device="cuda")
            M.matvec(1.0, torch.from_numpy(x[:, k].copy()).cuda(), 0.0, ys)
            assert rel(ym[:, k], ys.cpu().numpy()) <= 1e-6
    finally:
        M.close()


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("fmt", ["h", "uh", "h2"])
@pytest.mark.parametrize("leaf", [32, 64, 128])
def test_multi_rhs_wide_chunks(hm, fmt, leaf, engine):
    """Both row-chunk engines (0: tensor-core fragments, 1: FP32 pipes), with
    leaves of 32 and 64 rows (one and both warps of a pair) and of 128 rows (the
    shared-tile kernel, for chunks wider than 64 rows): every column of a
    40-column product equals the single-RHS product of that column to well
    within the compression tolerance, and repeated panels are bitwise equal."""
    r = 40
    pts = synth.sphere_points(N)
    x = synth.rhs(N, r, seed=11 + leaf)
    y0 = synth.rhs(N, r, seed=12 + leaf)
    M = hm.HMatrix(pts, "laplace", leaf, 2.0, fmt, EPS)
    try:
        M.compress(EPS, "aflp")
        assert M.multi_rhs_engine(engine) == engine
        outs = []
        for _ in range(2):
            yd = device_cols(y0)
            M.matvec(0.75, device_cols(x), 0.5, yd)
            torch.cuda.synchronize()
            outs.append(yd.cpu().numpy())
        assert M.sync_status() == 0
        assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
        for k in range(r):
            ys = torch.from_numpy(y0[:, k].copy()).cuda()
            M.matvec(0.75, torch.from_numpy(x[:, k].copy()).cuda(), 0.5, ys)
            assert rel(outs[0][:, k], ys.cpu().numpy()) <= 1e-6, k
    finally:
        M.close()


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("codec,eps", [("aflp", 1e-4), ("fpx", 1e-4), ("fpx", 1e-6)])
def test_multi_rhs_codecs_and_limbs(hm, engine, codec, eps):
    """Both engines on AFLP / FPX payloads whose pieces keep 1, 2 or 3 BF16 limbs
    (eps = 1e-4 leaves short mantissas): every column of a 33-column product
    within 4 eps of the oracle's uncompressed product."""
    r = 33
    pts = synth.sphere_points(N)
    h = hmatrix.build_h(pts, "laplace", 32, 2.0, eps)
    x = synth.rhs(N, r, seed=41)
    y0 = synth.rhs(N, r, seed=42)
    ref = matvec.h_mvm(h, 1.25, x, 0.5, y0)
    M = hm.HMatrix(pts, "laplace", 32, 2.0, "h", eps)
    try:
        M.compress(eps, codec)
        assert M.multi_rhs_engine(engine) == engine
        yd = device_cols(y0)
        M.matvec(1.25, device_cols(x), 0.5, yd)
        torch.cuda.synchronize()
        assert M.sync_status() == 0
        out = yd.cpu().numpy()
        for k in range(r):
            assert rel(out[:, k], ref[:, k]) <= 4 * eps, k
    finally:
        M.close()
