"""Triangular solves with compressed H-LU factors on the GPU (hm_lu_*), against
the CPU oracle (Sec. 5, Conclusion: the outlook's triangular solves).

The two sides share only the seeded inputs: the library factors the Matern
covariance matrix with its own host elimination and ACA/SVD truncation, the
oracle (``oracle/hlu.py``) with numpy elimination and exact SVD truncation.
Both solve x = U^-1 L^-1 b with their own factors, so both approximate the
exact solution x* = A^-1 b up to the perturbation of their factors
(||x~ - x*|| <= ||A^-1|| ||E|| ||x~||, E = L~U~ - A).  The checks:

* the GPU solution is within max(4 e_or, 4 eps) of x*, where e_or is the
  oracle's own relative error at the same eps and codec (the accuracy the
  method reaches), for FP64, AFLP and FPX factors at eps = 1e-4, 1e-6, 1e-8;
* its residual ||A x - b|| / (||A|| ||x||) is below eps;
* repeated solves are bitwise identical (no atomics in the arithmetic), several
  right-hand sides equal single solves, and the error word stays clear.
"""
import numpy as np
import pytest

import synth
from oracle import hlu, kernels

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

N = 1000


@pytest.fixture(scope="module")
def hm():
    from paper_2405_03456_gb300 import build, hm as _hm
    build.build()
    _hm.load()
    return _hm


@pytest.fixture(scope="module")
def problem():
    pts = synth.cube_points(N)
    a = kernels.entries("matern", pts, np.arange(N), np.arange(N), kernels.default_param("matern", N))
    b = synth.rhs(N, 3, seed=31)
    xs = np.linalg.solve(a, b)
    return pts, a, b, xs


def rel(u, v):
    return float(np.linalg.norm(u - v) / np.linalg.norm(v))


_oracle = {}


def oracle_error(pts, b, xs, eps, codec):
    if eps not in _oracle:
        _oracle[eps] = hlu.build_hlu(pts, "matern", 32, 2.0, eps)[0]
    f = _oracle[eps]
    if codec == "none":
        mL, mU = f.L, f.U
    else:
        mL, mU = hlu.compress_hlu(f, codec)
    return rel(hlu.hlu_solve(mL, mU, b[:, 0]), xs[:, 0])


def gpu_solve(F, b):
    bd = torch.from_numpy(np.asfortranarray(b)).cuda()
    if bd.dim() == 2:
        bd = bd.t().contiguous().t()
    xd = torch.zeros_like(bd)
    F.solve(bd, xd)
    torch.cuda.synchronize()
    return xd.cpu().numpy()


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_hlu_solve_against_oracle(hm, problem, eps):
    pts, a, b, xs = problem
    F = hm.HLU(pts, "matern", 32, 2.0, eps)
    try:
        for codec in ("none", "aflp", "fpx"):
            F.compress(eps, codec, True)
            x = gpu_solve(F, b[:, 0])
            assert F.sync_status() == 0
            e_or = oracle_error(pts, b, xs, eps, codec)
            assert rel(x, xs[:, 0]) <= max(4 * e_or, 4 * eps), (codec, rel(x, xs[:, 0]), e_or)
            res = np.linalg.norm(a @ x - b[:, 0]) / (np.linalg.norm(a) * np.linalg.norm(x))
            assert res <= eps, (codec, res)
            if codec != "none":
                info = F.info()
                assert info["bytes_values"] < 0.75 * info["bytes_fp64"]
    finally:
        F.close()


def test_hlu_solve_repeat_and_columns(hm, problem):
    pts, a, b, xs = problem
    eps = 1e-6
    F = hm.HLU(pts, "matern", 32, 2.0, eps)
    try:
        F.compress(eps, "aflp", True)
        x3 = gpu_solve(F, b)
        for k in range(3):
            xk = gpu_solve(F, b[:, k])
            assert np.array_equal(xk.view(np.uint64), x3[:, k].copy().view(np.uint64))
            assert rel(xk, xs[:, k]) <= 4e-5
        again = gpu_solve(F, b)
        assert np.array_equal(again.view(np.uint64), x3.view(np.uint64))
        assert F.sync_status() == 0
    finally:
        F.close()


def test_hlu_solve_larger(hm):
    """N = 4096 (128 leaves, a deeper dependency chain): the exact solution by
    a dense solve, the residual below eps."""
    n, eps = 4096, 1e-6
    pts = synth.cube_points(n)
    a = kernels.entries("matern", pts, np.arange(n), np.arange(n), kernels.default_param("matern", n))
    b = synth.rhs(n, 1, seed=33)[:, 0]
    xs = np.linalg.solve(a, b)
    F = hm.HLU(pts, "matern", 32, 2.0, eps)
    try:
        F.compress(eps, "aflp", True)
        x = gpu_solve(F, b)
        assert F.sync_status() == 0
        res = np.linalg.norm(a @ x - b) / (np.linalg.norm(a) * np.linalg.norm(x))
        assert res <= eps
        assert rel(x, xs) <= 20 * eps
    finally:
        F.close()
