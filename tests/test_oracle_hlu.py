"""Pins of the oracle's H-LU factors and triangular solves.

Checked against a hand-computed factorisation, LAPACK's partial-pivoting LU where
it picks no row swap, LAPACK's dense triangular solves of the expanded factors,
and the perturbation identity of the solve: with E = L U - A (factors as stored,
decoded for a codec), the solve returns x~ = (A + E)^{-1} b, hence
||x~ - A^{-1} b|| <= ||A^{-1}|| ||E|| ||x~||.
"""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import hlu, hmatrix, kernels

N = 1000            # not a power of two: leaf sizes vary below 32


@pytest.fixture(scope="module", params=[1e-4, 1e-6, 1e-8])
def factors(request):
    eps = request.param
    pts = synth.cube_points(N)
    f, lx, ux = hlu.build_hlu(pts, "matern", 32, 2.0, eps)
    perm = f.L.ct.perm
    ap = hmatrix.exact_matrix(pts, "matern", kernels.default_param("matern", N))[np.ix_(perm, perm)]
    return eps, pts, f, lx, ux, ap


def test_lu_nopivot_hand_example():
    a = np.array([[4.0, 2, 2], [2, 5, 3], [2, 3, 6]])
    L, U = hlu.lu_nopivot(a)
    assert np.array_equal(L, [[1, 0, 0], [0.5, 1, 0], [0.5, 0.5, 1]])
    assert np.array_equal(U, [[4, 2, 2], [0, 4, 2], [0, 0, 4]])


def test_lu_nopivot_equals_lapack_without_swaps():
    rng = np.random.default_rng(5)
    a = rng.uniform(-1, 1, (60, 60)) + 80 * np.eye(60)     # partial pivoting keeps the diagonal
    p, l, u = scipy.linalg.lu(a)
    assert np.array_equal(p, np.eye(60))
    L, U = hlu.lu_nopivot(a)
    assert np.allclose(L, l, rtol=0, atol=1e-14) and np.allclose(U, u, rtol=0, atol=1e-12)


def test_factor_blocks(factors):
    eps, pts, f, lx, ux, ap = factors
    assert np.abs(lx @ ux - ap).max() <= 1e-13 * np.abs(ap).max()
    cl = f.L.ct.clusters
    rows = lambda b: cl[b.row]
    cols = lambda b: cl[b.col]
    ldiag = [b for b in f.L.blocks if b.row == b.col]
    assert sorted(b.row for b in ldiag) == sorted(c.id for c in f.L.ct.leaves())
    assert all(rows(b).start >= cols(b).end for b in f.L.blocks if b.row != b.col)
    assert all(rows(b).end <= cols(b).start for b in f.U.blocks if b.row != b.col)
    area = sum(rows(b).size * cols(b).size for b in f.L.blocks + f.U.blocks if b.row != b.col)
    area += sum(rows(b).size ** 2 for b in ldiag)
    assert area == N * N                                    # the two factors tile I x I
    Ld, Ud = hlu.dense_factor(f.L), hlu.dense_factor(f.U)
    assert np.array_equal(np.triu(Ld, 1), np.zeros_like(Ld)) and np.array_equal(np.diag(Ld), np.ones(N))
    assert np.array_equal(np.tril(Ud, -1), np.zeros_like(Ud))
    # the expanded factors approximate the exact ones blockwise at eps (spectral), so
    # in the Frobenius norm within eps times the number of blocks
    nb = len(f.L.blocks) + len(f.U.blocks)
    assert np.linalg.norm(Ld - lx) <= eps * nb * np.linalg.norm(lx)
    assert np.linalg.norm(Ud - ux) <= eps * nb * np.linalg.norm(ux)
    assert np.linalg.norm(Ld - lx) > 0                      # low-rank blocks were truncated
    for m, ex in ((f.L, lx), (f.U, ux)):
        for b, d in zip(m.blocks, m.data):
            t, s = rows(b), cols(b)
            blk = ex[t.start:t.end, s.start:s.end]
            got = (d.W * d.s) @ d.X.T if b.adm else d
            if not b.adm:
                ref = np.tril(blk) if (m is f.L and b.row == b.col) else (np.triu(blk) if b.row == b.col else blk)
                assert np.array_equal(got, ref)
            else:                                           # truncation rule of eqn. epsilon
                assert np.linalg.norm(got - blk, 2) <= eps * np.linalg.norm(blk, 2) * (1 + 1e-9) + 1e-15


@pytest.mark.parametrize("codec", ["none", "aflp", "fpx"])
def test_block_substitution_equals_dense_triangular_solves(factors, codec):
    eps, pts, f, lx, ux, ap = factors
    cL, cU = hlu.compress_hlu(f, codec)
    Ld, Ud = hlu.dense_factor(cL), hlu.dense_factor(cU)
    b = np.random.default_rng(7).uniform(-1, 1, (N, 3))
    x = hlu.hlu_solve(cL, cU, b)
    perm = f.L.ct.perm
    z = scipy.linalg.solve_triangular(Ld, b[perm], lower=True, unit_diagonal=True)
    z = scipy.linalg.solve_triangular(Ud, z, lower=False)
    assert np.abs(x[perm] - z).max() <= 1e-12 * np.abs(z).max()
    x0 = hlu.hlu_solve(cL, cU, b[:, 1])
    assert np.abs(x0 - x[:, 1]).max() <= 1e-13 * np.abs(x[:, 1]).max()
    if codec == "none":                                     # the FP64 factors themselves
        xf = hlu.hlu_solve(f.L, f.U, b)
        assert np.abs(xf - x).max() <= 1e-13 * np.abs(x).max()


@pytest.mark.parametrize("codec", ["none", "aflp", "fpx"])
def test_solve_error_within_perturbation_bound(factors, codec):
    eps, pts, f, lx, ux, ap = factors
    cL, cU = hlu.compress_hlu(f, codec)
    E = hlu.dense_factor(cL) @ hlu.dense_factor(cU) - ap
    na = np.linalg.norm(ap, 2)
    assert np.linalg.norm(E, 2) <= eps * na                  # blockwise eps keeps L U near A
    b = np.random.default_rng(8).uniform(-1, 1, N)
    x = hlu.hlu_solve(cL, cU, b)
    a = hmatrix.exact_matrix(pts, "matern", kernels.default_param("matern", N))
    xe = np.linalg.solve(a, b)
    inv = 1.0 / np.linalg.svd(ap, compute_uv=False)[-1]
    bound = inv * np.linalg.norm(E, 2) * np.linalg.norm(x)
    assert np.linalg.norm(x - xe) <= 1.01 * bound + 1e-11 * np.linalg.norm(xe)


def test_single_leaf_is_dense_lu_solve():
    pts = synth.cube_points(24)
    f, lx, ux = hlu.build_hlu(pts, "matern", 32, 2.0, 1e-6)
    assert len(f.L.blocks) == 1 and len(f.U.blocks) == 1
    b = np.random.default_rng(9).uniform(-1, 1, 24)
    x = hlu.hlu_solve(f.L, f.U, b)
    a = hmatrix.exact_matrix(pts, "matern", kernels.default_param("matern", 24))
    assert np.allclose(a @ x, b, rtol=0, atol=1e-12)
