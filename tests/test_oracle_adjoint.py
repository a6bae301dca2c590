"""Pins of the oracle's adjoint products y := alpha M^H x + beta y (the remark
after Alg. 3: the same steps over the block columns; real data, M^H = M^T).

* H in FP64 against the transpose of its dense expansion (the plain definition);
* the adjoint identity <y, M x> = <M^T y, x> for H, UH and H^2, uncompressed and
  compressed (AFLP and FPX, VALR), which ties every adjoint to the forward
  product already pinned elsewhere: a dropped transpose of a coupling or a
  transfer matrix, or swapped row / column bases, breaks it;
* alpha / beta handling and several right-hand sides at once.
"""
import numpy as np
import pytest

import synth
from oracle import compress, hmatrix, matvec, nested

N = 768


@pytest.fixture(scope="module")
def mats():
    pts = synth.sphere_points(N)
    h = hmatrix.build_h(pts, "laplace", 32, 2.0, 1e-6)
    u = nested.build_uniform(h)
    h2 = nested.build_h2(h)
    return {"h": (h, matvec.h_mvm, matvec.h_mvm_adjoint, compress.compress_h),
            "uh": (u, matvec.uh_mvm, matvec.uh_mvm_adjoint, compress.compress_uh),
            "h2": (h2, matvec.h2_mvm, matvec.h2_mvm_adjoint, compress.compress_h2)}


def test_h_adjoint_is_the_dense_transpose(mats):
    h = mats["h"][0]
    a = hmatrix.dense_matrix(h)
    x = synth.rhs(N, 2, seed=11)
    y0 = synth.rhs(N, 2, seed=12)
    ref = 0.5 * (a.T @ x) - 2.0 * y0
    got = matvec.h_mvm_adjoint(h, 0.5, x, -2.0, y0)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("fmt", ["h", "uh", "h2"])
@pytest.mark.parametrize("codec", [None, "aflp", "fpx"])
def test_adjoint_identity(mats, fmt, codec):
    m, f, fa, comp = mats[fmt]
    if codec is not None:
        m = comp(m, codec)
    x = synth.rhs(N, 1, seed=21)[:, 0]
    y = synth.rhs(N, 1, seed=22)[:, 0]
    mx = f(m, 1.0, x, 0.0)
    mty = fa(m, 1.0, y, 0.0)
    lhs, rhs = float(y @ mx), float(mty @ x)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(y) * np.linalg.norm(mx) * 10
    assert np.linalg.norm(mty) > 0


@pytest.mark.parametrize("fmt", ["h", "uh", "h2"])
def test_adjoint_columns_and_scalars(mats, fmt):
    m, _, fa, _ = mats[fmt]
    x = synth.rhs(N, 3, seed=31)
    y0 = synth.rhs(N, 3, seed=32)
    full = fa(m, -1.25, x, 0.5, y0)
    for k in range(3):
        one = fa(m, 1.0, x[:, k], 0.0)
        ref = -1.25 * one + 0.5 * y0[:, k]
        assert np.allclose(full[:, k], ref, rtol=1e-13, atol=1e-13 * np.linalg.norm(ref))


@pytest.fixture(scope="module")
def weighted():
    """The row-weighted Laplace matrix diag(w) A: far from symmetric."""
    pts = synth.sphere_points(N)
    h = hmatrix.build_h(pts, "laplace_w", 32, 2.0, 1e-6)
    return h, nested.build_uniform(h), nested.build_h2(h)


def test_adjoint_of_a_non_symmetric_matrix(weighted):
    """H: adjoint = dense transpose (to 1e-13) and far from the forward product;
    UH, H^2: the adjoint identity and the same distance from the forward product."""
    h, u, h2 = weighted
    a = hmatrix.dense_matrix(h)
    x = synth.rhs(N, 1, seed=51)[:, 0]
    y = synth.rhs(N, 1, seed=52)[:, 0]
    at = matvec.h_mvm_adjoint(h, 1.0, x, 0.0)
    assert np.linalg.norm(at - a.T @ x) <= 1e-13 * np.linalg.norm(a.T @ x)
    fwd = matvec.h_mvm(h, 1.0, x, 0.0)
    assert np.linalg.norm(at - fwd) > 1e-2 * np.linalg.norm(fwd)
    for m, f, fa in ((u, matvec.uh_mvm, matvec.uh_mvm_adjoint), (h2, matvec.h2_mvm, matvec.h2_mvm_adjoint)):
        mx, mty = f(m, 1.0, x, 0.0), fa(m, 1.0, y, 0.0)
        assert abs(float(y @ mx) - float(mty @ x)) <= 1e-11 * np.linalg.norm(y) * np.linalg.norm(mx)
        adj = fa(m, 1.0, x, 0.0)
        assert np.linalg.norm(adj - a.T @ x) <= 4e-6 * np.linalg.norm(a.T @ x)
