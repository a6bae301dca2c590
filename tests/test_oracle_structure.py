"""Pins of the oracle's trees, construction and products.

Checked against the definitions (Def. Cluster Tree, Def. Block Tree), the exact
kernel matrix, numpy's LAPACK SVD, and the dense product A x written out.
"""
import numpy as np
import pytest

import synth
from oracle import compress, hmatrix, kernels, matvec, nested, trees


@pytest.fixture(scope="module")
def sphere512():
    pts = synth.sphere_points(512)
    h = hmatrix.build_h(pts, "laplace", 16, 2.0, 1e-6)
    return pts, h


@pytest.fixture(scope="module")
def sphere2048():
    pts = synth.sphere_points(2048)
    h = hmatrix.build_h(pts, "laplace", 32, 2.0, 1e-6)
    a = hmatrix.exact_matrix(pts, "laplace", h.param)
    return pts, h, a


def test_points_on_sphere_and_cube():
    p = synth.sphere_points(1000)
    assert np.allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-14)
    assert len(np.unique(p.round(12), axis=0)) == 1000
    q = synth.cube_points(1000)
    assert q.min() >= 0 and q.max() <= 1


def test_kernel_entries_closed_form():
    p = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, 2.0, 0]])
    idx = np.arange(3)
    a = kernels.entries("laplace", p, idx, idx, 0.5)
    assert a[0, 1] == pytest.approx(1 / (4 * np.pi))
    assert a[1, 2] == pytest.approx(1 / (4 * np.pi * np.sqrt(5)))
    assert a[0, 0] == pytest.approx(1 / (4 * np.pi * 0.5))
    b = kernels.entries("matern", p, idx, idx, 0.1)
    t = np.sqrt(3) * 1.0 / 0.1
    assert b[0, 1] == pytest.approx((1 + t) * np.exp(-t))
    assert b[2, 2] == 1.0
    assert kernels.default_param("laplace", 100) == pytest.approx(np.sqrt(4 * np.pi / 100))
    # general positions (every coordinate differs) against scipy's pairwise distances
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(11)
    q = rng.uniform(-1, 1, (7, 3))
    idx = np.arange(7)
    r = cdist(q, q)
    off = ~np.eye(7, dtype=bool)
    a = kernels.entries("laplace", q, idx, idx, 0.5)
    assert np.allclose(a[off], 1 / (4 * np.pi * r[off]), rtol=1e-14, atol=0)
    b = kernels.entries("matern", q, idx, idx, 0.1)
    t = np.sqrt(3) * r / 0.1
    assert np.allclose(b, (1 + t) * np.exp(-t), rtol=1e-13, atol=1e-300)
    # one pair by hand: |(0.1, 0.2, 0.3) - (0.4, -0.5, 0.9)|^2 = 0.09 + 0.49 + 0.36
    h = np.array([[0.1, 0.2, 0.3], [0.4, -0.5, 0.9]])
    assert kernels.entries("laplace", h, np.arange(2), np.arange(2), 0.5)[0, 1] == pytest.approx(
        1 / (4 * np.pi * np.sqrt(0.94)), rel=1e-15)


def test_row_weighted_kernel_is_diag_w_times_laplace():
    """laplace_w = diag(1 + x_i / 2) A: rows scaled by the weight of their own
    point (not the column's), so the matrix is not symmetric."""
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(12)
    q = rng.uniform(-1, 1, (6, 3))
    idx = np.arange(6)
    r = cdist(q, q)
    off = ~np.eye(6, dtype=bool)
    w = 1 + q[:, 0] / 2
    a = kernels.entries("laplace_w", q, idx, idx, 0.5)
    want = w[:, None] / (4 * np.pi * np.where(off, r, 1.0))
    want[~off] = w / (4 * np.pi * 0.5)
    assert np.allclose(a, want, rtol=1e-14, atol=0)
    assert not np.allclose(a, a.T, rtol=1e-3)
    # a sub-block is the same rows and columns of the whole matrix
    sub = kernels.entries("laplace_w", q, np.array([4, 1]), np.array([0, 5, 2]), 0.5)
    assert np.array_equal(sub, a[np.ix_([4, 1], [0, 5, 2])])
    assert kernels.default_param("laplace_w", 100) == kernels.default_param("laplace", 100)


def test_cluster_tree_definition(sphere512):
    pts, h = sphere512
    ct = h.ct
    n = pts.shape[0]
    assert sorted(ct.perm.tolist()) == list(range(n))
    root = ct.root
    assert (root.start, root.end) == (0, n)
    for c in ct.clusters:
        q = pts[ct.perm[c.start:c.end]]
        assert np.array_equal(c.lo, q.min(axis=0)) and np.array_equal(c.hi, q.max(axis=0))
        if c.is_leaf:
            assert c.size <= 16
            continue
        assert c.size > 16 and len(c.sons) == 2
        s0, s1 = (ct.clusters[s] for s in c.sons)
        assert s0.start == c.start and s0.end == s1.start and s1.end == c.end
        assert s0.level == s1.level == c.level + 1
        ext = c.hi - c.lo
        ax = int(np.argmax(ext))
        mid = 0.5 * (c.lo[ax] + c.hi[ax])
        assert np.all(pts[ct.perm[s0.start:s0.end], ax] < mid)
        assert np.all(pts[ct.perm[s1.start:s1.end], ax] >= mid)


def test_block_tree_definition(sphere512):
    pts, h = sphere512
    ct = h.ct
    n = pts.shape[0]
    cover = np.zeros((n, n), dtype=np.int32)
    for b in h.blocks:
        t, s = ct.clusters[b.row], ct.clusters[b.col]
        cover[t.start:t.end, s.start:s.end] += 1
        assert t.level == s.level
        # admissibility written with square roots (standard form)
        dt = np.linalg.norm(t.hi - t.lo)
        ds = np.linalg.norm(s.hi - s.lo)
        gap = np.maximum(0, np.maximum(s.lo - t.hi, t.lo - s.hi))
        dist = np.linalg.norm(gap)
        if b.adm:
            assert dist > 0 and min(dt, ds) <= 2.0 * dist * (1 + 1e-12)
        else:
            assert t.is_leaf or s.is_leaf
            assert dist == 0 or min(dt, ds) >= 2.0 * dist * (1 - 1e-12)
    assert np.all(cover == 1)


def test_truncated_svd_against_lapack(sphere2048):
    pts, h, a = sphere2048
    perm = h.ct.perm
    nlr = 0
    for b, d in zip(h.blocks, h.data):
        r = h.rows(b.row)
        c = h.rows(b.col)
        blk = a[np.ix_(r, c)]
        if not isinstance(d, hmatrix.LowRank):
            assert np.array_equal(d, blk)
            continue
        nlr += 1
        s = np.linalg.svd(blk, compute_uv=False)
        k = d.rank
        assert s[k] <= 1e-6 * s[0] < s[k - 1] if k < len(s) else True
        assert np.allclose(d.s, s[:k], rtol=1e-12)
        err = np.linalg.norm(blk - (d.W * d.s) @ d.X.T, 2)
        assert err <= 1e-6 * s[0] * (1 + 1e-8)
        assert np.allclose(d.W.T @ d.W, np.eye(k), atol=1e-12)
        assert np.allclose(d.X.T @ d.X, np.eye(k), atol=1e-12)
    assert nlr > 100
    assert perm.shape[0] == 2048


def test_h_mvm_alg1_against_dense(sphere2048):
    pts, h, a = sphere2048
    x = synth.rhs(2048, 3)
    y0 = synth.rhs(2048, 3, seed=99)
    yd = matvec.dense_mvm(a, 0.7, x, 0.3, y0)
    yh = matvec.h_mvm(h, 0.7, x, 0.3, y0)
    rel = np.linalg.norm(yh - yd) / np.linalg.norm(yd)
    assert rel <= 2e-6
    # Alg. 1 is a reordering of the product with the assembled H-matrix
    ah = hmatrix.dense_matrix(h)
    ye = matvec.dense_mvm(ah, 0.7, x, 0.3, y0)
    assert np.linalg.norm(yh - ye) / np.linalg.norm(ye) <= 1e-14


def test_uniform_and_h2_products(sphere2048):
    pts, h, a = sphere2048
    x = synth.rhs(2048, 2)
    yd = a @ x
    u = nested.build_uniform(h)
    for c in h.ct.clusters:
        for w in (u.W[c.id], u.X[c.id]):
            assert np.allclose(w.T @ w, np.eye(w.shape[1]), atol=1e-12)
    yu = matvec.uh_mvm(u, 1.0, x)
    assert np.linalg.norm(yu - yd) / np.linalg.norm(yd) <= 4e-6
    # Alg. 4 + 5 equal the product with the UH-matrix written out as dense blocks
    au = np.zeros_like(a)
    for b, s in zip(h.blocks, u.S):
        r, c = h.rows(b.row), h.rows(b.col)
        au[np.ix_(r, c)] = (u.W[b.row] @ s @ u.X[b.col].T) if b.adm else s
    assert np.linalg.norm(yu - au @ x) / np.linalg.norm(yu) <= 1e-14
    # per-block error of the shared bases: at most 3 eps relative (H error + two projections)
    for b, d, s in zip(h.blocks, h.data, u.S):
        if b.adm and d.rank:
            blk = a[np.ix_(h.rows(b.row), h.rows(b.col))]
            e = np.linalg.norm(blk - u.W[b.row] @ s @ u.X[b.col].T) / np.linalg.norm(blk)
            assert e <= 3e-6
    m2 = nested.build_h2(h)
    for c in h.ct.clusters:                    # nestedness and orthonormality
        w = m2.Wexp[c.id]
        assert np.allclose(w.T @ w, np.eye(w.shape[1]), atol=1e-11)
        if not c.is_leaf:
            s0, s1 = c.sons
            stacked = np.vstack([m2.Wexp[s0] @ m2.EW[s0], m2.Wexp[s1] @ m2.EW[s1]])
            assert np.allclose(stacked, w, atol=1e-14)
    y2 = matvec.h2_mvm(m2, 1.0, x)
    assert np.linalg.norm(y2 - yd) / np.linalg.norm(yd) <= 4e-6
    a2 = np.zeros_like(a)
    for b, s in zip(h.blocks, m2.S):
        r, c = h.rows(b.row), h.rows(b.col)
        a2[np.ix_(r, c)] = (m2.Wexp[b.row] @ s @ m2.Xexp[b.col].T) if b.adm else s
    assert np.linalg.norm(y2 - a2 @ x) / np.linalg.norm(y2) <= 1e-14


@pytest.mark.parametrize("codec", ["aflp", "fpx"])
def test_compressed_products_follow_eps(sphere2048, codec):
    pts, h, a = sphere2048
    x = synth.rhs(2048, 1)
    yd = a @ x
    yh = matvec.h_mvm(h, 1.0, x)
    ch = compress.compress_h(h, codec)
    yc = matvec.h_mvm(ch, 1.0, x)
    assert np.linalg.norm(yc - yh) / np.linalg.norm(yh) <= 1e-6
    assert np.linalg.norm(yc - yd) / np.linalg.norm(yd) <= 2e-6
    # VALR bound per block (eqn. valr with the compensated delta)
    for d, blk in zip(h.data, ch.blocks):
        if blk[0] != "lr" or d.rank == 0:
            continue
        W = compress.unvalr(blk[2], d.W.shape[0])
        X = compress.unvalr(blk[3], d.X.shape[0])
        e = np.linalg.norm((d.W * d.s) @ d.X.T - (W * d.s) @ X.T)
        k = d.rank
        delta = 1e-6 * np.linalg.norm(d.s) / (1 + 2 * k)
        assert e <= delta * (2 * k + delta * np.sum(1 / d.s)) * (1 + 1e-6)
        assert e <= 1e-6 * np.linalg.norm(d.s)
    u = nested.build_uniform(h)
    cu = compress.compress_uh(u, codec)
    yu = matvec.uh_mvm(u, 1.0, x)
    ycu = matvec.uh_mvm(cu, 1.0, x)
    assert np.linalg.norm(ycu - yu) / np.linalg.norm(yu) <= 2e-6
    # eqn. valrcb: ||W Sigma - W~ Sigma||_F <= k delta = eps
    for c in h.ct.clusters:
        w, sw = u.W[c.id], u.SW[c.id]
        if w.shape[1] == 0:
            continue
        wt = compress.unvalr(cu.W[c.id], c.size)
        assert np.linalg.norm((w - wt) * sw) <= 1e-6 * (1 + 1e-9)
    m2 = nested.build_h2(h)
    c2 = compress.compress_h2(m2, codec)
    y2 = matvec.h2_mvm(m2, 1.0, x)
    yc2 = matvec.h2_mvm(c2, 1.0, x)
    assert np.linalg.norm(yc2 - y2) / np.linalg.norm(y2) <= 2e-6
    assert compress.payload_bytes(ch) < compress.payload_bytes(compress.compress_h(h, "none")) / 2


@pytest.mark.parametrize("adm", ["hodlr", "blr"])
def test_block_tree_other_admissibility(adm):
    """HODLR (off-diagonal admissibility) and BLR (a single level), the remark
    after Def. H-Matrix: the leaves still partition I x I exactly once; HODLR
    keeps dense blocks only on the diagonal and every block of two distinct
    clusters low rank; BLR tests admissibility only where a leaf cluster is
    involved, so no low-rank block sits above the leaf level."""
    pts = synth.sphere_points(512)
    ct = trees.build_cluster_tree(pts, 16)
    blocks = trees.build_block_tree(ct, 2.0, adm)
    n = pts.shape[0]
    cover = np.zeros((n, n), dtype=np.int32)
    for b in blocks:
        t, s = ct.clusters[b.row], ct.clusters[b.col]
        cover[t.start:t.end, s.start:s.end] += 1
        if adm == "hodlr":
            assert b.adm == (b.row != b.col)
            if not b.adm:
                assert t.is_leaf and s.is_leaf
        else:
            assert t.is_leaf or s.is_leaf
            if b.adm:
                assert trees.admissible(t, s, 2.0)
    assert np.all(cover == 1)
    std = trees.build_block_tree(ct, 2.0, "std")
    if adm == "hodlr":
        # every level contributes its two off-diagonal sibling blocks
        nonleaf = sum(1 for c in ct.clusters if not c.is_leaf)
        assert sum(b.adm for b in blocks) == 2 * nonleaf
    else:
        assert len(blocks) > len(std)


@pytest.mark.parametrize("adm", ["hodlr", "blr"])
def test_other_admissibility_products_against_dense(adm):
    pts = synth.sphere_points(1024)
    h = hmatrix.build_h(pts, "laplace", 32, 2.0, 1e-6, adm=adm)
    a = hmatrix.exact_matrix(pts, "laplace", h.param)
    x = synth.rhs(1024, 2)
    yd = matvec.dense_mvm(a, 1.0, x)
    yh = matvec.h_mvm(h, 1.0, x)
    assert np.linalg.norm(yh - yd) / np.linalg.norm(yd) <= 2e-6
    ya = matvec.h_mvm_adjoint(h, 1.0, x)
    assert np.linalg.norm(ya - a.T @ x) / np.linalg.norm(a.T @ x) <= 2e-6


@pytest.mark.parametrize("codec", [None, "aflp"])
def test_uh_separate_couplings(sphere2048, codec):
    """The UH variant with separate row and column couplings (S = Sr Sc^H,
    discussed after Alg. 5): the factors reproduce the single coupling, the
    product equals the single-coupling UH product up to rounding (uncompressed)
    and follows eps against the dense kernel (compressed); its adjoint form
    satisfies the adjoint identity."""
    pts, h, a = sphere2048
    us = nested.build_uniform_sep(h)
    for b, r, c, s in zip(h.blocks, us.Sr, us.Sc, us.u.S):
        if b.adm:
            assert np.linalg.norm(r @ c.T - s) <= 1e-13 * max(1.0, np.linalg.norm(s))
    m = us if codec is None else compress.compress_uh_sep(us, codec)
    x = synth.rhs(2048, 2, seed=5)
    got = matvec.uhsep_mvm(m, 0.5, x, 0.0)
    if codec is None:
        ref = matvec.uh_mvm(us.u, 0.5, x, 0.0)
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    yd = matvec.dense_mvm(a, 0.5, x)
    assert np.linalg.norm(got - yd) / np.linalg.norm(yd) <= 4e-6
    y = synth.rhs(2048, 1, seed=6)[:, 0]
    lhs = float(y @ matvec.uhsep_mvm(m, 1.0, x[:, 0], 0.0))
    rhs = float(matvec.uhsep_mvm(m, 1.0, y, 0.0, adjoint=True) @ x[:, 0])
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_uncompressed_codec_and_payload_counts(sphere512):
    """codec "none" keeps FP64 values: the compressed-form products equal the FP64
    products, and the payload is 8 bytes per stored value, counted from the
    structure (dense entries, k (n_t + n_s) per low-rank block, basis, coupling
    and transfer entries)."""
    pts, h = sphere512
    x = synth.rhs(512, 2)
    cl = h.ct.clusters
    ch = compress.compress_h(h, "none")
    assert np.linalg.norm(matvec.h_mvm(ch, 1.0, x) - matvec.h_mvm(h, 1.0, x)) <= 1e-14 * np.linalg.norm(x)
    vals = sum(d.size if not b.adm else d.rank * (cl[b.row].size + cl[b.col].size)
               for b, d in zip(h.blocks, h.data))
    assert compress.payload_bytes(ch) == 8 * vals
    u = nested.build_uniform(h)
    cu = compress.compress_uh(u, "none")
    yu = matvec.uh_mvm(u, 1.0, x)
    assert np.linalg.norm(matvec.uh_mvm(cu, 1.0, x) - yu) <= 1e-13 * np.linalg.norm(yu)
    vals = sum(w.size for w in u.W) + sum(w.size for w in u.X) + sum(s.size for s in u.S)
    assert compress.payload_bytes(cu) == 8 * vals
    m2 = nested.build_h2(h)
    c2 = compress.compress_h2(m2, "none")
    y2 = matvec.h2_mvm(m2, 1.0, x)
    assert np.linalg.norm(matvec.h2_mvm(c2, 1.0, x) - y2) <= 1e-13 * np.linalg.norm(y2)
    vals = (sum(w.size for w in m2.Wleaf.values()) + sum(w.size for w in m2.Xleaf.values())
            + sum(e.size for e in m2.EW.values()) + sum(e.size for e in m2.EX.values())
            + sum(s.size for s in m2.S))
    assert compress.payload_bytes(c2) == 8 * vals


def test_bisection_point_on_the_midpoint_goes_to_the_second_son():
    # points at 0, 0.5, 1 on the x axis: mid = 0.5 exactly, "< mid" forms the first son
    p = np.array([[0.0, 0, 0], [0.5, 0, 0], [1.0, 0, 0]])
    ct = trees.build_cluster_tree(p, 1)
    root = ct.root
    s0, s1 = (ct.clusters[i] for i in root.sons)
    assert (s0.size, s1.size) == (1, 2)
    assert ct.perm[s0.start] == 0 and sorted(ct.perm[s1.start:s1.end].tolist()) == [1, 2]
