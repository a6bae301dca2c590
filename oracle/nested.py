"""Shared (UH, Sec. 2.3) and nested (H^2, Sec. 2.4) cluster bases.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper takes the basis constructions from the literature (BruHuyMee:2025 for
UH, Boerm:2010 for H^2) without printing them; these readings are used:

UH.  For a row cluster t the data matrix is the concatenation of
W_b diag(s_b) / ||s_b||_F over the low-rank blocks b of the block row of t.  Its
SVD gives the orthonormal basis W_t (columns with singular value > eps) and the
singular values Sigma_t.  Column bases X_s are formed in the same way from the
block column.  Each block's projection error is then at most eps relative
(Frobenius).  Coupling: S_ts = (W_t^T W_b) diag(s_b) (X_b^T X_s).  A cluster
without low-rank blocks gets a rank-0 basis.

H^2.  The row basis of t must represent every low-rank block of the block rows
of t and of all its ancestors, restricted to the rows of t (nestedness).  At t
each such block contributes W_b[t,:] diag(s_b) / ||W_b[t,:] diag(s_b)||_F.
At a leaf the SVD of that data gives the leaf basis W_t; at an inner cluster
the data is first projected onto the sons' bases,
[W_t0^T R_t|t0 ; W_t1^T R_t|t1], and the SVD gives the transfer matrices
E_t,0 = Q[:k0], E_t,1 = Q[k0:] with W_t = [W_t0 E_t,0 ; W_t1 E_t,1].  Columns
are kept while their singular value exceeds eps / sqrt(depth + 1), so that the
errors of all levels add up to at most eps relative per block.  Column bases
are built the same way from the block columns.  Couplings as for UH.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .hmatrix import HMatrix, LowRank


def _svd_basis(r: np.ndarray, thr: float):
    """Left singular vectors of r with singular value > thr, and those values."""
    if r.shape[0] == 0 or r.shape[1] == 0:
        return np.zeros((r.shape[0], 0)), np.zeros(0)
    u, s, _ = np.linalg.svd(r, full_matrices=False)
    k = int(np.count_nonzero(s > thr))
    return np.asfortranarray(u[:, :k]), s[:k].copy()


@dataclass
class Uniform:
    """UH-matrix: shared bases per cluster, one coupling matrix per low-rank block."""
    h: HMatrix
    W: list            # row basis per cluster id, (n_t, k_t)
    SW: list           # singular values of the row basis data
    X: list            # column basis per cluster id
    SX: list
    S: list            # per block: coupling (k_t, k_s) for low-rank, dense ndarray otherwise


@dataclass
class H2:
    """H^2-matrix: leaf bases, transfer matrices, one coupling per low-rank block."""
    h: HMatrix
    Wleaf: dict        # leaf cluster id -> (n_t, k_t)
    SWleaf: dict
    EW: dict           # non-root cluster id -> transfer (k_child, k_parent)
    Xleaf: dict
    SXleaf: dict
    EX: dict
    kW: list           # rank per cluster
    kX: list
    Wexp: list         # expanded bases (for construction and tests only)
    Xexp: list
    S: list


def _lowrank_blocks(h: HMatrix):
    return [(i, b, d) for i, (b, d) in enumerate(zip(h.blocks, h.data)) if isinstance(d, LowRank)]


def build_uniform(h: HMatrix) -> Uniform:
    """UH bases and couplings from an H-matrix (Sec. 2.3)."""
    nc = len(h.ct.clusters)
    rowdata = [[] for _ in range(nc)]
    coldata = [[] for _ in range(nc)]
    for _, b, d in _lowrank_blocks(h):
        if d.rank == 0:
            continue
        f = np.linalg.norm(d.s)
        rowdata[b.row].append(d.W * (d.s / f))
        coldata[b.col].append(d.X * (d.s / f))
    W, SW, X, SX = [], [], [], []
    for c in h.ct.clusters:
        n = c.size
        r = np.hstack(rowdata[c.id]) if rowdata[c.id] else np.zeros((n, 0))
        w, sw = _svd_basis(r, h.eps)
        W.append(w)
        SW.append(sw)
        r = np.hstack(coldata[c.id]) if coldata[c.id] else np.zeros((n, 0))
        x, sx = _svd_basis(r, h.eps)
        X.append(x)
        SX.append(sx)
    S = []
    for b, d in zip(h.blocks, h.data):
        if isinstance(d, LowRank):
            S.append((W[b.row].T @ d.W) @ np.diag(d.s) @ (d.X.T @ X[b.col]))
        else:
            S.append(d)
    return Uniform(h, W, SW, X, SX, S)


@dataclass
class UniformSep:
    """UH-matrix with separate row and column coupling matrices per low-rank
    block (the variant discussed after Alg. 5): S_ts = Sr_b Sc_b^H with
    Sr_b = (W_t^T W_b) diag(s_b) (k_t x k_b) and Sc_b = X_s^T X_b (k_s x k_b),
    the two factors of the coupling above, kept apart."""
    u: Uniform
    Sr: list           # per block: (k_t, k_b) for low-rank, None otherwise
    Sc: list           # per block: (k_s, k_b) for low-rank, None otherwise


def build_uniform_sep(h: HMatrix) -> UniformSep:
    u = build_uniform(h)
    Sr, Sc = [], []
    for b, d in zip(h.blocks, h.data):
        if isinstance(d, LowRank):
            Sr.append((u.W[b.row].T @ d.W) @ np.diag(d.s))
            Sc.append(u.X[b.col].T @ d.X)
        else:
            Sr.append(None)
            Sc.append(None)
    return UniformSep(u, Sr, Sc)


def _nested_side(h: HMatrix, side: str):
    """Nested bases for one side ('row' uses W_b, 'col' uses X_b)."""
    cl = h.ct.clusters
    nc = len(cl)
    own = [[] for _ in range(nc)]          # low-rank blocks whose row/col cluster is c
    for _, b, d in _lowrank_blocks(h):
        if d.rank == 0:
            continue
        cid = b.row if side == "row" else b.col
        own[cid].append(d.W if side == "row" else d.X)
        own[cid][-1] = own[cid][-1] * d.s   # factor times singular values
    # contributing blocks of c: own blocks of c and of every ancestor, with offset of c
    contrib = [[] for _ in range(nc)]
    for c in cl:
        a = c.id
        while a >= 0:
            off = c.start - cl[a].start
            for f in own[a]:
                contrib[c.id].append(f[off:off + c.size])
            a = cl[a].parent
    depth = h.ct.depth()
    thr = h.eps / np.sqrt(depth + 1.0)
    leafb, leafs, E = {}, {}, {}
    k = [0] * nc
    exp = [None] * nc

    def normed(fs):
        cols = []
        for f in fs:
            nf = np.linalg.norm(f)
            if nf > 0:
                cols.append(f / nf)
        return cols

    for c in sorted(cl, key=lambda c: -c.level):     # leaves to root
        fs = normed(contrib[c.id])
        if c.is_leaf:
            r = np.hstack(fs) if fs else np.zeros((c.size, 0))
            w, sw = _svd_basis(r, thr)
            leafb[c.id], leafs[c.id] = w, sw
            k[c.id] = w.shape[1]
            exp[c.id] = w
            continue
        s0, s1 = c.sons
        c0, c1 = cl[s0], cl[s1]
        if fs:
            r = np.hstack(fs)
            n0 = c0.size
            rh = np.vstack([exp[s0].T @ r[:n0], exp[s1].T @ r[n0:]])
        else:
            rh = np.zeros((k[s0] + k[s1], 0))
        q, _ = _svd_basis(rh, thr)
        k[c.id] = q.shape[1]
        E[s0] = np.asfortranarray(q[:k[s0]])
        E[s1] = np.asfortranarray(q[k[s0]:])
        exp[c.id] = np.vstack([exp[s0] @ E[s0], exp[s1] @ E[s1]])
    return leafb, leafs, E, k, exp


def build_h2(h: HMatrix) -> H2:
    """H^2 nested bases, transfers and couplings from an H-matrix (Sec. 2.4)."""
    wl, wls, ew, kw, wexp = _nested_side(h, "row")
    xl, xls, ex, kx, xexp = _nested_side(h, "col")
    S = []
    for b, d in zip(h.blocks, h.data):
        if isinstance(d, LowRank):
            S.append((wexp[b.row].T @ d.W) @ np.diag(d.s) @ (d.X.T @ xexp[b.col]))
        else:
            S.append(d)
    return H2(h, wl, wls, ew, xl, xls, ex, kw, kx, wexp, xexp, S)
