"""Triangular vector solves with H-LU factors (Sec. 5, Conclusion: the outlook names
triangular solves for H-LU factorisations as the next operation that reads the
same compressed blocks as the product).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper names the operation only; these are the readings:

* Factors.  A = L U without pivoting, L unit lower and U upper triangular, in
  the cluster (permuted) order.  The model problem is the Matern covariance
  matrix: it is symmetric positive definite, so the unpivoted factorisation
  exists and its entries stay bounded by those of A.  (The Laplace matrix of
  the point model is indefinite; unpivoted elimination shows pivot growth of
  about 10^4 there, so it is not used for the solve.)
* H-format factors.  L and U are approximated on the block tree of A: a leaf
  block (t, s) with t after s lies in L, one with t before s in U, and a
  diagonal leaf (t, t) carries the unit lower part of L_tt and the upper part
  of U_tt.  Admissible blocks keep the truncated SVD of the exact factor block
  with the rule of eqn. epsilon (relative spectral cut, ``hmatrix.truncate_rank``);
  inadmissible blocks are exact.  The exact factors come from dense elimination
  of the exact matrix -- the plain definition that an H-arithmetic LU reaches up
  to its own truncation errors.
* Solve.  x := U^{-1} L^{-1} b by block forward substitution and then block
  backward substitution over the cluster tree: at a leaf cluster t the dense
  triangle of the diagonal block is solved; at an inner cluster the sons are
  solved in order and each solved son t_i updates every later son t_j with the
  sub-block L_{t_j t_i} (backward: in reverse order with U_{t_j t_i}).  The
  off-diagonal updates are products with leaf blocks (``matvec.h_block_apply``,
  Alg. 1 per block, Alg. 8 decoding for compressed factors).
* Compression.  Each factor is compressed like an H-matrix (``compress.compress_h``):
  direct compression of dense blocks, VALR columns of low-rank blocks.  The unit
  diagonal of L is implied: the solve reads only the strict lower part of its
  diagonal blocks.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.linalg import solve_triangular

from . import kernels
from .compress import CH, compress_h, undirect, unvalr
from .hmatrix import HMatrix, LowRank, truncate_rank
from .matvec import h_block_apply
from .trees import build_block_tree, build_cluster_tree


@dataclass
class HLU:
    L: HMatrix         # blocks on and below the block diagonal
    U: HMatrix         # blocks on and above the block diagonal


def lu_nopivot(a: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Doolittle elimination without pivoting: a = L U, L unit lower, U upper."""
    u = np.array(a, dtype=np.float64, copy=True)
    n = u.shape[0]
    for k in range(n):
        u[k + 1:, k] /= u[k, k]
        u[k + 1:, k + 1:] -= np.outer(u[k + 1:, k], u[k, k + 1:])
    return np.tril(u, -1) + np.eye(n), np.triu(u)


def _truncated(a: np.ndarray, eps: float) -> LowRank:
    w, s, vt = np.linalg.svd(a, full_matrices=False)
    k = truncate_rank(s, eps)
    return LowRank(np.asfortranarray(w[:, :k]), s[:k].copy(), np.asfortranarray(vt[:k, :].T))


def build_hlu(pts: np.ndarray, kind: str, leaf: int, eta: float, eps: float,
              param: float | None = None) -> tuple[HLU, np.ndarray, np.ndarray]:
    """H-format factors of the model matrix on ``pts``; also returns the exact
    factors (cluster order) they approximate."""
    n = pts.shape[0]
    if param is None:
        param = kernels.default_param(kind, n)
    ct = build_cluster_tree(pts, leaf)
    blocks = build_block_tree(ct, eta)
    ap = kernels.entries(kind, pts, ct.perm, ct.perm, param)
    lx, ux = lu_nopivot(ap)
    lb, ld, ub, ud = [], [], [], []
    for b in blocks:
        t, s = ct.clusters[b.row], ct.clusters[b.col]
        rs, cs = slice(t.start, t.end), slice(s.start, s.end)
        if b.row == b.col:
            lb.append(b)
            ld.append(np.tril(lx[rs, cs]))
            ub.append(b)
            ud.append(np.triu(ux[rs, cs]))
            continue
        blk, tb, td = (lx[rs, cs], lb, ld) if t.start >= s.end else (ux[rs, cs], ub, ud)
        tb.append(b)
        td.append(_truncated(blk, eps) if b.adm else blk.copy())
    L = HMatrix(kind, param, eps, ct, lb, ld, pts)
    U = HMatrix(kind, param, eps, ct, ub, ud, pts)
    return HLU(L, U), lx, ux


def compress_hlu(f: HLU, codec: str) -> tuple[CH, CH]:
    return compress_h(f.L, codec), compress_h(f.U, codec)


def dense_factor(m) -> np.ndarray:
    """Expand an H-format factor (FP64 or compressed) in the cluster order."""
    h = m if isinstance(m, HMatrix) else m.h
    out = np.zeros((h.n, h.n))
    for i, b in enumerate(h.blocks):
        t, s = h.ct.clusters[b.row], h.ct.clusters[b.col]
        out[t.start:t.end, s.start:s.end] = _block(m, i)
    return out


def _block(m, i: int) -> np.ndarray:
    """Leaf block i of a factor as a dense array (compressed blocks decoded, Alg. 8)."""
    if isinstance(m, HMatrix):
        d = m.data[i]
        return (d.W * d.s) @ d.X.T if isinstance(d, LowRank) else d
    h = m.h
    t, s = h.ct.clusters[h.blocks[i].row], h.ct.clusters[h.blocks[i].col]
    blk = m.blocks[i]
    if blk[0] == "lr":
        return (unvalr(blk[2], t.size) * blk[1]) @ unvalr(blk[3], s.size).T
    return undirect(blk[1])


def _diag_blocks(h: HMatrix) -> dict:
    return {b.row: i for i, b in enumerate(h.blocks) if b.row == b.col}


def _sub_blocks(h: HMatrix, t, s) -> list:
    """Leaf blocks whose rows lie in cluster t and columns in cluster s: together
    they tile the sub-block M_ts (the block tree partitions I x I)."""
    cl = h.ct.clusters
    out = []
    for i, b in enumerate(h.blocks):
        r, c = cl[b.row], cl[b.col]
        if t.start <= r.start and r.end <= t.end and s.start <= c.start and c.end <= s.end:
            out.append(i)
    return out


def forward(mL, z: np.ndarray) -> None:
    """z := L^{-1} z in place (cluster order), block forward substitution."""
    h = mL if isinstance(mL, HMatrix) else mL.h
    cl = h.ct.clusters
    diag = _diag_blocks(h)

    def rec(t: int) -> None:
        c = cl[t]
        if c.is_leaf:
            z[c.start:c.end] = solve_triangular(_block(mL, diag[t]), z[c.start:c.end],
                                                lower=True, unit_diagonal=True)
            return
        for i, ti in enumerate(c.sons):
            rec(ti)
            for tj in c.sons[i + 1:]:
                for k in _sub_blocks(h, cl[tj], cl[ti]):
                    h_block_apply(mL, k, -1.0, z, z)

    rec(0)


def backward(mU, z: np.ndarray) -> None:
    """z := U^{-1} z in place (cluster order), block backward substitution."""
    h = mU if isinstance(mU, HMatrix) else mU.h
    cl = h.ct.clusters
    diag = _diag_blocks(h)

    def rec(t: int) -> None:
        c = cl[t]
        if c.is_leaf:
            z[c.start:c.end] = solve_triangular(_block(mU, diag[t]), z[c.start:c.end], lower=False)
            return
        for i in range(len(c.sons) - 1, -1, -1):
            ti = c.sons[i]
            rec(ti)
            for tj in c.sons[:i]:
                for k in _sub_blocks(h, cl[tj], cl[ti]):
                    h_block_apply(mU, k, -1.0, z, z)

    rec(0)


def hlu_solve(mL, mU, b) -> np.ndarray:
    """x := U^{-1} L^{-1} b for b in the original point order, shape (N,) or (N, r)."""
    h = mL if isinstance(mL, HMatrix) else mL.h
    perm = h.ct.perm
    z = np.array(np.asarray(b, dtype=np.float64)[perm], copy=True)
    forward(mL, z)
    backward(mU, z)
    x = np.empty_like(z)
    x[perm] = z
    return x
