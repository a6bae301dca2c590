"""H(T, eps) construction (Sec. 2.2, eqn. epsilon) by truncated SVD.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Reading of eqn. epsilon (the norm is not named): each admissible block keeps the
smallest rank k with sigma_k <= eps * sigma_0 (spectral, relative), computed
from the SVD of the exact block.  A block is stored as W diag(sigma) X^T with
orthonormal W (rows of the row cluster) and X (rows of the column cluster).
Dense (inadmissible) blocks hold the exact entries.  All data are indexed in
the cluster (permuted) order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import kernels
from .trees import ClusterTree, build_block_tree, build_cluster_tree


@dataclass
class LowRank:
    W: np.ndarray      # (n_t, k)
    s: np.ndarray      # (k,)
    X: np.ndarray      # (n_s, k)

    @property
    def rank(self) -> int:
        return self.s.shape[0]


@dataclass
class HMatrix:
    kind: str
    param: float
    eps: float
    ct: ClusterTree
    blocks: list       # trees.Block
    data: list         # LowRank for admissible blocks, ndarray for dense blocks
    pts: np.ndarray

    @property
    def n(self) -> int:
        return self.ct.perm.shape[0]

    def rows(self, cid: int) -> np.ndarray:
        c = self.ct.clusters[cid]
        return self.ct.perm[c.start:c.end]


def truncate_rank(s: np.ndarray, eps: float) -> int:
    """Rank k with sigma_k <= eps*sigma_0 < sigma_{k-1}: the count of sigma_i > eps*sigma_0."""
    if s.size == 0 or s[0] == 0.0:
        return 0
    return int(np.count_nonzero(s > eps * s[0]))


def build_h(pts: np.ndarray, kind: str, leaf: int, eta: float, eps: float,
            param: float | None = None, adm: str = "std") -> HMatrix:
    """Build an H-matrix of the model kernel on ``pts`` (exact SVD per block);
    ``adm`` picks the admissibility (``trees.block_admissible``: standard,
    HODLR, BLR)."""
    n = pts.shape[0]
    if param is None:
        param = kernels.default_param(kind, n)
    ct = build_cluster_tree(pts, leaf)
    blocks = build_block_tree(ct, eta, adm)
    data = []
    for b in blocks:
        rt = ct.perm[ct.clusters[b.row].start:ct.clusters[b.row].end]
        cs = ct.perm[ct.clusters[b.col].start:ct.clusters[b.col].end]
        a = kernels.entries(kind, pts, rt, cs, param)
        if not b.adm:
            data.append(a)
            continue
        u, s, vt = np.linalg.svd(a, full_matrices=False)
        k = truncate_rank(s, eps)
        data.append(LowRank(np.asfortranarray(u[:, :k]), s[:k].copy(),
                            np.asfortranarray(vt[:k, :].T)))
    return HMatrix(kind, param, eps, ct, blocks, data, pts)


def dense_matrix(h: HMatrix) -> np.ndarray:
    """Expand an H-matrix to a dense FP64 matrix in the original index order."""
    a = np.zeros((h.n, h.n))
    for b, d in zip(h.blocks, h.data):
        r = h.rows(b.row)
        c = h.rows(b.col)
        if isinstance(d, LowRank):
            a[np.ix_(r, c)] = (d.W * d.s) @ d.X.T
        else:
            a[np.ix_(r, c)] = d
    return a


def exact_matrix(pts: np.ndarray, kind: str, param: float) -> np.ndarray:
    n = pts.shape[0]
    idx = np.arange(n)
    return kernels.entries(kind, pts, idx, idx, param)
