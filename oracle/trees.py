"""Cluster tree (Def. Cluster Tree) and block tree (Def. Block Tree), Sec. 2.2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Readings (the paper only cites the constructions):

* Binary geometric bisection: a cluster with more than ``leaf`` points is split
  at the midpoint 0.5*(lo+hi) of the longest edge of its tight bounding box
  (ties: lowest axis); points with coordinate < mid form the first son, the
  others the second, both keeping their order.  If a side would be empty the
  cluster is split into its first floor(n/2) and remaining points.
* Standard admissibility (cited in Sec. 2.2), in squared form so that it is
  evaluated without square roots:
      adm(t, s)  <=>  dist^2 > 0  and  min(diam_t^2, diam_s^2) <= eta^2 dist^2,
  diam^2 = (dx*dx + dy*dy) + dz*dz of the bounding box, dist^2 the same sum of
  the squared axis gaps between the two boxes.
* Block tree: a block is a leaf if admissible or if either cluster is a leaf;
  otherwise its sons are all pairs of sons (Def. Block Tree).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Cluster:
    start: int                    # first position in the cluster (permuted) order
    end: int                      # one past the last position
    level: int
    lo: np.ndarray                # bounding box
    hi: np.ndarray
    sons: list = field(default_factory=list)
    parent: int = -1
    id: int = -1

    @property
    def size(self) -> int:
        return self.end - self.start

    @property
    def is_leaf(self) -> bool:
        return not self.sons


@dataclass
class ClusterTree:
    clusters: list                # Cluster objects, pre-order; clusters[0] is the root
    perm: np.ndarray              # perm[position] = original point index

    @property
    def root(self) -> Cluster:
        return self.clusters[0]

    def leaves(self):
        return [c for c in self.clusters if c.is_leaf]

    def depth(self) -> int:
        return max(c.level for c in self.clusters)


def build_cluster_tree(pts: np.ndarray, leaf: int) -> ClusterTree:
    """Binary geometric bisection cluster tree (Def. Cluster Tree)."""
    n = pts.shape[0]
    clusters: list = []
    perm = np.empty(n, dtype=np.int64)

    def rec(idx: np.ndarray, start: int, level: int, parent: int) -> int:
        p = pts[idx]
        lo = p.min(axis=0)
        hi = p.max(axis=0)
        c = Cluster(start, start + len(idx), level, lo, hi, parent=parent, id=len(clusters))
        clusters.append(c)
        if len(idx) <= leaf:
            perm[start:start + len(idx)] = idx
            return c.id
        ext = hi - lo
        axis = int(np.argmax(ext))
        mid = 0.5 * (lo[axis] + hi[axis])
        left = idx[p[:, axis] < mid]
        right = idx[p[:, axis] >= mid]
        if len(left) == 0 or len(right) == 0:
            h = len(idx) // 2
            left, right = idx[:h], idx[h:]
        c.sons.append(rec(left, start, level + 1, c.id))
        c.sons.append(rec(right, start + len(left), level + 1, c.id))
        return c.id

    rec(np.arange(n, dtype=np.int64), 0, 0, -1)
    return ClusterTree(clusters, perm)


def diam2(c: Cluster) -> float:
    d = c.hi - c.lo
    return float((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])


def dist2(a: Cluster, b: Cluster) -> float:
    g = [max(0.0, float(b.lo[i] - a.hi[i]), float(a.lo[i] - b.hi[i])) for i in range(3)]
    return (g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]


def admissible(a: Cluster, b: Cluster, eta: float) -> bool:
    d2 = dist2(a, b)
    return d2 > 0.0 and min(diam2(a), diam2(b)) <= (eta * eta) * d2


@dataclass
class Block:
    row: int                      # row cluster id
    col: int                      # column cluster id
    adm: bool


ADM_MODES = ("std", "hodlr", "blr")


def block_admissible(a: Cluster, b: Cluster, eta: float, mode: str) -> bool:
    """The admissibility condition of the block tree.  The remark after Def.
    H-Matrix: BLR and HODLR are H-matrices whose clustering or admissibility is
    chosen accordingly.

    * ``std``   -- standard admissibility with parameter eta (``admissible``);
    * ``hodlr`` -- off-diagonal admissibility: every block of two distinct
      clusters is admissible, inadmissibility restricted to the diagonal;
    * ``blr``   -- a single hierarchy level: only blocks of leaf clusters are
      tested (standard condition), larger blocks are always subdivided.
    """
    if mode == "std":
        return admissible(a, b, eta)
    if mode == "hodlr":
        return a.id != b.id
    if mode == "blr":
        return (a.is_leaf or b.is_leaf) and admissible(a, b, eta)
    raise ValueError(mode)


def build_block_tree(ct: ClusterTree, eta: float, mode: str = "std") -> list:
    """Leaves of the block tree T_{IxI} (Def. Block Tree), depth-first order."""
    out: list = []
    cl = ct.clusters

    def rec(t: int, s: int) -> None:
        a, b = cl[t], cl[s]
        if block_admissible(a, b, eta, mode):
            out.append(Block(t, s, True))
        elif a.is_leaf or b.is_leaf:
            out.append(Block(t, s, False))
        else:
            for ts in a.sons:
                for ss in b.sons:
                    rec(ts, ss)

    rec(0, 0)
    return out
