"""The oracle's Alg. 1 product timed on a bounded sample of a large workload.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``); used by the CPU
baseline of the benchmark.  The oracle cannot build the largest blocks of an
N = 131072 H-matrix by exact SVD in reasonable time, so the sample is a random
subset of the workload's leaf blocks with at most 2^20 entries each, drawn
until their expected FP64 storage (dense: m*n*8, low-rank: (m+n)*10*8) reaches
a byte budget.  The oracle builds those blocks
itself (exact truncated SVD, eqn. epsilon), compresses them (Sec. 4.1 / 4.2)
and the timed part is Alg. 1 over the sampled blocks, each decompressed as in
Alg. 8 and applied in FP64.  Throughput is reported per algorithmic byte:
packed values plus 8 bytes per x entry and 16 per y entry of every block.
"""
from __future__ import annotations

import time

import numpy as np

import synth

from . import compress, kernels, matvec
from .hmatrix import HMatrix, LowRank, truncate_rank
from .trees import build_block_tree, build_cluster_tree


def sample_h(n: int, eps: float, codec: str, budget_bytes: float, seed: int = 3,
             leaf: int = 64, eta: float = 2.0, part: tuple[int, int] = (0, 1), kind: str = "laplace"):
    """Oracle-built compressed H-matrix restricted to a random block sample.

    kind: "laplace" (sphere points) or "matern" (unit-cube points).
    part = (p, P): only every P-th block of the sample, starting at the p-th
    (in block-tree order), so that P processes each build and time a disjoint
    share of the same sample."""
    pts = synth.sphere_points(n) if kind == "laplace" else synth.cube_points(n)
    param = kernels.default_param(kind, n)
    ct = build_cluster_tree(pts, leaf)
    blocks = build_block_tree(ct, eta)
    cl = ct.clusters
    sizes = np.array([cl[b.row].size * cl[b.col].size for b in blocks])
    stored = np.array([(cl[b.row].size + cl[b.col].size) * 80.0 if b.adm else
                       cl[b.row].size * cl[b.col].size * 8.0 for b in blocks])
    elig = np.flatnonzero(sizes <= (1 << 20))
    rng = np.random.default_rng(seed)
    order = rng.permutation(elig)
    chosen, tot = [], 0.0
    for i in order:
        chosen.append(int(i))
        tot += stored[i]
        if tot >= budget_bytes:
            break
    chosen.sort()
    chosen = chosen[part[0]::part[1]]
    sub = [blocks[i] for i in chosen]
    data = []
    for b in sub:
        r = ct.perm[cl[b.row].start:cl[b.row].end]
        c = ct.perm[cl[b.col].start:cl[b.col].end]
        a = kernels.entries(kind, pts, r, c, param)
        if not b.adm:
            data.append(a)
            continue
        u, s, vt = np.linalg.svd(a, full_matrices=False)
        k = truncate_rank(s, eps)
        data.append(LowRank(np.asfortranarray(u[:, :k]), s[:k].copy(), np.asfortranarray(vt[:k].T)))
    h = HMatrix(kind, param, eps, ct, sub, data, pts)
    ch = compress.compress_h(h, codec)
    return h, ch, len(blocks)


def alg_bytes(ch) -> int:
    """Packed value bytes + 8 per x entry + 16 per y entry of every sampled block."""
    cl = ch.h.ct.clusters
    tot = compress.payload_bytes(ch)
    for b in ch.h.blocks:
        tot += 8 * cl[b.col].size + 16 * cl[b.row].size
    return tot


def run_pass(ch, xp, yp) -> None:
    for i in range(len(ch.h.blocks)):
        matvec.h_block_apply(ch, i, 1.0, xp, yp)


def time_passes(ch, steps: int, warmup: int, x=None):
    """Per-pass seconds of Alg. 1 over the sample (x in cluster order)."""
    n = ch.h.n
    xp = synth.rhs(n)[:, 0][ch.h.ct.perm] if x is None else x
    yp = np.zeros(n)
    for _ in range(warmup):
        run_pass(ch, xp, yp)
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        run_pass(ch, xp, yp)
        ts.append(time.perf_counter() - t0)
    return np.array(ts)
