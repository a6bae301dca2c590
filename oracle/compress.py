"""Direct and VALR compression of built H / UH / H^2 matrices (Sec. 4.1, 4.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Direct compression (Sec. 4.1) at key m_eps = ceil(-log2 eps): dense leaves,
  UH / H^2 coupling matrices and H^2 transfer matrices; one codec header per
  matrix (all its entries form one array).
* VALR for low-rank blocks (Sec. 4.2, eqn. valr): column i of W and of X is
  stored at accuracy delta_i = delta / sigma_i.  Reading of the garbled
  "delta = eps/||M||_F": the relative error delta = eps * ||M_ts||_F, divided by
  the factor (1 + 2k) of eqn. valr ("used to adjust local error bounds"), i.e.
  delta = eps * ||sigma||_2 / (1 + 2k).
* VALR for cluster bases (Sec. 4.2, eqn. valrcb): column i at delta_i =
  delta / Sigma_i with delta = tau / k (the factor k of eqn. valrcb
  compensated), tau the truncation threshold the basis was built with
  (eps for UH, eps / sqrt(depth + 1) for H^2).  UH compresses every basis, H^2
  only its leaf bases (Sec. 4.2).
* ``codec == "none"`` keeps FP64 (the uncompressed reference product).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import codec as cd
from .hmatrix import HMatrix, LowRank
from .nested import H2, Uniform


def direct(a: np.ndarray, codec: str, eps: float) -> dict:
    """Direct compression of a whole matrix (column-major entry order)."""
    c = cd.compress(np.asfortranarray(a).ravel(order="F"), codec, cd.m_eps(eps))
    c["shape"] = a.shape
    return c


def undirect(c: dict) -> np.ndarray:
    return cd.decompress(c).reshape(c["shape"], order="F")


def valr_columns(f: np.ndarray, keys: list, codec: str) -> list:
    """Compress column i of f at key keys[i] (VALR)."""
    return [cd.compress(f[:, i], codec, keys[i]) for i in range(f.shape[1])]


def unvalr(cols: list, n: int) -> np.ndarray:
    if not cols:
        return np.zeros((n, 0))
    return np.stack([cd.decompress(c) for c in cols], axis=1)


def lowrank_keys(s: np.ndarray, eps: float) -> list:
    """VALR keys of a low-rank block: delta = eps ||s||_2 / (1 + 2k)."""
    k = s.shape[0]
    if k == 0:
        return []
    delta = eps * float(np.linalg.norm(s)) / (1.0 + 2.0 * k)
    return [cd.valr_key(float(si), delta) for si in s]


def basis_keys(sig: np.ndarray, tau: float) -> list:
    """VALR keys of a cluster basis: delta = tau / k (eqn. valrcb)."""
    k = sig.shape[0]
    if k == 0:
        return []
    delta = tau / k
    return [cd.valr_key(float(si), delta) for si in sig]


@dataclass
class CH:
    h: HMatrix
    codec: str
    blocks: list       # per block: ("dense", comp) or ("lr", s, Wcols, Xcols)


def compress_h(h: HMatrix, codec: str) -> CH:
    out = []
    for d in h.data:
        if isinstance(d, LowRank):
            if codec == "none":
                keys = [52] * d.rank
            else:
                keys = lowrank_keys(d.s, h.eps)
            out.append(("lr", d.s.copy(), valr_columns(d.W, keys, codec),
                        valr_columns(d.X, keys, codec)))
        else:
            out.append(("dense", direct(d, codec, h.eps)))
    return CH(h, codec, out)


@dataclass
class CUH:
    u: Uniform
    codec: str
    W: list
    X: list
    S: list            # per block: ("dense", comp) or ("lr", comp)


def compress_uh(u: Uniform, codec: str) -> CUH:
    eps = u.h.eps
    W, X, S = [], [], []
    for i in range(len(u.W)):
        kw = [52] * u.W[i].shape[1] if codec == "none" else basis_keys(u.SW[i], eps)
        kx = [52] * u.X[i].shape[1] if codec == "none" else basis_keys(u.SX[i], eps)
        W.append(valr_columns(u.W[i], kw, codec))
        X.append(valr_columns(u.X[i], kx, codec))
    for b, s in zip(u.h.blocks, u.S):
        S.append(("lr" if b.adm else "dense", direct(s, codec, eps)))
    return CUH(u, codec, W, X, S)


@dataclass
class CUHSep:
    m: object          # nested.UniformSep
    codec: str
    W: list
    X: list
    Sr: list           # per block: direct(Sr) for low-rank, direct(D) for dense
    Sc: list           # per block: direct(Sc) for low-rank, None for dense


def compress_uh_sep(m, codec: str) -> CUHSep:
    """Bases as compress_uh (VALR), both coupling factors direct at eps."""
    cu = compress_uh(m.u, codec)
    eps = m.u.h.eps
    Sr, Sc = [], []
    for b, r, c, s in zip(m.u.h.blocks, m.Sr, m.Sc, m.u.S):
        if b.adm:
            Sr.append(direct(r, codec, eps))
            Sc.append(direct(c, codec, eps))
        else:
            Sr.append(direct(s, codec, eps))
            Sc.append(None)
    return CUHSep(m, codec, cu.W, cu.X, Sr, Sc)


@dataclass
class CH2:
    m: H2
    codec: str
    Wleaf: dict
    Xleaf: dict
    EW: dict
    EX: dict
    S: list


def compress_h2(m: H2, codec: str) -> CH2:
    eps = m.h.eps
    tau = eps / np.sqrt(m.h.ct.depth() + 1.0)

    def leaves(bases, sig):
        out = {}
        for cid, w in bases.items():
            keys = [52] * w.shape[1] if codec == "none" else basis_keys(sig[cid], tau)
            out[cid] = valr_columns(w, keys, codec)
        return out

    EW = {cid: direct(e, codec, eps) for cid, e in m.EW.items()}
    EX = {cid: direct(e, codec, eps) for cid, e in m.EX.items()}
    S = [("lr" if b.adm else "dense", direct(s, codec, eps)) for b, s in zip(m.h.blocks, m.S)]
    return CH2(m, codec, leaves(m.Wleaf, m.SWleaf), leaves(m.Xleaf, m.SXleaf), EW, EX, S)


def payload_bytes(obj) -> int:
    """Bytes of the packed values (codes only) of a compressed matrix."""
    tot = 0

    def add(c):
        nonlocal tot
        tot += c["B"] * c["codes"].shape[0]

    if isinstance(obj, CH):
        for blk in obj.blocks:
            if blk[0] == "dense":
                add(blk[1])
            else:
                for c in blk[2] + blk[3]:
                    add(c)
    elif isinstance(obj, CUH):
        for cols in obj.W + obj.X:
            for c in cols:
                add(c)
        for _, c in obj.S:
            add(c)
    elif isinstance(obj, CH2):
        for d in (obj.Wleaf, obj.Xleaf):
            for cols in d.values():
                for c in cols:
                    add(c)
        for d in (obj.EW, obj.EX):
            for c in d.values():
                add(c)
        for _, c in obj.S:
            add(c)
    return tot
