"""Matrix-vector products y := alpha*M*x + beta*y (eqn. mvm, Sec. 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sequential FP64 versions of the paper's algorithms, one block at a time:

* ``h_mvm``   -- Alg. 1 (loop over leaf blocks; low-rank t := V^H x, y|t += alpha U t).
* ``uh_mvm``  -- Alg. 4 (forward s_s := X_s^H x|s for every cluster), then
                 Alg. 5 root to leaves (t_t := sum S_ts s_s, eq. sumcoup;
                 y' := W_t t_t; y' += D x for dense blocks; y|t += y').
* ``h2_mvm``  -- Alg. 6 (leaf forward, then s_s += E_s'^H s_s' leaves to root),
                 then Alg. 7 root to leaves (couplings, t_t' += E_t' t_t at inner
                 clusters, y' := W_t t_t at leaves, dense blocks, y|t += y').
* ``*_adjoint`` -- y := alpha M^H x + beta y (the remark after Alg. 3: the same
                 steps over the block columns).

Compressed matrices are decompressed block by block before the product
(Alg. 8 computes the same sum, entry by entry).  beta extends the paper's
update y := alpha M x + y; beta = 1 is the paper's operation.  x and y are in
the original point order, shape (N,) or (N, r); the products run in the
cluster order and are permuted back.
"""
from __future__ import annotations

import numpy as np

from .compress import CH, CH2, CUH, undirect, unvalr
from .hmatrix import HMatrix, LowRank
from .nested import H2, Uniform


def _perm_in(ct, x, y, beta):
    xp = np.asarray(x, dtype=np.float64)[ct.perm]
    yp = beta * np.asarray(y, dtype=np.float64)[ct.perm]
    return xp, yp


def _perm_out(ct, yp):
    y = np.empty_like(yp)
    y[ct.perm] = yp
    return y


def h_mvm(m, alpha: float, x, beta: float = 1.0, y=None):
    """Alg. 1 on an HMatrix (FP64) or a CH (compressed, decoded per block)."""
    h = m if isinstance(m, HMatrix) else m.h
    ct = h.ct
    if y is None:
        y = np.zeros_like(np.asarray(x, dtype=np.float64))
    xp, yp = _perm_in(ct, x, y, beta)
    for i in range(len(h.blocks)):
        h_block_apply(m, i, alpha, xp, yp)
    return _perm_out(ct, yp)


def h_block_apply(m, i: int, alpha: float, xp, yp) -> None:
    """One step of Alg. 1: leaf block i of an HMatrix or CH, y|t += alpha M_ts x|s.

    Low-rank: t := V^H x|s with V = X diag(sigma), y|t += alpha W t; dense:
    y|t += alpha D x|s.  Compressed data are decompressed first (Alg. 8).
    """
    h = m if isinstance(m, HMatrix) else m.h
    cl = h.ct.clusters
    b = h.blocks[i]
    t, s = cl[b.row], cl[b.col]
    xs = xp[s.start:s.end]
    if isinstance(m, HMatrix):
        d = m.data[i]
        if isinstance(d, LowRank):
            tv = (d.X.T @ xs)
            tv = (d.s * tv.T).T
            yp[t.start:t.end] += alpha * (d.W @ tv)
        else:
            yp[t.start:t.end] += alpha * (d @ xs)
        return
    blk = m.blocks[i]
    if blk[0] == "lr":
        sv, wc, xc = blk[1], blk[2], blk[3]
        W = unvalr(wc, t.size)
        X = unvalr(xc, s.size)
        tv = (X.T @ xs)
        tv = (sv * tv.T).T
        yp[t.start:t.end] += alpha * (W @ tv)
    else:
        yp[t.start:t.end] += alpha * (undirect(blk[1]) @ xs)


def uh_mvm(m, alpha: float, x, beta: float = 1.0, y=None):
    """Alg. 4 + Alg. 5 on a Uniform (FP64) or CUH (compressed) matrix."""
    u = m if isinstance(m, Uniform) else m.u
    h = u.h
    ct = h.ct
    cl = ct.clusters
    if y is None:
        y = np.zeros_like(np.asarray(x, dtype=np.float64))
    xp, yp = _perm_in(ct, x, y, beta)
    comp = not isinstance(m, Uniform)
    Wb = [unvalr(m.W[c.id], c.size) for c in cl] if comp else u.W
    Xb = [unvalr(m.X[c.id], c.size) for c in cl] if comp else u.X
    # Alg. 4: forward transformation, every cluster independently
    s = [Xb[c.id].T @ xp[c.start:c.end] for c in cl]
    rows = [[] for _ in cl]
    for i, b in enumerate(h.blocks):
        rows[b.row].append(i)

    def coupling(i):
        return undirect(m.S[i][1]) if comp else u.S[i]

    def uni(tid: int) -> None:                      # Alg. 5
        t = cl[tid]
        shp = (Wb[tid].shape[1],) + xp.shape[1:]
        tt = np.zeros(shp)
        for i in rows[tid]:
            b = h.blocks[i]
            if b.adm:
                tt += coupling(i) @ s[b.col]
        yl = Wb[tid] @ tt
        for i in rows[tid]:
            b = h.blocks[i]
            if not b.adm:
                sc = cl[b.col]
                yl = yl + coupling(i) @ xp[sc.start:sc.end]
        yp[t.start:t.end] += alpha * yl
        for son in t.sons:
            uni(son)

    uni(0)
    return _perm_out(ct, yp)


def h2_mvm(m, alpha: float, x, beta: float = 1.0, y=None):
    """Alg. 6 + Alg. 7 on an H2 (FP64) or CH2 (compressed) matrix."""
    h2 = m if isinstance(m, H2) else m.m
    h = h2.h
    ct = h.ct
    cl = ct.clusters
    comp = not isinstance(m, H2)
    if y is None:
        y = np.zeros_like(np.asarray(x, dtype=np.float64))
    xp, yp = _perm_in(ct, x, y, beta)
    tail = xp.shape[1:]

    def leafW(cid):
        return unvalr(m.Wleaf[cid], cl[cid].size) if comp else h2.Wleaf[cid]

    def leafX(cid):
        return unvalr(m.Xleaf[cid], cl[cid].size) if comp else h2.Xleaf[cid]

    def EW(cid):
        return undirect(m.EW[cid]) if comp else h2.EW[cid]

    def EX(cid):
        return undirect(m.EX[cid]) if comp else h2.EX[cid]

    def coupling(i):
        return undirect(m.S[i][1]) if comp else h2.S[i]

    s = [None] * len(cl)

    def forward(sid: int) -> None:                  # Alg. 6
        c = cl[sid]
        if c.is_leaf:
            s[sid] = leafX(sid).T @ xp[c.start:c.end]
            return
        s[sid] = np.zeros((h2.kX[sid],) + tail)
        for son in c.sons:
            forward(son)
            s[sid] += EX(son).T @ s[son]

    forward(0)
    rows = [[] for _ in cl]
    for i, b in enumerate(h.blocks):
        rows[b.row].append(i)
    t = [np.zeros((h2.kW[c.id],) + tail) for c in cl]

    def h2mvm(tid: int) -> None:                     # Alg. 7
        c = cl[tid]
        for i in rows[tid]:
            b = h.blocks[i]
            if b.adm:
                t[tid] += coupling(i) @ s[b.col]
        if c.is_leaf:
            yl = leafW(tid) @ t[tid]
        else:
            yl = np.zeros((c.size,) + tail)
            for son in c.sons:
                t[son] += EW(son) @ t[tid]
        for i in rows[tid]:
            b = h.blocks[i]
            if not b.adm:
                sc = cl[b.col]
                yl = yl + coupling(i) @ xp[sc.start:sc.end]
        yp[c.start:c.end] += alpha * yl
        for son in c.sons:
            h2mvm(son)

    h2mvm(0)
    return _perm_out(ct, yp)


def uhsep_mvm(m, alpha: float, x, beta: float = 1.0, y=None, adjoint: bool = False):
    """UH product with separate row and column couplings (the variant discussed
    after Alg. 5): forward s_s := X_s^H x|s (Alg. 4); per low-rank block the
    first stage u_b := Sc_b^H s_s; per row cluster t_t := sum_b Sr_b u_b and
    y|t += alpha (W_t t_t + sum of the dense blocks D x).  adjoint: the same with
    the roles of rows and columns exchanged (M^H x)."""
    from .nested import UniformSep
    comp = not isinstance(m, UniformSep)
    ms = m.m if comp else m
    u = ms.u
    h = u.h
    ct = h.ct
    cl = ct.clusters
    if y is None:
        y = np.zeros_like(np.asarray(x, dtype=np.float64))
    xp, yp = _perm_in(ct, x, y, beta)
    Wb = [unvalr(m.W[c.id], c.size) for c in cl] if comp else u.W
    Xb = [unvalr(m.X[c.id], c.size) for c in cl] if comp else u.X
    if adjoint:
        Wb, Xb = Xb, Wb
    s = [Xb[c.id].T @ xp[c.start:c.end] for c in cl]
    t = [np.zeros((Wb[c.id].shape[1],) + xp.shape[1:]) for c in cl]
    dense = [[] for _ in cl]
    for i, b in enumerate(h.blocks):
        row, col = (b.col, b.row) if adjoint else (b.row, b.col)
        if b.adm:
            sr = undirect(m.Sr[i]) if comp else ms.Sr[i]
            sc = undirect(m.Sc[i]) if comp else ms.Sc[i]
            if adjoint:
                sr, sc = sc, sr
            ub = sc.T @ s[col]
            t[row] += sr @ ub
        else:
            d = undirect(m.Sr[i]) if comp else u.S[i]
            dense[row].append((col, d.T if adjoint else d))
    for c in cl:
        yl = Wb[c.id] @ t[c.id]
        for col, d in dense[c.id]:
            sc = cl[col]
            yl = yl + d @ xp[sc.start:sc.end]
        yp[c.start:c.end] += alpha * yl
    return _perm_out(ct, yp)


# ---------------------------------------------------------------- adjoint products
# The remark after Alg. 3: the adjoint product M^H x runs the same way over the
# block columns.  The data are real, so M^H = M^T: a low-rank block
# W diag(sigma) X^T contributes y|s += alpha X diag(sigma) (W^T x|t), a dense
# block y|s += alpha D^T x|t; for UH / H2 the roles of the row and column
# bases swap and every coupling is applied transposed.

def h_mvm_adjoint(m, alpha: float, x, beta: float = 1.0, y=None):
    """y := alpha M^H x + beta y, block by block over an HMatrix or CH."""
    h = m if isinstance(m, HMatrix) else m.h
    ct = h.ct
    cl = ct.clusters
    if y is None:
        y = np.zeros_like(np.asarray(x, dtype=np.float64))
    xp, yp = _perm_in(ct, x, y, beta)
    for i, b in enumerate(h.blocks):
        t, s = cl[b.row], cl[b.col]
        xt = xp[t.start:t.end]
        if isinstance(m, HMatrix):
            d = m.data[i]
            if isinstance(d, LowRank):
                tv = (d.s * (d.W.T @ xt).T).T
                yp[s.start:s.end] += alpha * (d.X @ tv)
            else:
                yp[s.start:s.end] += alpha * (d.T @ xt)
            continue
        blk = m.blocks[i]
        if blk[0] == "lr":
            sv = blk[1]
            W = unvalr(blk[2], t.size)
            X = unvalr(blk[3], s.size)
            tv = (sv * (W.T @ xt).T).T
            yp[s.start:s.end] += alpha * (X @ tv)
        else:
            yp[s.start:s.end] += alpha * (undirect(blk[1]).T @ xt)
    return _perm_out(ct, yp)


def uh_mvm_adjoint(m, alpha: float, x, beta: float = 1.0, y=None):
    """Adjoint of Alg. 4 + 5: forward with the row bases, S^T per block column,
    backward with the column bases, dense blocks transposed."""
    u = m if isinstance(m, Uniform) else m.u
    h = u.h
    ct = h.ct
    cl = ct.clusters
    if y is None:
        y = np.zeros_like(np.asarray(x, dtype=np.float64))
    xp, yp = _perm_in(ct, x, y, beta)
    comp = not isinstance(m, Uniform)
    Wb = [unvalr(m.W[c.id], c.size) for c in cl] if comp else u.W
    Xb = [unvalr(m.X[c.id], c.size) for c in cl] if comp else u.X
    sw = [Wb[c.id].T @ xp[c.start:c.end] for c in cl]     # forward with the row bases
    cols = [[] for _ in cl]
    for i, b in enumerate(h.blocks):
        cols[b.col].append(i)

    def coupling(i):
        return undirect(m.S[i][1]) if comp else u.S[i]

    for c in cl:                                          # block column c
        tt = np.zeros((Xb[c.id].shape[1],) + xp.shape[1:])
        yl = np.zeros((c.size,) + xp.shape[1:])
        for i in cols[c.id]:
            b = h.blocks[i]
            if b.adm:
                tt += coupling(i).T @ sw[b.row]
            else:
                rt = cl[b.row]
                yl += coupling(i).T @ xp[rt.start:rt.end]
        yp[c.start:c.end] += alpha * (Xb[c.id] @ tt + yl)
    return _perm_out(ct, yp)


def h2_mvm_adjoint(m, alpha: float, x, beta: float = 1.0, y=None):
    """Adjoint of Alg. 6 + 7: up-sweep with the row bases (leaf W, transfers
    E_W), S^T per block column, down-sweep with the column transfers E_X,
    leaf column bases X, dense blocks transposed."""
    h2 = m if isinstance(m, H2) else m.m
    h = h2.h
    ct = h.ct
    cl = ct.clusters
    comp = not isinstance(m, H2)
    if y is None:
        y = np.zeros_like(np.asarray(x, dtype=np.float64))
    xp, yp = _perm_in(ct, x, y, beta)
    tail = xp.shape[1:]

    def leafW(cid):
        return unvalr(m.Wleaf[cid], cl[cid].size) if comp else h2.Wleaf[cid]

    def leafX(cid):
        return unvalr(m.Xleaf[cid], cl[cid].size) if comp else h2.Xleaf[cid]

    def EW(cid):
        return undirect(m.EW[cid]) if comp else h2.EW[cid]

    def EX(cid):
        return undirect(m.EX[cid]) if comp else h2.EX[cid]

    def coupling(i):
        return undirect(m.S[i][1]) if comp else h2.S[i]

    s = [None] * len(cl)

    def up(tid: int) -> None:                         # row side, leaves to root
        c = cl[tid]
        if c.is_leaf:
            s[tid] = leafW(tid).T @ xp[c.start:c.end]
            return
        s[tid] = np.zeros((h2.kW[tid],) + tail)
        for son in c.sons:
            up(son)
            s[tid] += EW(son).T @ s[son]

    up(0)
    cols = [[] for _ in cl]
    for i, b in enumerate(h.blocks):
        cols[b.col].append(i)
    t = [np.zeros((h2.kX[c.id],) + tail) for c in cl]

    def down(sid: int) -> None:                       # column side, root to leaves
        c = cl[sid]
        for i in cols[sid]:
            b = h.blocks[i]
            if b.adm:
                t[sid] += coupling(i).T @ s[b.row]
        if c.is_leaf:
            yl = leafX(sid) @ t[sid]
        else:
            yl = np.zeros((c.size,) + tail)
            for son in c.sons:
                t[son] += EX(son) @ t[sid]
        for i in cols[sid]:
            b = h.blocks[i]
            if not b.adm:
                rt = cl[b.row]
                yl = yl + coupling(i).T @ xp[rt.start:rt.end]
        yp[c.start:c.end] += alpha * yl
        for son in c.sons:
            down(son)

    down(0)
    return _perm_out(ct, yp)


def dense_mvm(a: np.ndarray, alpha: float, x, beta: float = 1.0, y=None):
    """y := alpha A x + beta y with a dense FP64 matrix (the plain definition)."""
    x = np.asarray(x, dtype=np.float64)
    if y is None:
        y = np.zeros_like(x)
    return alpha * (a @ x) + beta * np.asarray(y, dtype=np.float64)
