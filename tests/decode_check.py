"""Shared helpers of the decoder checks: the oracle's value of every packed code.

Test code only.  A code's format word is B | fmt << 4 | e << 6 | m << 10 (fmt 0
FPX e8, 1 FPX e11, 2 AFLP, 3 raw FP64), as ``hm_decompress_debug`` reports it.
"""
import numpy as np

from oracle import codec as ocd


def fields(fmt):
    fmt = fmt.astype(np.int64)
    return fmt & 15, (fmt >> 4) & 3, (fmt >> 6) & 15, fmt >> 10


def oracle_values(code, fmt):
    """The oracle's FP64 value of every code (AFLP: vmin = 1, i.e. +-fl(s - 1))."""
    B, F, E, Mb = fields(fmt)
    out = np.empty(code.size)
    keys = np.stack([B, F, E, Mb], axis=1)
    for b, f, e, m in np.unique(keys, axis=0):
        sel = (B == b) & (F == f) & (E == e) & (Mb == m)
        c = code[sel]
        if f == 0:
            out[sel] = ocd.fpx_decode(c, 8, 8 * int(b) - 9)
        elif f == 1:
            out[sel] = ocd.fpx_decode(c, 11, 8 * int(b) - 12)
        elif f == 2:
            out[sel] = ocd.aflp_decode(c, int(b), int(e), int(m), 1.0, False)
        else:
            out[sel] = ocd.bits_f64(c)
    return out


def aflp_f(code, fmt):
    B, F, E, Mb = fields(fmt)
    f = np.zeros(code.size, dtype=np.int64)
    a = F == 2
    f[a] = ((code[a] >> Mb[a].astype(np.uint64)) & ((np.uint64(1) << E[a].astype(np.uint64)) - np.uint64(1))
            ).astype(np.int64)
    return f
