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


def f32_tier_head(code, fmt, v):
    """What the FP32-tier decoders give for each code: the oracle's value v
    rounded to nearest FP32 where the code fits 24 significant bits (FPX e8,
    AFLP up to 3 bytes), and for wider codes the stated approximation -- AFLP:
    fl32(s_h - 1) with s_h = s cut to 23 mantissa bits; FPX e11 and raw FP64:
    the top 24 significant bits (0 below 2^-126)."""
    B, F, E, Mb = fields(fmt)
    out = v.astype(np.float32)
    wide_aflp = (F == 2) & (B >= 4)
    if np.any(wide_aflp):
        c = code[wide_aflp]
        mb = Mb[wide_aflp].astype(np.uint64)
        eb = E[wide_aflp].astype(np.uint64)
        sign = (c >> (np.uint64(8) * B[wide_aflp].astype(np.uint64) - np.uint64(1))) & np.uint64(1)
        f = (c >> mb) & ((np.uint64(1) << eb) - np.uint64(1))
        mant = c & ((np.uint64(1) << mb) - np.uint64(1))
        sh = (((f + np.uint64(127)) << np.uint64(23)) | (mant >> (mb - np.uint64(23)))).astype(np.uint32)
        d = sh.view(np.float32) - np.float32(1.0)
        d = np.where(f == 0, np.float32(0.0), d).astype(np.float32)
        out[wide_aflp] = np.where(sign == 1, -d, d)
    wide64 = (F == 1) | (F == 3)
    if np.any(wide64):
        bits = ocd.f64_bits(v[wide64])
        ex = ((bits >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
        hb = (((ex - 896).clip(0).astype(np.uint64) << np.uint64(23)) |
              ((bits & np.uint64((1 << 52) - 1)) >> np.uint64(29))).astype(np.uint64)
        hb = np.where(ex >= 897, hb, np.uint64(0)) | ((bits >> np.uint64(32)) & np.uint64(0x80000000))
        out[wide64] = hb.astype(np.uint32).view(np.float32)
    return out
