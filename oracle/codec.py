"""Floating point codecs of Sec. 4.1 (AFLP, FPX) and the VALR widths of Sec. 4.2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Plain FP64 / integer definitions.  A code is an unsigned integer of 8*B bits
(B = bytes per value).  Readings of the paper where it is silent or ambiguous:

* Rounding is round-to-nearest, ties-to-even, for both codecs (Sec. 4.1 states
  round-to-nearest for FPX and is silent on ties and on AFLP).
* FPX (Fig. tab:fpx): the first table row (keys 0..10 -> e8m7) is taken for
  keys 0..8 only; keys 9 and 10 use e8m15.  Every other row satisfies
  m >= key - 1, i.e. the format's rounding error 2^-(m+1) is at most 2^-key,
  and the reading restores that rule for the first row.
* FPX e8 rows: the value is rounded once, from FP64, to m mantissa bits; if any
  value of the array then lies outside the FP32 normal range (or is an FP32
  subnormal), the whole array moves to the e11 row with the smallest m that is
  at least the requested one.  An array with a value that an e11 row rounds to
  infinity (beyond the FP64 maximum) moves to the exact row e11 m52.
* AFLP (Sec. 4.1, m_eps and e_dr formulas): s = fl(fl(|v|/vmin) + 1) >= 2 is
  rounded to m' mantissa bits; its binary exponent f >= 1 is stored in e bits,
  f = 0 is reserved for zero.  e is the bit length of the largest f (the data's
  dynamic range, as e_dr), at least 1; m' is the smallest value >= m with
  1 + m' + e a multiple of 8.  Layout: sign | f | mantissa, most significant
  first.  Decoding is v = +-fl(fl(s - 1) * vmin).  If 1 + m' + e > 56 (or
  m' > 52), or if s leaves the FP64 range (vmax/vmin + 1 overflows, or rounding
  carries s to 2^1024, where no f reproduces the value), the raw FP64 bits are
  stored (B = 8).  An all-zero array uses
  B = 1, e = 1, m' = 6, vmin = 1.  Parity unpinned: the paper does not print
  the AFLP bit layout, so only its stated properties are pinned.
"""
from __future__ import annotations

import math

import numpy as np

U64 = np.uint64
MASK52 = (1 << 52) - 1


# ----------------------------------------------------------------- helpers
def ceil_log2(r: float) -> int:
    """Exact ceil(log2 r) for finite r > 0 (via the binary exponent)."""
    if not (r > 0.0 and math.isfinite(r)):
        raise ValueError("ceil_log2 needs a positive finite value")
    mant, ex = math.frexp(r)          # r = mant * 2**ex, mant in [0.5, 1)
    return ex - 1 if mant == 0.5 else ex


def m_eps(eps: float) -> int:
    """m_eps = ceil(-log2 eps), the mantissa bits for accuracy eps (Sec. 4.1)."""
    return ceil_log2(1.0 / eps) if (1.0 / eps) != math.inf else 1075


def bitlen(x: int) -> int:
    """Number of bits needed to hold the non-negative integer x."""
    return int(x).bit_length()


def f64_bits(v: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(v, dtype=np.float64).view(U64)


def bits_f64(b: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(b, dtype=U64).view(np.float64)


def round_mag_bits(mag: np.ndarray, d: int) -> np.ndarray:
    """Round IEEE FP64 magnitude bit patterns to drop the low d bits (RNE).

    For a non-negative double the bit pattern is monotone in the value, so
    adding to the pattern carries from the mantissa into the exponent exactly
    as rounding the value does.
    """
    mag = np.asarray(mag, dtype=U64)
    if d == 0:
        return mag.copy()
    one = U64(1)
    half = U64(1 << (d - 1))
    low = mag & U64((1 << d) - 1)
    base = mag >> U64(d)
    up = (low > half) | ((low == half) & ((base & one) == one))
    return (base + up.astype(U64)) << U64(d)


# ----------------------------------------------------------------- FPX
# (key_lo, key_hi, e, m) rows of Fig. tab:fpx, first row read as keys 0..8.
FPX_TABLE = (
    (0, 8, 8, 7),
    (9, 15, 8, 15),
    (16, 23, 8, 23),
    (24, 28, 11, 28),
    (29, 36, 11, 36),
    (37, 44, 11, 44),
    (45, 52, 11, 52),
)


def fpx_format(key: int) -> tuple[int, int]:
    """(e, m) of the FPX format for key = ceil(-log2 accuracy), clamped to 0..52."""
    key = min(max(int(key), 0), 52)
    for lo, hi, e, m in FPX_TABLE:
        if lo <= key <= hi:
            return e, m
    raise AssertionError("unreachable")


def fpx_bytes(e: int, m: int) -> int:
    assert (1 + e + m) % 8 == 0
    return (1 + e + m) // 8


def fpx_encode(v: np.ndarray, e: int, m: int):
    """FPX codes of v in format (e, m), or None if a value is out of the format's
    range (e8: outside the FP32 normal range; e11: rounded to infinity)."""
    v = np.asarray(v, dtype=np.float64)
    if not np.all(np.isfinite(v)):
        raise ValueError("FPX needs finite values")
    nb = fpx_bytes(e, m)
    bits = f64_bits(v)
    sign = bits >> U64(63)
    mag = round_mag_bits(bits & U64(0x7FFFFFFFFFFFFFFF), 52 - m)
    if e == 11:
        if np.any((mag >> U64(52)) == U64(2047)):     # rounded past the FP64 maximum
            return None
        full = (sign << U64(63)) | mag
        return full >> U64(64 - 8 * nb)
    assert e == 8
    ex = (mag >> U64(52)).astype(np.int64) - 1023
    nz = mag != 0
    if np.any(nz & ((ex < -126) | (ex > 127))):
        return None
    exb = np.where(nz, ex + 127, 0).astype(U64)
    f32 = (exb << U64(23)) | ((mag & U64(MASK52)) >> U64(29))
    f32 = np.where(nz, f32, U64(0)) | (sign << U64(31))
    return f32 >> U64(32 - 8 * nb)


def fpx_decode(codes: np.ndarray, e: int, m: int) -> np.ndarray:
    """FP64 values of FPX codes (exact: every code is a double)."""
    nb = fpx_bytes(e, m)
    codes = np.asarray(codes, dtype=U64)
    if e == 11:
        return bits_f64(codes << U64(64 - 8 * nb))
    w = (codes << U64(32 - 8 * nb)).astype(np.uint32)
    return w.view(np.float32).astype(np.float64)


def fpx_compress(v: np.ndarray, key: int) -> dict:
    """Direct FPX compression of an array for accuracy key (table + promotion)."""
    e, m = fpx_format(key)
    codes = fpx_encode(v, e, m)
    if codes is None and e == 8:           # e8 out of range: smallest e11 row (m = 28 > 23)
        e, m = 11, 28
        codes = fpx_encode(v, e, m)
    if codes is None:                      # rounded past the FP64 maximum: the exact row
        e, m = 11, 52
        codes = fpx_encode(v, e, m)
    return {"codec": "fpx", "B": fpx_bytes(e, m), "e": e, "m": m, "codes": codes}


# ----------------------------------------------------------------- AFLP
def _aflp_mprime(m: int, e: int) -> int:
    mp = m
    while (1 + mp + e) % 8 != 0:
        mp += 1
    return mp


def aflp_compress(v: np.ndarray, m: int) -> dict:
    """AFLP compression of an array with m requested mantissa bits (Sec. 4.1)."""
    v = np.asarray(v, dtype=np.float64)
    if not np.all(np.isfinite(v)):
        raise ValueError("AFLP needs finite values")
    m = max(int(m), 1)
    bits = f64_bits(v)
    sign = bits >> U64(63)
    a = np.abs(v)
    nz = a > 0
    if not np.any(nz):
        return {"codec": "aflp", "B": 1, "e": 1, "mp": 6, "vmin": 1.0, "raw": False,
                "codes": sign << U64(7)}
    vmin = float(a[nz].min())
    vmax = float(a[nz].max())
    raw = {"codec": "aflp", "B": 8, "e": 0, "mp": 52, "vmin": vmin, "raw": True, "codes": bits.copy()}
    smax = (vmax / vmin) + 1.0
    if not np.isfinite(smax):                          # s beyond FP64: no exponent f reproduces v
        return raw
    s = np.where(nz, (a / vmin) + 1.0, 2.0)            # two FP64 RN operations
    f0 = (int(f64_bits(np.array([smax]))[0]) >> 52) - 1023
    e = max(1, bitlen(f0))
    for _ in range(2):
        mp = _aflp_mprime(m, e)
        if 1 + mp + e > 56 or mp > 52:
            return raw
        sr = round_mag_bits(f64_bits(s), 52 - mp)
        f = ((sr >> U64(52)).astype(np.int64) - 1023)
        fmax = int(f[nz].max())
        if fmax > 1023:                                # rounding carried s to 2^1024
            return raw
        if bitlen(fmax) <= e:
            break
        e = bitlen(fmax)
    else:
        raise AssertionError("AFLP exponent did not settle")
    nb = (1 + mp + e) // 8
    mant = (sr & U64(MASK52)) >> U64(52 - mp)
    code = (sign << U64(8 * nb - 1)) | (f.astype(U64) << U64(mp)) | mant
    code = np.where(nz, code, sign << U64(8 * nb - 1))
    return {"codec": "aflp", "B": nb, "e": e, "mp": mp, "vmin": vmin, "raw": False,
            "codes": code.astype(U64)}


def aflp_decode(codes: np.ndarray, B: int, e: int, mp: int, vmin: float, raw: bool) -> np.ndarray:
    """FP64 values of AFLP codes: v = +-fl(fl(s - 1) * vmin), f = 0 -> +-0."""
    codes = np.asarray(codes, dtype=U64)
    if raw:
        return bits_f64(codes)
    sign = (codes >> U64(8 * B - 1)) & U64(1)
    f = (codes >> U64(mp)) & U64((1 << e) - 1)
    mant = codes & U64((1 << mp) - 1)
    sbits = ((f + U64(1023)) << U64(52)) | (mant << U64(52 - mp))
    s = bits_f64(sbits)
    val = (s - 1.0) * vmin
    val = np.where(f == 0, 0.0, val)
    return np.where(sign == 1, -val, val)


# ----------------------------------------------------------------- generic
def compress(v: np.ndarray, codec: str, key: int) -> dict:
    """Compress an array to accuracy 2^-key with the named codec.

    For AFLP the requested mantissa is m = key (relative error 2^-m', m' >= m);
    for FPX the table row of the key is used (relative error 2^-(m+1)).
    ``codec == "none"`` stores raw FP64 (B = 8).
    """
    if codec == "aflp":
        return aflp_compress(v, key)
    if codec == "fpx":
        return fpx_compress(v, key)
    if codec == "none":
        return {"codec": "none", "B": 8, "codes": f64_bits(v).copy()}
    raise ValueError(codec)


def decompress(c: dict) -> np.ndarray:
    if c["codec"] == "aflp":
        return aflp_decode(c["codes"], c["B"], c["e"], c["mp"], c["vmin"], c["raw"])
    if c["codec"] == "fpx":
        return fpx_decode(c["codes"], c["e"], c["m"])
    if c["codec"] == "none":
        return bits_f64(c["codes"])
    raise ValueError(c["codec"])


def unit_error(c: dict) -> float:
    """Per-value relative error bound of a compressed array's format."""
    if c["codec"] == "aflp":
        return 0.0 if c["raw"] else 2.0 ** (-c["mp"])
    if c["codec"] == "fpx":
        return 2.0 ** (-(c["m"] + 1))
    return 0.0


# ----------------------------------------------------------------- VALR
def valr_key(sigma_i: float, delta: float) -> int:
    """Accuracy key of column i: ceil(-log2 delta_i) with delta_i = delta / sigma_i.

    Sec. 4.2 stores column i at accuracy delta_i; the key is ceil(log2(sigma_i /
    delta)), clamped to 1..52 (a column whose sigma_i <= delta keeps one bit).
    """
    r = sigma_i / delta
    if r <= 1.0:
        return 1
    return min(max(ceil_log2(r), 1), 52)
