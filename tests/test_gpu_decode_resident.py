"""Bit-exact decompression of the RESIDENT payload by the product kernels' own decoders.

``hm_decompress_debug`` runs, over the packed units of a compressed matrix as
they sit in device memory, the decoder template instances the product kernels
run: ``decode8p`` (FP32 tier: column dots, row chunks, multi-RHS panels) and
``decode8s<TIER_FF>`` (float-float tier).  Each value is compared with the CPU
oracle's decoder (Sec. 4.1, Alg. 8: ``oracle.codec.aflp_decode`` /
``fpx_decode``) applied to the same code:

* float-float tier: head + tail (summed in FP64) equals the oracle's value bit
  for bit.  AFLP values are compared as +-(s - 1), i.e. the oracle's decode with
  vmin = 1 (the kernels fold each array's vmin into the coefficient and tile
  scales).  The stated exceptions (raw FP64 and FPX e11 m52, whose low 29
  mantissa bits the tail keeps rounded to 24, 2^-48 relative; AFLP codes with
  m' >= 48 or f > 46, whose tail is one rounding of a sum wider than FP32,
  2^-46 relative) are held to 2^-46 relative, the float-float tier's own
  precision, instead, and counted.
* FP32 tier: head equals the oracle's value rounded to nearest FP32 (ties to
  even, numpy's float64 -> float32 cast), bit for bit, for every code that fits
  24 significant bits (FPX e8, AFLP up to 3 bytes); wider codes (4..7-byte AFLP,
  FPX e11, raw) follow the tier's stated approximation -- the mantissa cut to
  FP32's 23 bits, then s - 1 rounded once for AFLP -- bit for bit, within
  2^-22 + 2^-24 relative of the value; the number of values that differ from RN32 is
  counted.  The tail is zero.

Matrices: every format (H, UH, H^2, UH with separate couplings) at N = 2048,
AFLP and FPX at eps = 1e-4 .. 1e-14 and uncompressed; together they hold every
decode class the kernels instantiate (FPX e8 B = 2..4, e11 B = 5..8, AFLP
B = 1..7, raw FP64), zero codes and both signs (checked at the end).
"""
import numpy as np
import pytest

import synth
from decode_check import aflp_f, f32_tier_head, fields, oracle_values

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ALL_CLASSES = {(0, 2), (0, 3), (0, 4), (1, 5), (1, 6), (1, 7), (1, 8),
               (2, 1), (2, 2), (2, 3), (2, 4), (2, 5), (2, 6), (2, 7), (3, 8)}
SEEN = {"classes": set(), "zero": 0, "neg": 0, "pos": 0, "cases": 0}
NCASES = 4 * 3 + 3
COUNTS = {}
CUT = [0, 0]      # FP32-tier values that differ from RN32(value), of all checked


@pytest.fixture(scope="module")
def hm():
    from paper_2405_03456_gb300 import build, hm as _hm
    build.build()
    _hm.load()
    return _hm


def check_resident(hm, M, record=True):
    """Both tiers over every unit of M's payload; returns the number of
    compressed (non-raw) values held to the stated bound instead of bit
    equality in the float-float tier."""
    info = M.info()
    d_ff = hm.hm_decompress_debug(M.h, 1, 0, info["nunits"])
    d_32 = hm.hm_decompress_debug(M.h, 0, 0, info["nunits"])
    assert M.sync_status() == 0
    code, fmt = d_ff["code"], d_ff["fmt"]
    assert np.array_equal(code, d_32["code"]) and np.array_equal(fmt, d_32["fmt"])
    assert code.size > 0
    # hm_info's code bytes by width are the resident codes' widths
    widths = np.bincount((fmt.astype(np.int64) & 15), minlength=9)[1:9] * np.arange(1, 9)
    assert list(widths) == info["bytes_by_width"] and int(widths.sum()) == info["bytes_values"]
    v = oracle_values(code, fmt)
    B, F, E, Mb = fields(fmt)
    f = aflp_f(code, fmt)
    wide = ((F == 3) | ((F == 1) & (B == 8)) | ((F == 2) & ((Mb >= 48) | (f > 46))))
    tiny = np.abs(v) < 2.0 ** -74
    exact = ~(wide | tiny)
    # float-float tier: head + tail == value
    got = d_ff["head"].astype(np.float64) + d_ff["tail"].astype(np.float64)
    assert np.array_equal(got[exact].view(np.uint64), v[exact].view(np.uint64)), \
        np.flatnonzero(got[exact] != v[exact])[:5]
    rest = wide & ~tiny
    assert np.all(np.abs(got[rest] - v[rest]) <= 2.0 ** -46 * np.abs(v[rest]))
    small = tiny & (np.abs(v) >= 2.0 ** -126)      # FP64 entries whose tail falls below 2^-126: head only
    assert np.all(np.abs(got[small] - v[small]) <= 2.0 ** -23 * np.abs(v[small]))
    # FP32 tier: head == RN32(value) for codes that fit 24 bits, the stated
    # approximation (mantissa cut to 23 bits) for wider ones -- bit for bit --
    # and within 2^-22 + 2^-24 relative of the value; tail == 0
    want32 = f32_tier_head(code, fmt, v)
    ok32 = np.abs(v) >= 2.0 ** -126
    assert np.array_equal(d_32["head"][ok32].view(np.uint32), want32[ok32].view(np.uint32)), \
        np.flatnonzero(d_32["head"][ok32] != want32[ok32])[:5]
    h32 = d_32["head"].astype(np.float64)
    assert np.all(np.abs(h32[ok32] - v[ok32]) <= (2.0 ** -22 + 2.0 ** -24) * np.abs(v[ok32]))
    assert not np.any(d_32["tail"])
    rn = v.astype(np.float32)
    CUT[0] += int(np.count_nonzero(ok32 & (d_32["head"].view(np.uint32) != rn.view(np.uint32))))
    CUT[1] += int(np.count_nonzero(ok32))
    if record:
        SEEN["classes"] |= {(int(a), int(b)) for a, b in np.unique(np.stack([F, B], 1), axis=0)}
        SEEN["zero"] += int(np.count_nonzero(v == 0))
        SEEN["neg"] += int(np.count_nonzero(v < 0))
        SEEN["pos"] += int(np.count_nonzero(v > 0))
    return int(np.count_nonzero(~exact & ~tiny & ~(F == 3) & ~((F == 1) & (B == 8))))


N = 2048


@pytest.fixture(scope="module")
def pts():
    return synth.sphere_points(N)


@pytest.mark.parametrize("fmt", ["h", "uh", "h2", "uh_sep"])
@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_resident_decode_bit_exact(hm, pts, fmt, eps):
    M = hm.HMatrix(pts, "laplace", 32, 2.0, fmt, eps)
    try:
        for codec in ("aflp", "fpx", "none"):
            M.compress(eps, codec, True)
            nb = check_resident(hm, M)
            # the values held to the bound instead of bit equality are exactly the
            # AFLP codes of arrays whose dynamic range exceeds 2^46 (f > 46: the
            # value needs more than the 48 bits of a float-float pair), counted
            COUNTS[(fmt, eps, codec)] = nb
        SEEN["cases"] += 1
    finally:
        M.close()


@pytest.mark.parametrize("eps", [1e-10, 1e-12, 1e-14])
def test_resident_decode_wide_codes(hm, pts, eps):
    """Tight accuracies reach the wide classes: AFLP B = 5..7, FPX e11 B = 6..8, raw."""
    M = hm.HMatrix(pts, "laplace", 32, 2.0, "h", eps)
    try:
        for codec in ("aflp", "fpx"):
            M.compress(eps, codec, True)
            check_resident(hm, M)
        SEEN["cases"] += 1
    finally:
        M.close()


def test_resident_decode_partial_ranges(hm, pts):
    """Unit ranges concatenate to the whole payload; an empty range gives nothing."""
    M = hm.HMatrix(pts, "laplace", 32, 2.0, "h", 1e-6)
    try:
        M.compress(1e-6, "aflp", True)
        nu = M.info()["nunits"]
        whole = hm.hm_decompress_debug(M.h, 0, 0, nu)
        cut = nu // 3
        a = hm.hm_decompress_debug(M.h, 0, 0, cut)
        b = hm.hm_decompress_debug(M.h, 0, cut, nu + 5)
        for k in ("code", "fmt", "head"):
            assert np.array_equal(np.concatenate([a[k], b[k]]), whole[k])
        assert hm.hm_decompress_debug(M.h, 1, cut, cut)["code"].size == 0
    finally:
        M.close()


def test_zz_every_decode_class_seen():
    """The matrices above exercised every decode class, zero codes and both signs."""
    if SEEN["cases"] < NCASES:
        pytest.skip("needs every matrix case of this module in the same run")
    assert SEEN["classes"] >= ALL_CLASSES, sorted(ALL_CLASSES - SEEN["classes"])
    assert SEEN["zero"] > 0 and SEEN["neg"] > 0 and SEEN["pos"] > 0
    print(f"FP32 tier: {CUT[0]} of {CUT[1]} values differ from RN32 (the wide codes' stated approximation); "
          f"float-float values held to 2^-46 (f > 46): {COUNTS}")
