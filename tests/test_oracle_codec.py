"""Pins of the oracle's codecs (Sec. 4.1 AFLP / FPX, Sec. 4.2 VALR widths).

Each check ties the oracle to something other than itself: values the paper
prints (tests/golden/paper_values.json), IEEE casts done by numpy, exact
rational rounding with ``fractions``, and the stated error bounds.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import codec as cd

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ------------------------------------------------------------ exact rounding
def rne_fraction(v: float, m: int) -> Fraction:
    """Round v to m mantissa bits (unbounded exponent), ties to even, exactly."""
    if v == 0.0:
        return Fraction(0)
    x = Fraction(v)
    a = abs(x)
    e = math.floor(math.log2(a))
    # make the exponent exact
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    ulp = Fraction(2) ** (e - m)
    q = a / ulp
    lo = math.floor(q)
    rem = q - lo
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    r = lo * ulp
    return r if x > 0 else -r


def test_m_eps_worked_examples():
    for k, v in GOLD["m_eps_examples"].items():
        if k.startswith("_"):
            continue
        assert cd.m_eps(float(k)) == v


def test_ceil_log2_brute_force():
    rng = np.random.default_rng(3)
    vals = list(10.0 ** rng.uniform(-20, 20, 2000)) + [2.0 ** k for k in range(-30, 30)]
    vals += [math.nextafter(2.0 ** k, 0) for k in range(-5, 5)] + [math.nextafter(2.0 ** k, 10) for k in range(-5, 5)]
    for r in vals:
        k = cd.ceil_log2(r)
        assert Fraction(2) ** (k - 1) < Fraction(r) <= Fraction(2) ** k


def test_fpx_table_matches_paper_except_first_row_reading():
    rows = GOLD["fpx_table"]["rows"]
    for lo, hi, e, m in rows:
        for key in range(lo, hi + 1):
            if key in (9, 10):        # reading: e8m7 cannot reach 2^-9 / 2^-10
                assert cd.fpx_format(key) == (8, 15)
            else:
                assert cd.fpx_format(key) == (e, m)
    # the rule the reading restores: rounding error 2^-(m+1) <= 2^-key for every key
    for key in range(0, 53):
        e, m = cd.fpx_format(key)
        assert m + 1 >= key


def test_fpx_bytes_examples():
    for k, nb in GOLD["fpx_bytes_examples"].items():
        if k.startswith("_"):
            continue
        e, m = cd.fpx_format(cd.m_eps(float(k)))
        assert cd.fpx_bytes(e, m) == nb


def test_fpx_e8m23_is_ieee_float32_cast():
    v = np.concatenate([synth.codec_values(20000, 1e6, seed=s) for s in range(5)])
    c = cd.fpx_encode(v, 8, 23)
    d = cd.fpx_decode(c, 8, 23)
    assert np.array_equal(d, v.astype(np.float32).astype(np.float64))


def test_fpx_e11m52_is_identity():
    v = np.concatenate([synth.codec_values(5000, 1e12, zero_frac=0.1, seed=s) for s in range(3)])
    v = np.concatenate([v, [0.0, -0.0, 5e-324, -1e300]])
    c = cd.fpx_encode(v, 11, 52)
    d = cd.fpx_decode(c, 11, 52)
    assert np.array_equal(d.view(np.uint64), v.view(np.uint64))


def test_unit_roundoff_matches_paper_table():
    """FPX e8m23 and e8m7 have the unit roundoffs the paper prints for FP32 and BF16."""
    ur = GOLD["unit_roundoff"]
    v = synth.codec_values(200000, 1e4, seed=11)
    for (e, m), name in [((8, 23), "FP32"), ((8, 7), "BF16")]:
        d = cd.fpx_decode(cd.fpx_encode(v, e, m), e, m)
        rel = np.max(np.abs(d - v) / np.abs(v) / (1 + 0 * v))
        u = 2.0 ** (-(m + 1))
        assert rel <= u
        assert rel > 0.9 * u          # the bound is attained closely on random data
        assert abs(u - ur[name]) / ur[name] < 5e-3
        key = {23: 20, 7: 5}[m]                 # table rows e8m23 and e8m7
        assert cd.unit_error(cd.fpx_compress(v, key)) == u
    assert abs(2.0 ** -53 - ur["FP64"]) / ur["FP64"] < 5e-3
    # AFLP: the stated per-value relative bound 2^-m' of its mantissa width
    c = cd.aflp_compress(v, 20)
    assert not c["raw"] and cd.unit_error(c) == 2.0 ** -c["mp"]
    d = cd.decompress(c)
    rel = np.max(np.abs(d - v) / np.abs(v))
    assert 2.0 ** -(c["mp"] + 2) < rel <= cd.unit_error(c)


def _fpx_cases():
    rng = np.random.default_rng(5)
    base = list(synth.codec_values(300, 1e5, zero_frac=0.05, seed=21))
    # exact ties and carries for each m
    extra = []
    for m in (7, 15, 23, 28, 36, 44):
        for _ in range(20):
            e = int(rng.integers(-20, 20))
            j = int(rng.integers(1 << m, 1 << (m + 1)))
            extra.append(float(Fraction(2 * j + 1, 2) * Fraction(2) ** (e - m)))   # tie
        extra.append(float(Fraction(2) ** 3 * (2 - Fraction(1, 2 ** (m + 3)))))    # carry to 2^4
    return base + extra


@pytest.mark.parametrize("e,m", [(8, 7), (8, 15), (8, 23), (11, 28), (11, 36), (11, 44), (11, 52)])
def test_fpx_is_round_to_nearest_even_brute_force(e, m):
    vals = np.array([v for v in _fpx_cases() if v == 0 or abs(v) < 2.0 ** 126 and abs(v) > 2.0 ** -120])
    c = cd.fpx_encode(vals, e, m)
    assert c is not None
    d = cd.fpx_decode(c, e, m)
    for v, dv in zip(vals, d):
        assert Fraction(float(dv)) == rne_fraction(float(v), m), (v, dv)


def test_fpx_idempotent_and_promotion():
    v = synth.codec_values(5000, 1e8, seed=31)
    for key in (5, 14, 20, 27, 33, 40, 50):
        c = cd.fpx_compress(v, key)
        d = cd.decompress(c)
        c2 = cd.fpx_encode(d, c["e"], c["m"])
        assert np.array_equal(c2, c["codes"])
        assert np.all(np.abs(d - v) <= cd.unit_error(c) * np.abs(v))
    big = np.array([1.0, 3e40, -2.0])
    c = cd.fpx_compress(big, 20)
    assert (c["e"], c["m"]) == (11, 28)
    tiny = np.array([1.0, 1e-40])
    assert (cd.fpx_compress(tiny, 14)["e"]) == 11


def test_aflp_bytes_examples():
    for case in GOLD["aflp_bytes_examples"]["cases"]:
        v = np.array([1.0, case["ratio"], -3.0, 7.5])
        c = cd.aflp_compress(v, cd.m_eps(case["eps"]))
        assert (c["e"], c["mp"], c["B"]) == (case["e"], case["mprime"], case["bytes"])
        # e agrees with the paper's e_dr formula for this ratio
        assert c["e"] == math.ceil(math.log2(math.log2(case["ratio"])))


@pytest.mark.parametrize("m", [1, 5, 8, 14, 20, 27, 33, 44])
@pytest.mark.parametrize("dr", [1.0, 2.0, 1e2, 1e6, 1e30])
def test_aflp_brute_force_and_bound(m, dr):
    v = synth.codec_values(400, dr, zero_frac=0.05, seed=int(m * 7 + math.log10(dr + 1)))
    c = cd.aflp_compress(v, m)
    d = cd.decompress(c)
    if c["raw"]:
        assert np.array_equal(d.view(np.uint64), v.view(np.uint64))
        return
    B, e, mp, vmin = c["B"], c["e"], c["mp"], c["vmin"]
    assert (1 + mp + e) % 8 == 0 and mp >= m and 1 + mp + e == 8 * B
    nz = v != 0
    assert vmin == np.min(np.abs(v[nz]))
    # codes: s rounded to m' bits (exact rationals), f >= 1 stored, e minimal
    fs = []
    for vi, code in zip(v, c["codes"]):
        code = int(code)
        assert (code >> (8 * B - 1)) == (1 if math.copysign(1, vi) < 0 else 0)
        f = (code >> mp) & ((1 << e) - 1)
        if vi == 0:
            assert f == 0 and (code & ((1 << mp) - 1)) == 0
            continue
        s = (abs(vi) / vmin) + 1.0
        st = rne_fraction(s, mp)
        mant = code & ((1 << mp) - 1)
        assert Fraction(2) ** f * (1 + Fraction(mant, 2 ** mp)) == st
        fs.append(f)
    assert e == max(1, max(fs).bit_length())
    # per-value bound: |v - v~| <= 2^-(m'+1) (|v| + vmin) plus FP64 rounding
    err = np.abs(d - v)
    bound = 2.0 ** (-(mp + 1)) * (np.abs(v) + vmin) + 8 * 2.0 ** -53 * (np.abs(v) + vmin)
    assert np.all(err <= bound)
    assert np.all(np.abs(d[nz]) > 0) and np.all(d[~nz] == 0)
    # relative error at most 2^-m' (so at most 2^-m), Sec. 4.1
    assert np.all(err[nz] <= (2.0 ** -mp + 2.0 ** -50) * np.abs(v[nz]))


def test_aflp_exact_points_and_full_width():
    v = np.array([0.25, -0.25, 1.0, 0.0, -0.0])
    c = cd.aflp_compress(v, 10)
    d = cd.decompress(c)
    assert d[0] == 0.25 and d[1] == -0.25 and d[2] == 1.0
    assert np.array_equal(d[3:].view(np.uint64), v[3:].view(np.uint64))
    w = synth.codec_values(1000, 1e3, seed=2)
    c = cd.aflp_compress(w, 52)
    assert c["raw"] and np.array_equal(cd.decompress(c), w)
    z = np.zeros(10)
    c = cd.aflp_compress(z, 20)
    assert c["B"] == 1 and np.array_equal(cd.decompress(c), z)


def test_aflp_rounding_carry_raises_exponent_bits():
    # s = 2^4 - tiny rounds up to 2^4: f = 4 needs 3 bits although 2^4 - tiny has f = 3
    vmin = 1.0
    s_minus = 16.0 - 2.0 ** -20
    v = np.array([vmin, s_minus - 1.0])
    c = cd.aflp_compress(v, 6)
    assert c["e"] == 3
    assert cd.decompress(c)[1] == 15.0


@pytest.mark.parametrize("v", [
    np.array([1e-300, 1e-200, 5e-324, -7.0]),            # |v|/vmin + 1 overflows
    np.array([1.0, -np.finfo(np.float64).max]),           # finite s rounds up to 2^1024
])
def test_aflp_beyond_fp64_range_stays_exact(v):
    # no exponent f of s = |v|/vmin + 1 fits FP64: the array is kept as raw FP64
    for m in (1, 7, 20, 30):
        c = cd.aflp_compress(v, m)
        d = cd.decompress(c)
        assert np.all(np.isfinite(d))
        assert c["raw"] and np.array_equal(d.view(np.uint64), v.view(np.uint64))


def test_fpx_beyond_fp64_maximum_moves_to_exact_row():
    big = np.finfo(np.float64).max
    v = np.array([1.0, -big, 3.0])
    for key in (5, 20, 24, 30, 40):
        c = cd.fpx_compress(v, key)
        assert (c["e"], c["m"]) == (11, 52)
        assert np.array_equal(cd.decompress(c), v)
    w = np.array([1.0, -2.0 ** 1023 * 1.5])                 # exact in e11m28: no promotion
    c = cd.fpx_compress(w, 24)
    assert (c["e"], c["m"]) == (11, 28) and np.array_equal(cd.decompress(c), w)


def test_fpx_e8_range_boundaries():
    # the FP32 normal range is [2^-126, 2^128): its ends stay in the e8 rows
    lo, hi = 2.0 ** -126, 1.5 * 2.0 ** 127
    c = cd.fpx_compress(np.array([lo, -hi, 1.0]), 20)
    assert (c["e"], c["m"]) == (8, 23)
    assert np.array_equal(cd.decompress(c), np.array([lo, -hi, 1.0]))
    for out in (2.0 ** -127, (2.0 - 2.0 ** -30) * 2.0 ** 127):   # subnormal; rounds up to 2^128
        c = cd.fpx_compress(np.array([out, 1.0]), 20)
        assert (c["e"], c["m"]) == (11, 28)


def test_aflp_largest_exponent_fits():
    # s just below 2^1024 (f = 1023) is still an AFLP code; the next carry is raw
    v = np.array([1.0, 1.5 * 2.0 ** 1023])
    c = cd.aflp_compress(v, 20)
    assert not c["raw"] and c["e"] == 10
    assert np.all(np.abs(cd.decompress(c) - v) <= cd.unit_error(c) * np.abs(v))


def test_ceil_log2_rejects_nonpositive():
    for r in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(ValueError):
            cd.ceil_log2(r)


def test_valr_key_brute_force():
    rng = np.random.default_rng(9)
    for _ in range(3000):
        s = 10.0 ** rng.uniform(-8, 3)
        d = 10.0 ** rng.uniform(-12, 0)
        k = cd.valr_key(s, d)
        r = Fraction(s) / Fraction(d) if False else Fraction(s / d)
        if r <= 1:
            assert k == 1
        else:
            kk = min(max(math.ceil(math.log2(s / d) - 1e-12), 1), 52)
            if abs(math.log2(s / d) - round(math.log2(s / d))) > 1e-9:
                assert k == kk
            assert Fraction(2) ** (k - 1) < r or k == 1
            assert r <= Fraction(2) ** k or k == 52
