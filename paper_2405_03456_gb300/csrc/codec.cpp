// Host encoders of the floating point codecs of Sec. 4.1 (AFLP, FPX) and the
// VALR accuracy keys of Sec. 4.2.
//
// FPX (Fig. tab:fpx): a value is rounded once, to nearest with ties to even,
// from FP64 to the row's m mantissa bits (bit-pattern rounding carries into the
// exponent); e8 rows keep the FP32 exponent range and an array with any value
// outside the FP32 normal range moves to the e11 m28 row; an array with a value
// that rounds past the FP64 maximum moves to the exact e11 m52 row.  The code is the top
// B bytes of the FP32 (e8) or FP64 (e11) pattern.  The first table row (keys
// 0..10 -> e8m7) covers keys 0..8; keys 9 and 10 use e8m15 so that the
// rounding error 2^-(m+1) never exceeds 2^-key, as for every other row.
//
// AFLP: s = fl(fl(|v|/vmin) + 1) in [2, ...) is rounded to m' mantissa bits,
// its exponent f >= 1 stored in e bits (f = 0 encodes zero), e the bit length
// of the largest f (at least 1), m' >= m the smallest with 1+m'+e = 8B.
// Code layout: sign | f | mantissa.  If 1+m'+e > 56 or m' > 52, raw FP64; raw
// FP64 as well when s leaves the FP64 range (vmax/vmin + 1 overflows, or the
// rounded s reaches 2^1024), since no f then reproduces the value.
// Decoding: v = +-fl(fl(s - 1) * vmin).
//
// Compile with -ffp-contract=off: the divisions and additions must round as
// written.
#include <cmath>
#include <cstring>

#include "hm_internal.h"

namespace hm {

namespace {

inline uint64_t dbits(double v) {
  uint64_t u;
  std::memcpy(&u, &v, 8);
  return u;
}
inline double bitsd(uint64_t u) {
  double v;
  std::memcpy(&v, &u, 8);
  return v;
}

// round a non-negative FP64 bit pattern to drop d low bits, ties to even
inline uint64_t round_bits(uint64_t mag, int d) {
  if (d <= 0) return mag;
  uint64_t half = 1ull << (d - 1);
  uint64_t low = mag & ((1ull << d) - 1);
  uint64_t base = mag >> d;
  if (low > half || (low == half && (base & 1ull))) base += 1;
  return base << d;
}

inline int bit_length(uint64_t x) {
  int n = 0;
  while (x) {
    ++n;
    x >>= 1;
  }
  return n;
}

int aflp_mprime(int m, int e) {
  int mp = m;
  while ((1 + mp + e) % 8 != 0) ++mp;
  return mp;
}

}  // namespace

int ceil_log2(double r) {
  int ex;
  double mant = std::frexp(r, &ex);   // r = mant * 2^ex, mant in [0.5, 1)
  return mant == 0.5 ? ex - 1 : ex;
}

int m_eps(double eps) { return ceil_log2(1.0 / eps); }

int valr_key(double sigma, double delta) {
  double r = sigma / delta;
  if (!(r > 1.0)) return 1;
  int k = ceil_log2(r);
  return k < 1 ? 1 : (k > 52 ? 52 : k);
}

void fpx_format(int key, int& e, int& m) {
  if (key < 0) key = 0;
  if (key > 52) key = 52;
  if (key <= 8) { e = 8; m = 7; }
  else if (key <= 15) { e = 8; m = 15; }
  else if (key <= 23) { e = 8; m = 23; }
  else if (key <= 28) { e = 11; m = 28; }
  else if (key <= 36) { e = 11; m = 36; }
  else if (key <= 44) { e = 11; m = 44; }
  else { e = 11; m = 52; }
}

namespace {

bool fpx_try(const double* v, int64_t n, int64_t inc, int e, int m, uint64_t* codes) {
  const int B = (1 + e + m) / 8;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t b = dbits(v[i * inc]);
    uint64_t sign = b >> 63;
    uint64_t mag = round_bits(b & 0x7FFFFFFFFFFFFFFFull, 52 - m);
    if (e == 11) {
      if ((mag >> 52) == 0x7FF) return false;     // rounded to infinity
      codes[i] = ((sign << 63) | mag) >> (64 - 8 * B);
      continue;
    }
    uint32_t f32 = 0;
    if (mag != 0) {
      int ex = (int)(mag >> 52) - 1023;
      if (ex < -126 || ex > 127) return false;
      f32 = ((uint32_t)(ex + 127) << 23) | (uint32_t)((mag & ((1ull << 52) - 1)) >> 29);
    }
    f32 |= (uint32_t)sign << 31;
    codes[i] = (uint64_t)(f32 >> (32 - 8 * B));
  }
  return true;
}

}  // namespace

bool encode_values(const double* v, int64_t n, int64_t inc, int codec, int key, CodeHdr& h,
                   uint64_t* codes) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i * inc])) return false;
  if (codec == HM_CODEC_NONE) {
    h = CodeHdr();
    for (int64_t i = 0; i < n; ++i) codes[i] = dbits(v[i * inc]);
    return true;
  }
  if (codec == HM_CODEC_FPX) {
    int e, m;
    fpx_format(key, e, m);
    bool ok = fpx_try(v, n, inc, e, m, codes);
    if (!ok && e == 8) {          // out of the FP32 normal range
      e = 11;
      m = 28;
      ok = fpx_try(v, n, inc, e, m, codes);
    }
    if (!ok) {                    // rounded past the FP64 maximum
      e = 11;
      m = 52;
      fpx_try(v, n, inc, e, m, codes);
    }
    h.B = (1 + e + m) / 8;
    h.fmt = e == 8 ? FMT_FPX8 : FMT_FPX11;
    h.e = e;
    h.m = m;
    h.vmin = 1.0;
    return true;
  }
  // AFLP
  int m = key < 1 ? 1 : key;
  double vmin = 0, vmax = 0;
  bool any = false;
  for (int64_t i = 0; i < n; ++i) {
    double a = std::fabs(v[i * inc]);
    if (a > 0) {
      if (!any || a < vmin) vmin = a;
      if (!any || a > vmax) vmax = a;
      any = true;
    }
  }
  if (!any) {
    h.B = 1;
    h.fmt = FMT_AFLP;
    h.e = 1;
    h.m = 6;
    h.vmin = 1.0;
    for (int64_t i = 0; i < n; ++i) codes[i] = (dbits(v[i * inc]) >> 63) << 7;
    return true;
  }
  auto raw = [&]() {
    h.B = 8;
    h.fmt = FMT_RAW;
    h.e = 0;
    h.m = 52;
    h.vmin = vmin;
    for (int64_t i = 0; i < n; ++i) codes[i] = dbits(v[i * inc]);
    return true;
  };
  double smax = (vmax / vmin) + 1.0;
  if (!std::isfinite(smax)) return raw();
  int f0 = (int)(dbits(smax) >> 52) - 1023;
  int e = bit_length((uint64_t)f0);
  if (e < 1) e = 1;
  int mp = 0;
  for (int it = 0; it < 2; ++it) {
    mp = aflp_mprime(m, e);
    if (1 + mp + e > 56 || mp > 52) return raw();
    int fmax = 0;
    for (int64_t i = 0; i < n; ++i) {
      double a = std::fabs(v[i * inc]);
      if (!(a > 0)) continue;
      double s = (a / vmin) + 1.0;
      uint64_t sr = round_bits(dbits(s), 52 - mp);
      int f = (int)(sr >> 52) - 1023;
      if (f > fmax) fmax = f;
    }
    if (fmax > 1023) return raw();
    if (bit_length((uint64_t)fmax) <= e) break;
    e = bit_length((uint64_t)fmax);
    if (it == 1) return false;
  }
  const int B = (1 + mp + e) / 8;
  for (int64_t i = 0; i < n; ++i) {
    double x = v[i * inc];
    uint64_t sign = dbits(x) >> 63;
    double a = std::fabs(x);
    uint64_t code = sign << (8 * B - 1);
    if (a > 0) {
      double s = (a / vmin) + 1.0;
      uint64_t sr = round_bits(dbits(s), 52 - mp);
      uint64_t f = (sr >> 52) - 1023;
      uint64_t mant = (sr & ((1ull << 52) - 1)) >> (52 - mp);
      code |= (f << mp) | mant;
    }
    codes[i] = code;
  }
  h.B = B;
  h.fmt = FMT_AFLP;
  h.e = e;
  h.m = mp;
  h.vmin = vmin;
  return true;
}

double decode_value(uint64_t code, const CodeHdr& h) {
  switch (h.fmt) {
    case FMT_RAW:
      return bitsd(code);
    case FMT_FPX11:
      return bitsd(code << (64 - 8 * h.B));
    case FMT_FPX8: {
      uint32_t w = (uint32_t)(code << (32 - 8 * h.B));
      float f;
      std::memcpy(&f, &w, 4);
      return (double)f;
    }
    default: {
      uint64_t sign = (code >> (8 * h.B - 1)) & 1ull;
      uint64_t f = (code >> h.m) & ((1ull << h.e) - 1);
      uint64_t mant = code & ((1ull << h.m) - 1);
      double v = 0.0;
      if (f != 0) {
        double s = bitsd(((f + 1023) << 52) | (mant << (52 - h.m)));
        v = (s - 1.0) * h.vmin;
      }
      return sign ? -v : v;
    }
  }
}

}  // namespace hm
