// Device helpers of libhm: float-float arithmetic and the on-the-fly decoders
// of the packed formats (Sec. 4.1: AFLP and FPX; raw FP64 for the uncompressed
// baseline), and the bulk-copy / mbarrier primitives of the streaming kernels.
//
// Arithmetic (GB300 runs FP64 FMA at 1/60 of the FP32 rate):
//  * every packed value is decoded with integer and FP32 operations; AFLP
//    values are decoded as +-(s - 1), their per-array vmin being folded into
//    the coefficient vectors or tile scales;
//  * TIER_F32 (eps > 2^-22): one FP32 value per entry, the stored value
//    rounded to nearest FP32 (ties to even) where it fits 24 bits, wider codes
//    cut to 23 mantissa bits first (see decode4);
//  * TIER_FF (eps <= 2^-22 and the uncompressed baseline): entries as
//    float-float pairs that equal the stored value exactly (see decode4), and
//    vector values as float-float pairs, products accumulated with the
//    compensated dot product of Ogita, Rump and Oishi (2005, "Dot2":
//    TwoProduct by FMA, TwoSum of Knuth), about 2^-46 relative.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dev_types.h"

namespace hm {

#define HM_FULL 0xffffffffu

__device__ __forceinline__ uint32_t pad8u(uint32_t x) { return (x + 7u) & ~7u; }

__device__ __forceinline__ void latch_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------- float-float
struct FF {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  float h = s + e;
  return {h, e - (h - s)};
}

__device__ __forceinline__ FF ff_add_f(FF a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e += a.lo;
  float h = s + e;
  return {h, e - (h - s)};
}

// (a.hi + a.lo) * (b.hi + b.lo) to about 2^-46
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  float h = p + e;
  return {h, e - (h - p)};
}

__device__ __forceinline__ FF ff_from_d(double v) {
  float h = (float)v;
  return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double ff_to_d(FF a) { return (double)a.hi + (double)a.lo; }

// Dot2 accumulation of d*v into (s, c)
__device__ __forceinline__ void dot2(float& s, float& c, float dh, float dl, float vh, float vl) {
  float p = dh * vh;
  float pe = fmaf(dh, vh, -p);
  float tail = fmaf(dh, vl, fmaf(dl, vh, pe));
  float s1 = s + p;
  float bp = s1 - s;
  float e = (s - (s1 - bp)) + (p - bp);
  s = s1;
  c += e + tail;
}

// ---------------------------------------------------------------- decoding
// Value i of 4 consecutive B-byte codes held in B little-endian words, placed
// at the top of a 32-bit (B <= 4) or 64-bit (B >= 5) window.
template <int B, int I>
__device__ __forceinline__ uint32_t top32(const uint32_t (&w)[B]) {
  constexpr int o = I * B + B - 4;
  if constexpr (o < 0) {
    return w[0] << (8 * (-o));
  } else {
    constexpr int wi = o >> 2, sh = (o & 3) * 8;
    if constexpr (sh == 0)
      return w[wi];
    else
      return __funnelshift_r(w[wi], w[wi + 1], sh);
  }
}

template <int B, int I>
__device__ __forceinline__ uint64_t top64(const uint32_t (&w)[B]) {
  constexpr int o = I * B + B - 8;
  if constexpr (o < 0) {
    uint64_t v = ((uint64_t)w[1] << 32) | w[0];
    return v << (8 * (-o));
  } else {
    constexpr int wi = o >> 2, sh = (o & 3) * 8;
    uint64_t v = ((uint64_t)w[wi + 1] << 32) | w[wi];
    if constexpr (sh == 0) {
      return v;
    } else {
      return (v >> sh) | ((uint64_t)w[wi + 2] << (64 - sh));
    }
  }
}

// FP64 bit pattern -> value.  hi = the top 24 significant bits (the mantissa
// cut to FP32's 23 bits); TIER_FF: lo = the rest, exact when the pattern has at
// most 48 significant bits (every FPX e11 code up to m = 44; the 52-bit
// mantissa of a raw FP64 value keeps its lo part rounded to 24 bits);
// TIER_F32: lo = 0 (the FP32 tier's stated approximation: within 2^-22 + 2^-24
// relative).  Values below 2^-126 give hi = 0, and lo is dropped below 2^-74.
template <int TIER>
__device__ __forceinline__ void split_f64bits(uint64_t P, float& hi, float& lo) {
  const uint32_t sgn = (uint32_t)(P >> 32) & 0x80000000u;
  const int E = (int)((P >> 52) & 0x7ff);
  const uint64_t M = P & ((1ull << 52) - 1);
  const uint32_t hb = (E >= 897) ? (((uint32_t)(E - 896) << 23) | (uint32_t)(M >> 29)) : 0u;
  hi = __uint_as_float(hb | sgn);
  lo = 0.0f;
  if constexpr (TIER == TIER_FF) {
    if (E >= 949) {
      float l = __uint2float_rn((uint32_t)(M & ((1u << 29) - 1)));
      l *= __uint_as_float((uint32_t)(E - 948) << 23);
      lo = __uint_as_float(__float_as_uint(l) ^ sgn);
    }
  }
}

// AFLP difference s - 1 of s = 2^f (1 + mant 2^-m') as float-float d + err,
// given s_h (FP32, exact: s with its mantissa cut to 23 bits): d = fl(s_h - 1)
// and err = (s_h - d) - 1, the exact rounding error of that subtraction (the
// Fast2Sum error term: s_h >= 2 > 1, so both operations are exact).  err is 0
// unless f >= 24.
__device__ __forceinline__ void aflp_sub1(float sh, float& d, float& err) {
  d = sh - 1.0f;
  err = (sh - d) - 1.0f;
}

// Decode 4 consecutive values of format (F, B).
//   TIER_FF: h + l equals the stored value exactly (AFLP as +-(s - 1): every
//     code whose low mantissa part fits FP32, i.e. m' <= 47, and f <= 46; FPX
//     codes up to e11 m44; see split_f64bits for raw FP64).
//   TIER_F32: l = 0 and h = the stored value rounded to nearest FP32 (ties to
//     even) for every code that fits 24 significant bits (FPX e8, AFLP up to 3
//     bytes); wider codes are cut to FP32's 23 mantissa bits first (AFLP:
//     h = fl(s_h - 1) with s_h = s cut to 23 mantissa bits; FPX e11 and raw:
//     the top 24 significant bits), within 2^-22 + 2^-24 relative of the value -- the
//     FP32 tier's stated approximation, which keeps its decode as cheap as the
//     short codes' (the tier computes in FP32 anyway).
template <int TIER, int F, int B>
__device__ __forceinline__ void decode4(const uint32_t (&w)[B], int e, int m, float (&h)[4],
                                        float (&l)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) l[i] = 0.0f;
  if constexpr (F == 0) {                                   // FPX e8: the code is the FP32 top
    constexpr uint32_t mask = 0xffffffffu << (8 * (4 - B));
    h[0] = __uint_as_float(top32<B, 0>(w) & mask);
    h[1] = __uint_as_float(top32<B, 1>(w) & mask);
    h[2] = __uint_as_float(top32<B, 2>(w) & mask);
    h[3] = __uint_as_float(top32<B, 3>(w) & mask);
  } else if constexpr (F == 2 && B <= 3) {
    // AFLP with s exact in FP32 (m' <= 22); d = fl(s - 1) is the value rounded
    // to FP32, and the FF tier keeps its rounding error (nonzero when f >= 24).
    // Values in pairs (FADD2 on Blackwell).
    constexpr uint32_t mask = (0xffffffffu << (8 * (4 - B))) & 0x7fffffffu;
    const int sh = 8 - e;
    const uint32_t t[4] = {top32<B, 0>(w), top32<B, 1>(w), top32<B, 2>(w), top32<B, 3>(w)};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t t0 = t[2 * k], t1 = t[2 * k + 1];
      const float2 sv = make_float2(__uint_as_float(((t0 & mask) >> sh) + (127u << 23)),
                                    __uint_as_float(((t1 & mask) >> sh) + (127u << 23)));
      const float2 d = __fadd2_rn(sv, make_float2(-1.0f, -1.0f));
      h[2 * k] = __uint_as_float(__float_as_uint(d.x) ^ (t0 & 0x80000000u));
      h[2 * k + 1] = __uint_as_float(__float_as_uint(d.y) ^ (t1 & 0x80000000u));
      if constexpr (TIER == TIER_FF) {
        const float2 err = __fadd2_rn(__ffma2_rn(d, make_float2(-1.0f, -1.0f), sv), make_float2(-1.0f, -1.0f));
        l[2 * k] = __uint_as_float(__float_as_uint(err.x) ^ (t0 & 0x80000000u));
        l[2 * k + 1] = __uint_as_float(__float_as_uint(err.y) ^ (t1 & 0x80000000u));
      }
    }
  } else if constexpr (F == 2 && B == 4) {
    // AFLP in 32 bits.  The code fills the word (m' = 31 - e): the head
    // s_h = 2^f (1 + top 23 mantissa bits) is exact in FP32, the sh = 8 - e = m' - 23
    // bits shifted out form the tail t 2^(f - m'), t < 2^sh (exact: t via the
    // 2^23 bit pattern).  s - 1 = d + err + tail; err + tail is exact for f <= 46.
    // The FP32 tier keeps d = fl(s_h - 1), the value with its mantissa cut to
    // 23 bits and then rounded once (within 2^-22 + 2^-24 relative).  Values in pairs.
    const int sh = 8 - e;
    const uint32_t tmask = (1u << sh) - 1u, mexp = (uint32_t)m << 23;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t c0 = w[2 * k], c1 = w[2 * k + 1];
      const uint32_t s0 = ((c0 & 0x7fffffffu) >> sh) + (127u << 23), s1 = ((c1 & 0x7fffffffu) >> sh) + (127u << 23);
      const float2 sv = make_float2(__uint_as_float(s0), __uint_as_float(s1));
      const float2 d = __fadd2_rn(sv, make_float2(-1.0f, -1.0f));
      h[2 * k] = __uint_as_float(__float_as_uint(d.x) ^ (c0 & 0x80000000u));
      h[2 * k + 1] = __uint_as_float(__float_as_uint(d.y) ^ (c1 & 0x80000000u));
      if constexpr (TIER == TIER_FF) {
        const float2 err = __fadd2_rn(__ffma2_rn(d, make_float2(-1.0f, -1.0f), sv), make_float2(-1.0f, -1.0f));
        const float2 tv = __fadd2_rn(make_float2(__uint_as_float((c0 & tmask) | 0x4B000000u),
                                                 __uint_as_float((c1 & tmask) | 0x4B000000u)),
                                     make_float2(-8388608.0f, -8388608.0f));
        const float2 sc = make_float2(__uint_as_float((s0 & 0x7f800000u) - mexp),
                                      __uint_as_float((s1 & 0x7f800000u) - mexp));
        const float2 lv = __ffma2_rn(tv, sc, err);
        l[2 * k] = __uint_as_float(__float_as_uint(lv.x) ^ (c0 & 0x80000000u));
        l[2 * k + 1] = __uint_as_float(__float_as_uint(lv.y) ^ (c1 & 0x80000000u));
      }
    }
  } else if constexpr (F == 2) {                           // AFLP with m' > 23, B >= 5
    uint64_t c[4];
    constexpr int rs = 64 - 8 * B;
    c[0] = top64<B, 0>(w) >> rs;
    c[1] = top64<B, 1>(w) >> rs;
    c[2] = top64<B, 2>(w) >> rs;
    c[3] = top64<B, 3>(w) >> rs;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t sg = (uint32_t)(c[i] >> (8 * B - 1)) << 31;
      const uint32_t f = (uint32_t)(c[i] >> m) & ((1u << e) - 1u);
      const uint64_t mant = c[i] & ((1ull << m) - 1ull);
      const uint32_t hb = ((f + 127u) << 23) | (uint32_t)(mant >> (m - 23));
      float d, err;
      aflp_sub1(__uint_as_float(hb), d, err);
      h[i] = __uint_as_float(__float_as_uint(d) ^ sg);
      if constexpr (TIER == TIER_FF) {
        const uint64_t ml = mant & ((1ull << (m - 23)) - 1ull);
        const float lv = __ull2float_rn(ml) * __uint_as_float((uint32_t)(f + 127 - m) << 23) + err;
        l[i] = __uint_as_float(__float_as_uint(lv) ^ sg);
      }
    }
  } else {                                                  // FPX e11 or raw FP64
    constexpr uint64_t mask = (B == 8) ? ~0ull : (~0ull << (8 * (8 - B)));
    split_f64bits<TIER>(top64<B, 0>(w) & mask, h[0], l[0]);
    split_f64bits<TIER>(top64<B, 1>(w) & mask, h[1], l[1]);
    split_f64bits<TIER>(top64<B, 2>(w) & mask, h[2], l[2]);
    split_f64bits<TIER>(top64<B, 3>(w) & mask, h[3], l[3]);
  }
}

// Shared-memory loads by 32-bit shared address.
__device__ __forceinline__ uint2 lds64(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint4 lds128(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}

// A lane's 8 consecutive codes of one column in shared memory: 8*B bytes at
// an 8-byte aligned shared address, read as B 64-bit loads, decoded to 8
// values (hi, and lo for TIER_FF).
template <int TIER, int F, int B>
__device__ __forceinline__ void decode8s(uint32_t a, int e, int m, float (&h)[8], float (&l)[8]) {
  uint32_t w[2 * B];
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const uint2 t = lds64(a + 8u * i);
    w[2 * i] = t.x;
    w[2 * i + 1] = t.y;
  }
  uint32_t w0[B], w1[B];
#pragma unroll
  for (int i = 0; i < B; ++i) {
    w0[i] = w[i];
    w1[i] = w[B + i];
  }
  float h0[4], l0[4], h1[4], l1[4];
  decode4<TIER, F, B>(w0, e, m, h0, l0);
  decode4<TIER, F, B>(w1, e, m, h1, l1);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    h[u] = h0[u];
    h[4 + u] = h1[u];
    l[u] = l0[u];
    l[4 + u] = l1[u];
  }
}

// ---------------------------------------------------------------- FP32-tier paired decode
// Blackwell issues two FP32 operations per instruction on register pairs
// (__fadd2_rn / __ffma2_rn); the FP32 tier decodes and accumulates rows in
// pairs (2k, 2k+1).

// a - b per component, one rounding (FFMA2 with a -1 multiplier).
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// two_sum on pairs: (s, e) with s + e = a + b exactly, per component (Knuth).
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  const float2 bp = sub2(s, a);
  e = __fadd2_rn(sub2(a, sub2(s, bp)), sub2(b, bp));
}

// (hi, lo) += s per component (float-float accumulation of FP32 partial sums).
__device__ __forceinline__ void ff_add_f2(float2& hi, float2& lo, float2 s) {
  float2 t, e;
  two_sum2(hi, s, t, e);
  e = __fadd2_rn(e, lo);
  const float2 h = __fadd2_rn(t, e);
  lo = sub2(e, sub2(h, t));
  hi = h;
}

// Dot2 (Ogita-Rump-Oishi) on pairs: (s, c) += d * v per component, with d and
// v float-float (dh + dl, vh + vl): TwoProduct by FMA, TwoSum of Knuth.
__device__ __forceinline__ void dot2_2(float2& s, float2& c, float2 dh, float2 dl, float2 vh, float2 vl) {
  const float2 p = __fmul2_rn(dh, vh);
  const float2 pe = __ffma2_rn(dh, vh, make_float2(-p.x, -p.y));
  const float2 tail = __ffma2_rn(dh, vl, __ffma2_rn(dl, vh, pe));
  const float2 s1 = __fadd2_rn(s, p);
  const float2 bp = sub2(s1, s);
  const float2 e = __fadd2_rn(sub2(s, sub2(s1, bp)), sub2(p, bp));
  s = s1;
  c = __fadd2_rn(c, __fadd2_rn(e, tail));
}

// (hi, lo) += (s + c) per component, float-float (the Dot2 pair folded first).
__device__ __forceinline__ void ff_add_dot2(float2& hi, float2& lo, float2 s, float2 c) {
  const float2 h = __fadd2_rn(s, c);
  const float2 l = sub2(c, sub2(h, s));
  float2 t, e;
  two_sum2(hi, h, t, e);
  e = __fadd2_rn(e, __fadd2_rn(lo, l));
  const float2 hh = __fadd2_rn(t, e);
  lo = sub2(e, sub2(hh, t));
  hi = hh;
}

// 8 consecutive codes of format (F, B) at shared address a -> 4 FP32 pairs
// (FP32 tier: AFLP as +-(s - 1), FPX e8 exactly, e11 / raw cut to FP32; see
// decode4 for what each class gives).
template <int F, int B>
__device__ __forceinline__ void decode8p(uint32_t a, int e, int m, float2 (&h2)[4]) {
  uint32_t w[2 * B];
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const uint2 t = lds64(a + 8u * i);
    w[2 * i] = t.x;
    w[2 * i + 1] = t.y;
  }
  uint32_t w0[B], w1[B];
#pragma unroll
  for (int i = 0; i < B; ++i) {
    w0[i] = w[i];
    w1[i] = w[B + i];
  }
  if constexpr (F == 2 && B <= 4) {
    // AFLP: s with its mantissa cut to the 23 bits of FP32 (exact for B <= 3),
    // then fl(s - 1): the value rounded to FP32 for B <= 3; for 4-byte codes
    // (m' = 24 .. 30) the bits below FP32's mantissa are dropped first (the FP32
    // tier's stated approximation: within 2^-22 + 2^-24 relative of the value)
    constexpr uint32_t mask = (0xffffffffu << (8 * (4 - B))) & 0x7fffffffu;
    const int sh = 8 - e;
    const uint32_t t[8] = {top32<B, 0>(w0), top32<B, 1>(w0), top32<B, 2>(w0), top32<B, 3>(w0),
                           top32<B, 0>(w1), top32<B, 1>(w1), top32<B, 2>(w1), top32<B, 3>(w1)};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 sv = make_float2(__uint_as_float(((t[2 * k] & mask) >> sh) + (127u << 23)),
                                    __uint_as_float(((t[2 * k + 1] & mask) >> sh) + (127u << 23)));
      const float2 d = __fadd2_rn(sv, make_float2(-1.0f, -1.0f));
      h2[k] = make_float2(__uint_as_float(__float_as_uint(d.x) ^ (t[2 * k] & 0x80000000u)),
                          __uint_as_float(__float_as_uint(d.y) ^ (t[2 * k + 1] & 0x80000000u)));
    }
  } else if constexpr (F == 0) {
    constexpr uint32_t mask = 0xffffffffu << (8 * (4 - B));
    h2[0] = make_float2(__uint_as_float(top32<B, 0>(w0) & mask), __uint_as_float(top32<B, 1>(w0) & mask));
    h2[1] = make_float2(__uint_as_float(top32<B, 2>(w0) & mask), __uint_as_float(top32<B, 3>(w0) & mask));
    h2[2] = make_float2(__uint_as_float(top32<B, 0>(w1) & mask), __uint_as_float(top32<B, 1>(w1) & mask));
    h2[3] = make_float2(__uint_as_float(top32<B, 2>(w1) & mask), __uint_as_float(top32<B, 3>(w1) & mask));
  } else {
    float h0[4], l0[4], h1[4], l1[4];
    decode4<TIER_F32, F, B>(w0, e, m, h0, l0);
    decode4<TIER_F32, F, B>(w1, e, m, h1, l1);
    h2[0] = make_float2(h0[0], h0[1]);
    h2[1] = make_float2(h0[2], h0[3]);
    h2[2] = make_float2(h1[0], h1[1]);
    h2[3] = make_float2(h1[2], h1[3]);
  }
}

// ---------------------------------------------------------------- tensor-core helpers
// x = t0 + t1 + t2 with BF16 limbs t by truncation (each step keeps the top 8
// significant bits of the remainder; the remainders are exact FP32
// differences); limbs of x in the low half, of y in the high half.
__device__ __forceinline__ void limbs2(float x, float y, uint32_t& l0, uint32_t& l1, uint32_t& l2) {
  const uint32_t xu = __float_as_uint(x), yu = __float_as_uint(y);
  l0 = __byte_perm(xu, yu, 0x7632);
  const float2 r1 = sub2(make_float2(x, y), make_float2(__uint_as_float(xu & 0xffff0000u), __uint_as_float(yu & 0xffff0000u)));
  const uint32_t ru = __float_as_uint(r1.x), rv = __float_as_uint(r1.y);
  l1 = __byte_perm(ru, rv, 0x7632);
  const float2 r2 = sub2(r1, make_float2(__uint_as_float(ru & 0xffff0000u), __uint_as_float(rv & 0xffff0000u)));
  l2 = __byte_perm(__float_as_uint(r2.x), __float_as_uint(r2.y), 0x7632);
}

// The decode classes (F, B) the kernels instantiate.
#define HM_FORMATS(X) \
  X(0, 2) X(0, 3) X(0, 4) X(1, 5) X(1, 6) X(1, 7) X(1, 8) \
  X(2, 1) X(2, 2) X(2, 3) X(2, 4) X(2, 5) X(2, 6) X(2, 7) X(3, 8)

// ---------------------------------------------------------------- bulk copies and mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait: each try suspends the thread until the phase completes or
// about `hint_ns` pass; gives up after `limit` tries (about 2 s) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = 2000u) {
  const uint32_t hint_ns = 1000000u;
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Arrival on a counter at GPU scope with release semantics (this thread's
// earlier writes, and those of threads ordered before it by a barrier, become
// visible to whoever acquires the counter) and acquire semantics (writes
// released by earlier arrivals become visible to this thread).
// arrive (release, CTA scope) on an mbarrier
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Order this thread's earlier generic-proxy shared-memory accesses before its
// later async-proxy (bulk copy) writes.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Global -> shared bulk copy of `bytes` (multiple of 16; both addresses
// 16-byte aligned) completing on `bar` (transaction bytes).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One RP-wide FP32 row (RP * 4 bytes, 16-byte aligned at both ends) copied by
// this thread with 16-byte cp.async (L2 only), and the arrival of this thread
// on an mbarrier once all its earlier cp.async have landed (noinc: the barrier's
// expected count includes one such arrival per thread).
__device__ __forceinline__ void cp_row(uint32_t dst, const float* src) {
#pragma unroll
  for (int c = 0; c < RP / 4; ++c)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * c), "l"(src + 4 * c) : "memory");
}
__device__ __forceinline__ void cp_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// L2 policy for data read exactly once (the packed payload): evict it first,
// so that the vectors the kernels gather from stay resident in L2.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// bulk_g2s with an L2 cache policy.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

}  // namespace hm
