// sm_103a kernels of libhm: on-the-fly decompression (Sec. 4.1, Alg. 8) fused
// into the column-dot and row-chunk products of the H / UH / H^2 matvec (Sec. 3).
//
// Arithmetic (GB300 runs FP64 FMA at 1/60 of the FP32 rate):
//  * every packed value is decoded to FP32 with integer operations; AFLP
//    values are decoded as +-(s - 1), their per-array vmin being folded into
//    the coefficient vectors or tile scales;
//  * TIER_F32 (eps > 2^-22): one FP32 value per entry, FP32 products summed
//    per column (or per tile), sums carried in float-float (hi, lo);
//  * TIER_FF (eps <= 2^-22 and the uncompressed baseline): entries and vector
//    values as float-float pairs, products accumulated with the compensated
//    dot product of Ogita, Rump and Oishi (2005, "Dot2": TwoProduct by FMA,
//    TwoSum of Knuth), about 2^-46 relative;
//  * vectors are float2 (hi, lo) pairs; y is FP64.
// Race freedom (Sec. 3.1, Alg. 3): every output row belongs to exactly one
// chunk and every chunk to one thread block, so there are no atomics and the
// result is bitwise reproducible.
#include <cstdint>
#include <cuda_runtime.h>

#include "dev_types.h"

namespace hm {

#define HM_FULL 0xffffffffu

// lanes (a power of two, <= 32) that hold 8 rows each of a column of `rows`
__device__ __forceinline__ int lanes_for_rpl(int rows) {
  int g = (rows + 7) >> 3;
  int p = 1;
  while (p < g) p <<= 1;
  return p > 32 ? 32 : p;
}

__device__ __forceinline__ uint32_t pad4(uint32_t x) { return (x + 3u) & ~3u; }

__device__ __forceinline__ void latch_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------- float-float helpers
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

struct Fmt {
  int B, f, e, m;
};

__device__ __forceinline__ Fmt unpack_fmt(uint32_t w) {
  return {(int)(w & 0xff), (int)((w >> 8) & 0xff), (int)((w >> 16) & 0xff), (int)(w >> 24)};
}

// FP64 bit pattern -> float-float (hi truncated to 24 bits, lo the rest).
template <int TIER>
__device__ __forceinline__ void split_f64bits(uint64_t P, float& hi, float& lo) {
  uint32_t sgn = (uint32_t)(P >> 32) & 0x80000000u;
  int E = (int)((P >> 52) & 0x7ff);
  uint64_t M = P & ((1ull << 52) - 1);
  uint32_t hb = (E >= 897) ? (((uint32_t)(E - 896) << 23) | (uint32_t)(M >> 29)) : 0u;
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

// Decode 4 consecutive values of format (F, B) into hi (and lo for TIER_FF).
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
  } else if constexpr (F == 2 && (B <= 3 || (B == 4 && TIER == TIER_F32))) {
    // AFLP with s in FP32 (exact for B <= 3; for B = 4 the mantissa is cut to
    // 23 bits, which is the F32 tier's own precision)
    constexpr uint32_t mask = (0xffffffffu << (8 * (4 - B))) & 0x7fffffffu;
    const int sh = 8 - e;
    uint32_t t[4] = {top32<B, 0>(w), top32<B, 1>(w), top32<B, 2>(w), top32<B, 3>(w)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t sb = ((t[i] & mask) >> sh) + (127u << 23);
      float d = __uint_as_float(sb) - 1.0f;
      h[i] = __uint_as_float(__float_as_uint(d) ^ (t[i] & 0x80000000u));
    }
  } else if constexpr (F == 2) {                           // AFLP with m' > 23
    uint64_t c[4];
    if constexpr (B == 4) {
      c[0] = w[0]; c[1] = w[1]; c[2] = w[2]; c[3] = w[3];
    } else {
      constexpr int rs = 64 - 8 * B;
      c[0] = top64<B, 0>(w) >> rs;
      c[1] = top64<B, 1>(w) >> rs;
      c[2] = top64<B, 2>(w) >> rs;
      c[3] = top64<B, 3>(w) >> rs;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t sgn = (uint32_t)(c[i] >> (8 * B - 1)) << 31;
      uint32_t f = (uint32_t)(c[i] >> m) & ((1u << e) - 1u);
      uint64_t mant = c[i] & ((1ull << m) - 1ull);
      uint32_t hb = ((f + 127u) << 23) | (uint32_t)(mant >> (m - 23));
      float d = __uint_as_float(hb) - 1.0f;
      h[i] = __uint_as_float(__float_as_uint(d) ^ sgn);
      if constexpr (TIER == TIER_FF) {
        uint64_t ml = mant & ((1ull << (m - 23)) - 1ull);
        float lv = __ull2float_rn(ml) * __uint_as_float((uint32_t)(f + 127 - m) << 23);
        l[i] = __uint_as_float(__float_as_uint(lv) ^ sgn);
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


// ---------------------------------------------------------------- loads and 8-value decode
// A lane decodes 8 consecutive values of one column: 2B 32-bit words read as B
// streaming 64-bit loads (the column and the lane's offset 8*q*B are 8-byte
// aligned); the payload is read once, so it is loaded with the evict-first hint.
template <int B>
__device__ __forceinline__ void ld8(const uint8_t* __restrict__ p, uint32_t (&w0)[B], uint32_t (&w1)[B]) {
  const uint2* q = reinterpret_cast<const uint2*>(p);
  uint32_t w[2 * B];
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const uint2 t = __ldcs(q + i);
    w[2 * i] = t.x;
    w[2 * i + 1] = t.y;
  }
#pragma unroll
  for (int i = 0; i < B; ++i) {
    w0[i] = w[i];
    w1[i] = w[B + i];
  }
}

template <int TIER, int F, int B>
__device__ __forceinline__ void decode8(const uint8_t* __restrict__ p, int e, int m, float (&h)[8], float (&l)[8]) {
  uint32_t w0[B], w1[B];
  ld8<B>(p, w0, w1);
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

__device__ __forceinline__ uint32_t pad8(uint32_t x) { return (x + 7u) & ~7u; }

// Visit (F, B) as template arguments; false for an unknown format word.
#define HM_FORMATS(X) \
  X(0, 2) X(0, 3) X(0, 4) X(1, 5) X(1, 6) X(1, 7) X(1, 8) \
  X(2, 1) X(2, 2) X(2, 3) X(2, 4) X(2, 5) X(2, 6) X(2, 7) X(3, 8)

// ---------------------------------------------------------------- prefetched columns
// A lane's 8 codes of a column occupy 8*B bytes = B words of 64 bits.  The
// fetch is format-blind: W such words (W = 4 covers B <= 4, the F32 tier;
// W = 8 covers every width) are loaded for the next column while the current one is decoded, so
// two columns' loads are in flight per lane with a single decode path.  The
// extra bytes of a short code belong to the neighbouring lane's rows and are
// fetched by the same coalesced request.
template <int W>
struct Words {
  uint2 w[W];
};

template <int W>
__device__ __forceinline__ void fetch(const uint8_t* __restrict__ p, Words<W>& out) {
  const uint2* q = reinterpret_cast<const uint2*>(p);
#pragma unroll
  for (int i = 0; i < W; ++i) out.w[i] = __ldcs(q + i);
}

// decode the 8 codes (format F, width B <= W: 8*B bytes = B 64-bit words) held in `in`
template <int TIER, int F, int B, int W>
__device__ __forceinline__ void decode8w(const Words<W>& in, int e, int m, float (&h)[8], float (&l)[8]) {
  static_assert(B <= W, "fetch window too small");
  uint32_t w[2 * W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    w[2 * i] = in.w[i].x;
    w[2 * i + 1] = in.w[i].y;
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

// Dispatch on the format word; formats wider than the window are decoded from
// a direct reload at p.  Returns false for an unknown word.
template <int TIER, int W>
__device__ __forceinline__ bool decode_any(uint32_t fw, const Words<W>& in, const uint8_t* __restrict__ p,
                                           float (&h)[8], float (&l)[8]) {
  const Fmt f = unpack_fmt(fw);
#define HM_DW(F, B)                                \
  case ((F) << 4) | (B):                           \
    if constexpr ((B) <= W) {                      \
      decode8w<TIER, F, B, W>(in, f.e, f.m, h, l); \
    } else {                                       \
      Words<(B)> big;                              \
      fetch(p, big);                               \
      decode8w<TIER, F, B, (B)>(big, f.e, f.m, h, l); \
    }                                              \
    return true;
  switch ((f.f << 4) | f.B) {
    HM_FORMATS(HM_DW)
    default:
      return false;
  }
#undef HM_DW
}

// ---------------------------------------------------------------- column dots (phase A)
// One warp per item (a segment of <= 128 rows of a column set).  G lanes (a
// power of two) hold 8 rows each of a column, S = 32/G columns are processed
// side by side, and each column's sum is reduced over its G lanes.  Column
// offsets come from a warp prefix scan of the widths pad8(nrows * B_j), 32
// columns at a time.
template <int TIER>
__device__ __forceinline__ void lane_reduce(float& s, float& c, int G) {
  for (int d = G >> 1; d > 0; d >>= 1) {
    if constexpr (TIER == TIER_F32) {
      s += __shfl_xor_sync(HM_FULL, s, d);
    } else {
      const float so = __shfl_xor_sync(HM_FULL, s, d);
      const float co = __shfl_xor_sync(HM_FULL, c, d);
      float t, ee;
      two_sum(s, so, t, ee);
      s = t;
      c += co + ee;
    }
  }
}

__device__ __forceinline__ void cdot_out(const Item& I, int j, float s, float c, const F2* __restrict__ cscale,
                                         F2 alpha, F2* __restrict__ partial, float2* __restrict__ vout) {
  const float h = s + c;
  FF v = {h, c - (h - s)};
  if (I.flags & ITEM_FINAL) {
    const F2 sc = cscale[I.fmt + j];
    v = ff_mul(v, FF{sc.hi, sc.lo});
    if (I.flags & ITEM_ALPHA) v = ff_mul(v, FF{alpha.hi, alpha.lo});
    vout[I.out + j] = make_float2(v.hi, v.lo);
  } else {
    partial[I.out + j] = F2{v.hi, v.lo};
  }
}

template <int TIER, int W>
__global__ void __launch_bounds__(256, (TIER == TIER_F32) ? 4 : 2) k_cdot(const Item* __restrict__ items, int nitems,
                                              const uint8_t* __restrict__ pay,
                                              const uint32_t* __restrict__ fmts,
                                              const F2* __restrict__ cscale, const float2* __restrict__ vin,
                                              F2 alpha, F2* __restrict__ partial,
                                              float2* __restrict__ vout, int* err) {
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int it = wid; it < nitems; it += nw) {
    const Item I = items[it];
    const int G = lanes_for_rpl(I.nrows);
    const int S = 32 / G;
    const int slot = lane / G, q = lane % G;
    float xh[8], xl[8];
    bool ok[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int r = RPL * q + u;
      ok[u] = r < I.nrows;
      const float2 v = ok[u] ? vin[I.vin + r] : make_float2(0.f, 0.f);
      xh[u] = v.x;
      xl[u] = v.y;
    }
    const uint8_t* base = pay + I.off;
    uint32_t run = 0;                                 // bytes of the columns before this group of 32
    for (int g0 = 0; g0 < I.ncols; g0 += 32) {
      const int gj = g0 + lane;
      const uint32_t fwl = gj < I.ncols ? fmts[I.fmt + gj] : 0u;
      const uint32_t wl = gj < I.ncols ? pad8((uint32_t)I.nrows * (fwl & 0xff)) : 0u;
      uint32_t inc = wl;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(HM_FULL, inc, d);
        if (lane >= d) inc += t;
      }
      const uint32_t exl = inc - wl;
      const uint32_t gtot = __shfl_sync(HM_FULL, inc, 31);
      const int gn = min(32, I.ncols - g0);
      // software pipeline over this slot's columns k = slot, slot + S, ...
      int k = slot;
      uint32_t fw = __shfl_sync(HM_FULL, fwl, k < gn ? k : 0);
      uint32_t off = __shfl_sync(HM_FULL, exl, k < gn ? k : 0);
      const uint8_t* p = base + run + off + (size_t)RPL * q * (fw & 0xff);
      Words<W> cur;
      if (k < gn && ok[0]) fetch(p, cur);
      for (int k0 = 0; k0 < gn; k0 += S) {
        const int kn = k + S;
        const uint32_t fwn = __shfl_sync(HM_FULL, fwl, kn < gn ? kn : 0);
        const uint32_t offn = __shfl_sync(HM_FULL, exl, kn < gn ? kn : 0);
        const uint8_t* pn = base + run + offn + (size_t)RPL * q * (fwn & 0xff);
        Words<W> nxt;
        if (kn < gn && ok[0]) fetch(pn, nxt);
        float s = 0.f, c = 0.f;
        if (k < gn && ok[0]) {
          float h[8], l[8];
          if (!decode_any<TIER, W>(fw, cur, p, h, l)) latch_error(err, 1);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float dh = ok[u] ? h[u] : 0.0f;
            if constexpr (TIER == TIER_F32) {
              s = fmaf(dh, xh[u], s);
            } else {
              const float dl = ok[u] ? l[u] : 0.0f;
              dot2(s, c, dh, dl, xh[u], xl[u]);
            }
          }
        }
        lane_reduce<TIER>(s, c, G);
        if (q == 0 && k < gn) cdot_out(I, g0 + k, s, c, cscale, alpha, partial, vout);
        k = kn;
        fw = fwn;
        p = pn;
        cur = nxt;
      }
      run += gtot;
    }
  }
}

// ---------------------------------------------------------------- row chunks (phase C)
constexpr int RG_WARPS = 4;
constexpr int RG_BATCH = 256;      // merged columns staged in shared memory per batch

// s/c: FP32 partial sums of the lane's 8 rows (F32) or Dot2 pairs (FF)
template <int TIER, int F, int B>
__device__ __forceinline__ void rg_col8(const uint8_t* __restrict__ p, int e, int m, float vh, float vl,
                                        float (&s)[8], float (&c)[8]) {
  float h[8], l[8];
  decode8<TIER, F, B>(p, e, m, h, l);
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if constexpr (TIER == TIER_F32)
      s[u] = fmaf(h[u], vh, s[u]);
    else
      dot2(s[u], c[u], h[u], l[u], vh, vl);
  }
}

// multiplier of a column: v * scale (scale = vmin, times alpha if asked)
template <int TIER>
__device__ __forceinline__ void scaled(float2 v, FF sc, float& vh, float& vl) {
  if constexpr (TIER == TIER_F32) {
    vh = v.x * sc.hi;
    vl = 0.f;
  } else {
    const FF r = ff_mul(FF{v.x, v.y}, sc);
    vh = r.hi;
    vl = r.lo;
  }
}

// fold the FP32 / Dot2 partials into the float-float row sums and clear them
template <int TIER>
__device__ __forceinline__ void rg_flush(FF (&acc)[8], float (&s)[8], float (&c)[8]) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if constexpr (TIER == TIER_F32) {
      acc[u] = ff_add_f(acc[u], s[u]);
    } else {
      const float h = s[u] + c[u];
      acc[u] = ff_add(acc[u], FF{h, c[u] - (h - s[u])});
    }
    s[u] = 0.f;
    c[u] = 0.f;
  }
}

// columns [j0, j1) of a uniform tile (format F, B) for the lane's 8 rows
template <int TIER, int F, int B>
__device__ __forceinline__ void rg_tile(const uint8_t* __restrict__ p0, uint32_t stride, int j0, int j1,
                                        const float2* __restrict__ v, FF sc, int e, int m, float (&s)[8],
                                        float (&c)[8]) {
#pragma unroll 2
  for (int j = j0; j < j1; ++j) {
    float vh, vl;
    scaled<TIER>(v[j], sc, vh, vl);
    rg_col8<TIER, F, B>(p0 + (size_t)j * stride, e, m, vh, vl, s, c);
  }
}

template <int TIER, int MODE>
__global__ void __launch_bounds__(RG_WARPS * 32) k_rgemv(
    const Chunk* __restrict__ chunks, int nchunks, const Tile* __restrict__ tiles,
    const ColMeta* __restrict__ cols, const uint8_t* __restrict__ pay, const float2* __restrict__ vin,
    double alpha, F2 alpha_ff, double beta, double* __restrict__ y, const int32_t* __restrict__ perm,
    float2* __restrict__ vout, const double* __restrict__ rowscale, int* err) {
  __shared__ float2 red[RG_WARPS * 32 * RPL];
  __shared__ uint32_t s_off[RG_BATCH];
  __shared__ uint32_t s_fw[RG_BATCH];
  __shared__ float2 s_v[RG_BATCH];
  __shared__ uint32_t s_wsum[RG_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int ci = blockIdx.x; ci < nchunks; ci += gridDim.x) {
    const Chunk C = chunks[ci];
    uint64_t coff = C.coff;
    const int R = C.nrows;
    const int G = (R + RPL - 1) / RPL;          // lanes per column (any count)
    const int S = 32 / G;                        // column slots per warp
    const int slot = lane / G, q = lane % G;
    const bool lane_on = slot < S && RPL * q < R;
    FF acc[8];
    float s[8], c[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      acc[u] = {0.f, 0.f};
      s[u] = 0.f;
      c[u] = 0.f;
    }
    // uniform tiles (dense blocks, couplings, transfers): warps round-robin, slots split the columns
    for (int t = C.t0 + warp; t < C.t1; t += RG_WARPS) {
      const Tile T = tiles[t];
      if (!lane_on) continue;
      const Fmt f = unpack_fmt(T.fw);
      const uint32_t stride = pad8((uint32_t)R * f.B);
      const int j0 = (slot * T.ncols) / S, j1 = ((slot + 1) * T.ncols) / S;
      const FF sc = (T.flags & 1) ? ff_mul(FF{T.scale.hi, T.scale.lo}, FF{alpha_ff.hi, alpha_ff.lo})
                                  : FF{T.scale.hi, T.scale.lo};
      const uint8_t* p0 = pay + T.off + (size_t)RPL * q * f.B;
      switch ((f.f << 4) | f.B) {
#define HM_RT(F, B)                                                                              \
  case ((F) << 4) | (B):                                                                         \
    rg_tile<TIER, F, B>(p0, stride, j0, j1, vin + T.vin, sc, f.e, f.m, s, c); break;
        HM_FORMATS(HM_RT)
#undef HM_RT
        default:
          latch_error(err, 2);
      }
      rg_flush<TIER>(acc, s, c);
    }
    // merged VALR columns, staged in batches: format words, multipliers, offsets
    for (int b0 = C.c0; b0 < C.c1; b0 += RG_BATCH) {
      const int nb = min(RG_BATCH, C.c1 - b0);
      __syncthreads();
      uint32_t wv[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int i = threadIdx.x * 2 + k;
        wv[k] = 0u;
        if (i < nb) {
          const ColMeta cm = cols[b0 + i];
          s_fw[i] = cm.fw;
          s_v[i] = vin[cm.vin];
          wv[k] = pad8((uint32_t)R * (cm.fw & 0xff));
        }
      }
      // exclusive scan of the widths (2 per thread) over the block
      uint32_t tsum = wv[0] + wv[1];
      uint32_t inc = tsum;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(HM_FULL, inc, d);
        if (lane >= d) inc += t;
      }
      if (lane == 31) s_wsum[warp] = inc;
      __syncthreads();
      uint32_t wbase = 0;
      for (int w = 0; w < warp; ++w) wbase += s_wsum[w];
      const uint32_t ex = wbase + inc - tsum;
      if (threadIdx.x * 2 < nb) s_off[threadIdx.x * 2] = ex;
      if (threadIdx.x * 2 + 1 < nb) s_off[threadIdx.x * 2 + 1] = ex + wv[0];
      uint32_t btot = 0;
      for (int w = 0; w < RG_WARPS; ++w) btot += s_wsum[w];
      __syncthreads();
      if (lane_on) {
        // column i -> warp (i / S) % RG_WARPS, slot i % S: neighbouring columns share a format
        for (int i = warp * S + slot; i < nb; i += RG_WARPS * S) {
          const uint32_t fw = s_fw[i];
          const Fmt f = unpack_fmt(fw);
          const float2 v = s_v[i];
          const uint8_t* p = pay + coff + s_off[i] + (size_t)RPL * q * f.B;
          switch ((f.f << 4) | f.B) {
#define HM_RC(F, B)                                                                     \
  case ((F) << 4) | (B): rg_col8<TIER, F, B>(p, f.e, f.m, v.x, v.y, s, c); break;
            HM_FORMATS(HM_RC)
#undef HM_RC
            default:
              latch_error(err, 3);
          }
        }
        rg_flush<TIER>(acc, s, c);
      }
      coff += btot;
    }
    // reduce over slots and warps in shared memory (fixed order)
    if (lane_on) {
#pragma unroll
      for (int u = 0; u < 8; ++u) red[(warp * 32 + lane) * RPL + u] = make_float2(acc[u].hi, acc[u].lo);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      const int qq = r / RPL, u = r % RPL;
      FF t = {0.f, 0.f};
      for (int w = 0; w < RG_WARPS; ++w)
        for (int sl = 0; sl < S; ++sl) {
          const float2 v = red[(w * 32 + sl * G + qq) * RPL + u];
          t = ff_add(t, FF{v.x, v.y});
        }
      const int g = C.row0 + r;
      double val = ff_to_d(t);
      if constexpr (MODE == MODE_Y) {
        const int o = perm[g];
        y[o] = (beta == 0.0) ? val : fma(beta, y[o], val);
      } else {
        if constexpr (MODE == MODE_VEC_ADD) {
          const float2 old = vout[g];
          val += (double)old.x + (double)old.y;
        }
        if (rowscale) val *= rowscale[g];
        if (C.flags & 1) val *= alpha;
        const FF ff = ff_from_d(val);
        vout[g] = make_float2(ff.hi, ff.lo);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- segment sums (phase A2)
__global__ void k_gsum(const GsumOut* __restrict__ outs, int nouts, const int32_t* __restrict__ plist,
                       const F2* __restrict__ pscale, const F2* __restrict__ partial, F2 alpha,
                       float2* __restrict__ vout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nouts) return;
  const GsumOut O = outs[i];
  FF s = {0.f, 0.f};
  for (int p = O.p0; p < O.p1; ++p) {
    const F2 v = partial[plist[p]];
    const F2 w = pscale[p];
    s = ff_add(s, ff_mul(FF{v.hi, v.lo}, FF{w.hi, w.lo}));
  }
  s = ff_mul(s, FF{O.scale.hi, O.scale.lo});
  if (O.flags & 1) s = ff_mul(s, FF{alpha.hi, alpha.lo});
  vout[O.out] = make_float2(s.hi, s.lo);
}

// ---------------------------------------------------------------- gather x
__global__ void k_gather(const double* __restrict__ x, const int32_t* __restrict__ perm, int n,
                         float2* __restrict__ xo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  FF f = ff_from_d(x[perm[i]]);
  xo[i] = make_float2(f.hi, f.lo);
}

// ---------------------------------------------------------------- K0: bit-exact decode to FP64
__global__ void k_decode(const uint8_t* __restrict__ p, int64_t n, int B, int fmt, int e, int m,
                         double vmin, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t c = 0;
  for (int b = 0; b < B; ++b) c |= (uint64_t)p[i * B + b] << (8 * b);
  double v;
  if (fmt == 3) {
    v = __longlong_as_double((long long)c);
  } else if (fmt == 1) {
    v = __longlong_as_double((long long)(c << (64 - 8 * B)));
  } else if (fmt == 0) {
    v = (double)__uint_as_float((uint32_t)(c << (32 - 8 * B)));
  } else {
    uint64_t sg = (c >> (8 * B - 1)) & 1ull;
    uint64_t f = (c >> m) & ((1ull << e) - 1ull);
    uint64_t mant = c & ((1ull << m) - 1ull);
    v = 0.0;
    if (f != 0) {
      double s = __longlong_as_double((long long)(((f + 1023ull) << 52) | (mant << (52 - m))));
      v = __dmul_rn(__dsub_rn(s, 1.0), vmin);
    }
    if (sg) v = -v;
  }
  out[i] = v;
}

// ---------------------------------------------------------------- launchers
cudaError_t kernels_init() { return cudaSuccess; }

cudaError_t launch_gather(const double* x, const int32_t* perm, int n, float2* xo, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<(n + 255) / 256, 256, 0, st>>>(x, perm, n, xo);
  return cudaGetLastError();
}

cudaError_t launch_cdot(int tier, const Item* items, int nitems, const uint8_t* pay, const uint32_t* fmts,
                        const F2* cscale, const float2* vin, F2 alpha, F2* partial, float2* vout, int* err,
                        int grid, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  const int need = (nitems + 7) / 8;
  const int g = need < grid ? need : grid;
  if (tier == TIER_F32)
    k_cdot<TIER_F32, 4><<<g, 256, 0, st>>>(items, nitems, pay, fmts, cscale, vin, alpha, partial, vout, err);
  else
    k_cdot<TIER_FF, 8><<<g, 256, 0, st>>>(items, nitems, pay, fmts, cscale, vin, alpha, partial, vout, err);
  return cudaGetLastError();
}

cudaError_t launch_gsum(const GsumOut* outs, int nouts, const int32_t* plist, const F2* pscale, const F2* partial,
                        F2 alpha, float2* vout, cudaStream_t st) {
  if (nouts <= 0) return cudaSuccess;
  k_gsum<<<(nouts + 255) / 256, 256, 0, st>>>(outs, nouts, plist, pscale, partial, alpha, vout);
  return cudaGetLastError();
}

cudaError_t launch_rgemv(int tier, int mode, const Chunk* chunks, int nchunks, const Tile* tiles,
                         const ColMeta* cols, const uint8_t* pay, const float2* vin, double alpha, F2 alpha_ff,
                         double beta, double* y, const int32_t* perm, float2* vout, const double* rowscale,
                         int* err, cudaStream_t st) {
  if (nchunks <= 0) return cudaSuccess;
#define HM_RG(T, M)                                                                                    \
  k_rgemv<T, M><<<nchunks, RG_WARPS * 32, 0, st>>>(chunks, nchunks, tiles, cols, pay, vin, alpha, alpha_ff, beta, \
                                                   y, perm, vout, rowscale, err)
  if (tier == TIER_F32) {
    if (mode == MODE_Y) HM_RG(TIER_F32, MODE_Y);
    else if (mode == MODE_VEC) HM_RG(TIER_F32, MODE_VEC);
    else HM_RG(TIER_F32, MODE_VEC_ADD);
  } else {
    if (mode == MODE_Y) HM_RG(TIER_FF, MODE_Y);
    else if (mode == MODE_VEC) HM_RG(TIER_FF, MODE_VEC);
    else HM_RG(TIER_FF, MODE_VEC_ADD);
  }
#undef HM_RG
  return cudaGetLastError();
}

cudaError_t launch_decode(const uint8_t* p, int64_t n, int B, int fmt, int e, int m, double vmin,
                          double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_decode<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, n, B, fmt, e, m, vmin, out);
  return cudaGetLastError();
}

}  // namespace hm
