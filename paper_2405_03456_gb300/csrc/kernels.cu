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

__device__ __forceinline__ int lanes_for(int rows) {
  int g = (rows + 3) >> 2;
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
  } else if constexpr (F == 2 && B <= 3) {                 // AFLP, s exact in FP32
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

template <int B>
__device__ __forceinline__ void load_words(const uint8_t* __restrict__ p, uint32_t (&w)[B]) {
  const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
#pragma unroll
  for (int i = 0; i < B; ++i) w[i] = __ldg(q + i);
}

// ---------------------------------------------------------------- column dots (phase A)
template <int TIER>
struct ColAcc {
  float s = 0.0f, c = 0.0f;
};

template <int TIER, int F, int B, int R>
__device__ __forceinline__ void cdot_col(const uint8_t* __restrict__ base, int G, int e, int m,
                                         const float (&xh)[R][4], const float (&xl)[R][4],
                                         const bool (&ok)[R][4], int q, ColAcc<TIER>& acc) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (!ok[r][0]) continue;          // whole group beyond the segment: no load
    uint32_t w[B];
    load_words<B>(base + (size_t)4 * B * (q + G * r), w);
    float h[4], l[4];
    decode4<TIER, F, B>(w, e, m, h, l);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float dh = ok[r][u] ? h[u] : 0.0f;
      if constexpr (TIER == TIER_F32) {
        acc.s = fmaf(dh, xh[r][u], acc.s);
      } else {
        float dl = ok[r][u] ? l[u] : 0.0f;
        dot2(acc.s, acc.c, dh, dl, xh[r][u], xl[r][u]);
      }
    }
  }
}

template <int TIER, int R>
__device__ __forceinline__ bool cdot_dispatch(uint32_t fw, const uint8_t* base, int G,
                                              const float (&xh)[R][4], const float (&xl)[R][4],
                                              const bool (&ok)[R][4], int q, ColAcc<TIER>& acc) {
  Fmt f = unpack_fmt(fw);
  switch ((f.f << 4) | f.B) {
#define HM_CASE(F, B) \
  case ((F) << 4) | (B): cdot_col<TIER, F, B, R>(base, G, f.e, f.m, xh, xl, ok, q, acc); return true;
    HM_CASE(0, 2) HM_CASE(0, 3) HM_CASE(0, 4)
    HM_CASE(1, 5) HM_CASE(1, 6) HM_CASE(1, 7) HM_CASE(1, 8)
    HM_CASE(2, 1) HM_CASE(2, 2) HM_CASE(2, 3) HM_CASE(2, 4) HM_CASE(2, 5) HM_CASE(2, 6) HM_CASE(2, 7)
    HM_CASE(3, 8)
#undef HM_CASE
    default: return false;
  }
}

// Width-exclusive prefix over the column slots of a warp (slots of G lanes each).
__device__ __forceinline__ uint32_t slot_prefix(uint32_t w, int G, int lane, uint32_t& total) {
  uint32_t v = w;
  for (int d = G; d < 32; d <<= 1) {
    uint32_t t = __shfl_up_sync(HM_FULL, v, d);
    if (lane >= d) v += t;
  }
  total = __shfl_sync(HM_FULL, v, 31);
  return v - w;
}

template <int TIER, int R>
__device__ void cdot_item(const CdotItem& I, const uint8_t* __restrict__ pay,
                          const uint32_t* __restrict__ fmts, const float2* __restrict__ vin,
                          double* __restrict__ partial, int lane, int* err) {
  const int G = I.seg >= 128 ? 32 : lanes_for(I.seg);
  const int slots = 32 / G;
  const int slot = lane / G, q = lane % G;
  float xh[R][4], xl[R][4];
  bool ok[R][4];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int rr = 4 * (q + G * r) + u;
      ok[r][u] = rr < I.seg;
      float2 v = ok[r][u] ? vin[I.vin + I.row0 + rr] : make_float2(0.f, 0.f);
      xh[r][u] = v.x;
      xl[r][u] = v.y;
    }
  const bool direct = I.fmt < 0;
  uint64_t coloff = I.off;
  for (int j0 = 0; j0 < I.ncols; j0 += slots) {
    const int j = j0 + slot;
    const bool active = j < I.ncols;
    uint32_t fw = direct ? fmts[~I.fmt] : fmts[I.fmt + (active ? j : j0)];
    uint32_t width = active ? pad4((uint32_t)I.nrows * (fw & 0xff)) : 0u;
    uint32_t total;
    uint32_t pre = slot_prefix(width, G, lane, total);
    ColAcc<TIER> acc;
    if (active && 4 * q < I.seg) {
      const uint8_t* base = pay + coloff + pre + (size_t)I.row0 * (fw & 0xff);
      if (!cdot_dispatch<TIER, R>(fw, base, G, xh, xl, ok, q, acc)) latch_error(err, 1);
    }
    coloff += total;
    // reduce over the G lanes of the slot
    for (int d = G >> 1; d > 0; d >>= 1) {
      float so = __shfl_xor_sync(HM_FULL, acc.s, d);
      float co = __shfl_xor_sync(HM_FULL, acc.c, d);
      if constexpr (TIER == TIER_F32) {
        acc.s += so;
      } else {
        float s, e;
        two_sum(acc.s, so, s, e);
        acc.s = s;
        acc.c += co + e;
      }
    }
    if (active && q == 0) partial[I.pout + j] = (double)acc.s + (double)acc.c;
  }
}

template <int TIER>
__global__ void __launch_bounds__(256) k_cdot(const CdotItem* __restrict__ items, int nitems,
                                              const uint8_t* __restrict__ pay,
                                              const uint32_t* __restrict__ fmts,
                                              const float2* __restrict__ vin,
                                              double* __restrict__ partial, int* err) {
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int it = wid; it < nitems; it += nw) {
    CdotItem I = items[it];
    const int G = I.seg >= 128 ? 32 : lanes_for(I.seg);
    const int R = (I.seg + 4 * G - 1) / (4 * G);
    if (R <= 1)
      cdot_item<TIER, 1>(I, pay, fmts, vin, partial, lane, err);
    else if (R <= 2)
      cdot_item<TIER, 2>(I, pay, fmts, vin, partial, lane, err);
    else
      cdot_item<TIER, 4>(I, pay, fmts, vin, partial, lane, err);
  }
}

// ---------------------------------------------------------------- segment sums (phase A2)
__global__ void k_gsum(const GsumOut* __restrict__ outs, int nouts, const int32_t* __restrict__ plist,
                       const double* __restrict__ pscale, const double* __restrict__ partial,
                       double alpha, float2* __restrict__ vout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nouts) return;
  GsumOut O = outs[i];
  double s = 0.0;
  for (int p = O.p0; p < O.p1; ++p) {
    double v = partial[plist[p]];
    s += pscale ? pscale[p] * v : v;
  }
  s *= O.scale;
  if (O.flags & 1) s *= alpha;
  FF f = ff_from_d(s);
  vout[O.out] = make_float2(f.hi, f.lo);
}

// ---------------------------------------------------------------- row chunks (phase C)
template <int TIER, int F, int B>
__device__ __forceinline__ void rg_col(const uint8_t* __restrict__ base, int e, int m, float2 v,
                                       float (&ps)[4], float (&pc)[4]) {
  uint32_t w[B];
  load_words<B>(base, w);
  float h[4], l[4];
  decode4<TIER, F, B>(w, e, m, h, l);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if constexpr (TIER == TIER_F32)
      ps[u] = fmaf(h[u], v.x, ps[u]);
    else
      dot2(ps[u], pc[u], h[u], l[u], v.x, v.y);
  }
}

template <int TIER>
__device__ __forceinline__ bool rg_dispatch(uint32_t fw, const uint8_t* base, float2 v, float (&ps)[4],
                                            float (&pc)[4]) {
  Fmt f = unpack_fmt(fw);
  switch ((f.f << 4) | f.B) {
#define HM_CASE(F, B) \
  case ((F) << 4) | (B): rg_col<TIER, F, B>(base, f.e, f.m, v, ps, pc); return true;
    HM_CASE(0, 2) HM_CASE(0, 3) HM_CASE(0, 4)
    HM_CASE(1, 5) HM_CASE(1, 6) HM_CASE(1, 7) HM_CASE(1, 8)
    HM_CASE(2, 1) HM_CASE(2, 2) HM_CASE(2, 3) HM_CASE(2, 4) HM_CASE(2, 5) HM_CASE(2, 6) HM_CASE(2, 7)
    HM_CASE(3, 8)
#undef HM_CASE
    default: return false;
  }
}

constexpr int RG_WARPS = 4;

template <int TIER, int MODE>
__global__ void __launch_bounds__(RG_WARPS * 32) k_rgemv(
    const Chunk* __restrict__ chunks, int nchunks, const Tile* __restrict__ tiles,
    const uint8_t* __restrict__ pay, const uint32_t* __restrict__ fmts,
    const float2* __restrict__ vin, double alpha, double beta, double* __restrict__ y,
    const int32_t* __restrict__ perm, float2* __restrict__ vout, const double* __restrict__ rowscale,
    int* err) {
  __shared__ float2 red[RG_WARPS][128];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  for (int ci = blockIdx.x; ci < nchunks; ci += gridDim.x) {
    const Chunk C = chunks[ci];
    const int G = lanes_for(C.nrows);
    const int slots = 32 / G;
    const int slot = lane / G, q = lane % G;
    const bool rows_ok = 4 * q < C.nrows;
    FF acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = {0.0f, 0.0f};
    for (int t = C.t0 + warp; t < C.t1; t += RG_WARPS) {
      const Tile T = tiles[t];
      float ps[4] = {0.f, 0.f, 0.f, 0.f}, pc[4] = {0.f, 0.f, 0.f, 0.f};
      const bool direct = T.fmt < 0;
      uint64_t coloff = T.off;
      for (int j0 = 0; j0 < T.ncols; j0 += slots) {
        const int j = j0 + slot;
        const bool active = j < T.ncols;
        uint32_t fw = direct ? fmts[~T.fmt] : fmts[T.fmt + (active ? j : j0)];
        uint32_t width = active ? pad4((uint32_t)C.nrows * (fw & 0xff)) : 0u;
        uint32_t total;
        uint32_t pre = slot_prefix(width, G, lane, total);
        if (active && rows_ok) {
          const float2 v = vin[T.vin + j];
          const uint8_t* base = pay + coloff + pre + (size_t)4 * q * (fw & 0xff);
          if (!rg_dispatch<TIER>(fw, base, v, ps, pc)) latch_error(err, 2);
        }
        coloff += total;
      }
      const double sc = (T.flags & 1) ? T.scale * alpha : T.scale;
      if constexpr (TIER == TIER_F32) {
        const float s = (float)sc;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float p = ps[u] * s;
          float pe = fmaf(ps[u], s, -p);
          acc[u] = ff_add(acc[u], FF{p, pe});
        }
      } else {
        const FF s = ff_from_d(sc);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float h = ps[u] + pc[u];
          FF p = {h, pc[u] - (h - ps[u])};
          acc[u] = ff_add(acc[u], ff_mul(p, s));
        }
      }
    }
    // reduce the column slots of this warp (lanes with equal q)
    for (int d = G; d < 32; d <<= 1) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        FF o;
        o.hi = __shfl_xor_sync(HM_FULL, acc[u].hi, d);
        o.lo = __shfl_xor_sync(HM_FULL, acc[u].lo, d);
        acc[u] = ff_add(acc[u], o);
      }
    }
    if (slot == 0 && rows_ok) {
#pragma unroll
      for (int u = 0; u < 4; ++u) red[warp][4 * q + u] = make_float2(acc[u].hi, acc[u].lo);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < C.nrows; r += blockDim.x) {
      FF s = {red[0][r].x, red[0][r].y};
#pragma unroll
      for (int w = 1; w < RG_WARPS; ++w) s = ff_add(s, FF{red[w][r].x, red[w][r].y});
      const int g = C.row0 + r;
      double v = ff_to_d(s);
      if constexpr (MODE == MODE_Y) {
        const int o = perm[g];
        y[o] = (beta == 0.0) ? v : fma(beta, y[o], v);
      } else {
        if constexpr (MODE == MODE_VEC_ADD) {
          float2 old = vout[g];
          v += (double)old.x + (double)old.y;
        }
        if (rowscale) v *= rowscale[g];
        if (C.flags & 1) v *= alpha;
        FF f = ff_from_d(v);
        vout[g] = make_float2(f.hi, f.lo);
      }
    }
    __syncthreads();
  }
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
cudaError_t launch_gather(const double* x, const int32_t* perm, int n, float2* xo, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<(n + 255) / 256, 256, 0, st>>>(x, perm, n, xo);
  return cudaGetLastError();
}

cudaError_t launch_cdot(int tier, const CdotItem* items, int nitems, const uint8_t* pay,
                        const uint32_t* fmts, const float2* vin, double* partial, int* err, int grid,
                        cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  int need = (nitems + 7) / 8;
  int g = need < grid ? need : grid;
  if (tier == TIER_F32)
    k_cdot<TIER_F32><<<g, 256, 0, st>>>(items, nitems, pay, fmts, vin, partial, err);
  else
    k_cdot<TIER_FF><<<g, 256, 0, st>>>(items, nitems, pay, fmts, vin, partial, err);
  return cudaGetLastError();
}

cudaError_t launch_gsum(const GsumOut* outs, int nouts, const int32_t* plist, const double* pscale,
                        const double* partial, double alpha, float2* vout, cudaStream_t st) {
  if (nouts <= 0) return cudaSuccess;
  k_gsum<<<(nouts + 255) / 256, 256, 0, st>>>(outs, nouts, plist, pscale, partial, alpha, vout);
  return cudaGetLastError();
}

cudaError_t launch_rgemv(int tier, int mode, const Chunk* chunks, int nchunks, const Tile* tiles,
                         const uint8_t* pay, const uint32_t* fmts, const float2* vin, double alpha,
                         double beta, double* y, const int32_t* perm, float2* vout,
                         const double* rowscale, int* err, int grid, cudaStream_t st) {
  if (nchunks <= 0) return cudaSuccess;
  int g = nchunks < grid ? nchunks : grid;
#define HM_RG(T, M)                                                                                  \
  k_rgemv<T, M><<<g, RG_WARPS * 32, 0, st>>>(chunks, nchunks, tiles, pay, fmts, vin, alpha, beta, y, \
                                             perm, vout, rowscale, err)
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
