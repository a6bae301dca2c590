// Multi-RHS products on the FP32 pipes (the precision / multi-RHS form, FP32
// tier): y := alpha*M*X + beta*y for panels of up to RP right-hand sides, one
// FP32 FMA per product as in the single-RHS kernels (the tensor-core engine is
// mrhs_tc.cu).  The matrix is streamed once per panel; the vectors are
// RP-wide rows v[entry * RP + k].
//  * k_gather_mr: x to cluster order, FP32;
//  * k_cdot_ws: column dots, one warp per range of pieces;
//  * k_gsum_mr: segment sums of the column-dot partials, float-float;
//  * k_rgemv_ms: row chunks, two warps (a pair) per range of pieces, each warp
//    32 rows of a chunk, sums per piece in FP32 and across pieces in
//    float-float; chunks are at most MP_ROWS rows (wider ones run on the
//    tensor-core kernel).
#include <cstdint>
#include <cuda_runtime.h>

#include "decode.cuh"

namespace hm {

__device__ __forceinline__ uint32_t pad16m(uint32_t x) { return (x + 15u) & ~15u; }

// ---------------------------------------------------------------- gather, segment sums
// v[i * RP + k] = x[perm[i] + k * ldx] (FP32 hi part), k < r; zero for k >= r.
__global__ void k_gather_mr(const double* __restrict__ x, int64_t ldx, int r, const int32_t* __restrict__ perm, int n,
                            float* __restrict__ v) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * RP) return;
  const int i = (int)(t / RP), k = (int)(t % RP);
  v[t] = k < r ? (float)x[(int64_t)perm[i] + k * ldx] : 0.0f;
}

__global__ void k_gsum_mr(const GsumOut* __restrict__ outs, int nouts, const F2* __restrict__ pscale,
                          const float* __restrict__ partial, F2 alpha, float* __restrict__ v) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nouts * RP) return;
  const GsumOut O = outs[t / RP];
  const int k = (int)(t % RP);
  const bool ws = (O.flags & 2) != 0;
  FF s = {0.f, 0.f};
  // partials in order p0, p0 + 1, ...; four loads in flight per step
  int p = O.p0;
  for (; p + 4 <= O.p1; p += 4) {
    float x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = __ldcs(partial + (int64_t)(p + u) * RP + k);
    if (ws) {
      F2 wv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) wv[u] = pscale[O.ps + (p + u - O.p0)];
#pragma unroll
      for (int u = 0; u < 4; ++u) s = ff_add(s, ff_mul(FF{x[u], 0.f}, FF{wv[u].hi, wv[u].lo}));
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) s = ff_add_f(s, x[u]);
    }
  }
  for (; p < O.p1; ++p) {
    const float x = __ldcs(partial + (int64_t)p * RP + k);
    if (ws) {
      const F2 w = pscale[O.ps + (p - O.p0)];
      s = ff_add(s, ff_mul(FF{x, 0.f}, FF{w.hi, w.lo}));
    } else {
      s = ff_add_f(s, x);
    }
  }
  s = ff_mul(s, FF{O.scale.hi, O.scale.lo});
  if (O.flags & 1) s = ff_mul(s, FF{alpha.hi, alpha.lo});
  v[(int64_t)O.out * RP + k] = s.hi + s.lo;
}

// ---------------------------------------------------------------- row chunks
// A pair of warps owns a range of pieces and a ring of MP_NS stages (piece +
// its multiplier rows, filled by the pair's warp 0: the piece by one bulk copy,
// each multiplier row -- the RP values of the coefficient it stands for -- by
// 16-byte cp.async); warp wi of the pair takes rows 32 wi .. 32 wi + 31 of every
// piece and all RP right-hand sides.  Lane (g = lane / 4, tq = lane % 4) holds
// rows 32 wi + 4 g .. + 3 and right-hand sides 8 nt + 2 tq + {0, 1}, nt < NT.
constexpr int NT = RP / 8;
constexpr int MP_NS = 3;                                   // stages per pair
constexpr int MP_TP = RP * 4 + 16;                         // multiplier row pitch in a stage (bytes)
constexpr int MP_STAGE = STAGE_BYTES + PIECE_MAX_COLS * MP_TP;
constexpr int MP_THREADS = MP_PAIRS * 64;
constexpr size_t MP_SMEM = (size_t)MP_PAIRS * MP_NS * MP_STAGE + (size_t)MP_PAIRS * MP_NS * 8;
static_assert(MP_STAGE % 128 == 0, "stage alignment");
static_assert(MP_SMEM <= 227 * 1024, "row-chunk pairs per block");

// Named barrier of the 64 threads of pair bid - 1 / its OR vote.
__device__ __forceinline__ void pair_sync(int bid) { asm volatile("bar.sync %0, 64;" ::"r"(bid) : "memory"); }
__device__ __forceinline__ bool pair_any(int bid, bool v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, %2, 64, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((int)v), "r"(bid)
      : "memory");
  return r != 0;
}

// One piece for warp wi of the pair on the FP32 pipes: every product is one
// FP32 FMA (FFMA2 over right-hand-side pairs), as in the single-RHS kernels,
// summed per piece in FP32 and folded into the float-float sums fhi / flo
// [mt][nt][h] of rows 32 wi + 4 g + 2 mt + h, right-hand sides 8 nt + 2 tq +
// {0, 1}.  Per column the lane decodes its 4 codes and reads its 8 multipliers.
template <int F, int B>
__device__ __forceinline__ void ms_piece(uint32_t sa, const PieceHdr& H, F2 alpha_ff, int wi, int lane,
                                         float2 (&fhi)[2][NT][2], float2 (&flo)[2][NT][2]) {
  const int R = H.nrows, nc = H.ncols;
  const bool tile = (H.flags & PH_TILE) != 0;
  const uint32_t stride = pad8u((uint32_t)R * B);
  const uint32_t cm = sa + (uint32_t)sizeof(PieceHdr);
  const int g = lane >> 2, tq = lane & 3;
  const uint32_t cb = cm + (tile ? 0u : pad8u(2u * nc)) + (uint32_t)((32 * wi + 4 * g) * B);
  const uint32_t tv = sa + STAGE_BYTES + 8u * tq;
  const int e_t = H.em & 0xff, m_t = H.em >> 8;
  float2 acc[4][NT];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) acc[u][nt] = make_float2(0.f, 0.f);
#pragma unroll 2
  for (int j = 0; j < nc; ++j) {
    int e = e_t, m = m_t;
    if constexpr (F == 2) {
      if (!tile) {
        const uint32_t em = lds32((cm + 2u * j) & ~3u) >> (16u * (j & 1));
        e = em & 0xff;
        m = (em >> 8) & 0xff;
      }
    }
    uint32_t w[B];
#pragma unroll
    for (int b = 0; b < B; ++b) w[b] = lds32(cb + (uint32_t)j * stride + 4u * b);
    float v[4], l[4];
    decode4<TIER_F32, F, B>(w, e, m, v, l);
    float2 t[NT];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const uint2 q = lds64(tv + (uint32_t)j * MP_TP + 32u * nt);
      t[nt] = make_float2(__uint_as_float(q.x), __uint_as_float(q.y));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 vv = make_float2(v[u], v[u]);
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) acc[u][nt] = __ffma2_rn(vv, t[nt], acc[u][nt]);
    }
  }
  float2 sc2 = make_float2(1.f, 1.f);
  if (tile) {
    FF f = {H.scale.hi, H.scale.lo};
    if (H.flags & PH_TALPHA) f = ff_mul(f, FF{alpha_ff.hi, alpha_ff.lo});
    sc2 = make_float2(f.hi, f.hi);
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
        ff_add_f2(fhi[mt][nt][h], flo[mt][nt][h], tile ? __fmul2_rn(acc[2 * mt + h][nt], sc2) : acc[2 * mt + h][nt]);
}

template <int MODE>
__global__ void __launch_bounds__(MP_THREADS, 1)
    k_rgemv_ms(const PieceCopy* __restrict__ cps, const int32_t* __restrict__ wbeg, int nrange,
               const uint8_t* __restrict__ pay, const float* __restrict__ vec, double alpha, F2 alpha_ff,
               double beta, double* __restrict__ y, int64_t ldy, int r, const int32_t* __restrict__ perm,
               float* __restrict__ vout, const F2* __restrict__ rowscale, F2* __restrict__ fix,
               int32_t* __restrict__ fixcnt, const Split* __restrict__ splits, const int32_t* __restrict__ fan,
               int32_t fan_base, int* err) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ int4 info[MP_PAIRS][MP_NS];
  __shared__ int s_last[MP_PAIRS];
  const int pair = threadIdx.x >> 6, wi = (threadIdx.x >> 5) & 1, lane = threadIdx.x & 31;
  const int gp = blockIdx.x * MP_PAIRS + pair;
  if (gp >= nrange) return;   // the whole pair
  const int p0 = wbeg[gp], n = wbeg[gp + 1] - p0;
  if (n <= 0) return;
  uint8_t* ring = smem + (size_t)pair * MP_NS * MP_STAGE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)MP_PAIRS * MP_NS * MP_STAGE) + pair * MP_NS;
  const int bid = 1 + pair;
  const uint64_t pol = policy_evict_first();
  // warp 0 of the pair issues the copies; its lanes hold the copy descriptors 32 at a time
  const PieceCopy zero{0, 0, 0, -1};
  PieceCopy dc = zero, dn = zero;
  int dbase = 0;
  if (wi == 0) {
    dc = lane < n ? cps[p0 + lane] : zero;
    dn = 32 + lane < n ? cps[p0 + 32 + lane] : zero;
  }
  // the sources of a piece's multiplier rows j = lane, lane + 32 (vector entries
  // moff + j, or fan[moff - fan_base + j] for a fan-out run), loaded one piece
  // ahead so that their latency overlaps the work on the pieces before
  int32_t src[2] = {0, 0};
  auto sources = [&](int i) {   // warp 0 of the pair
    const int sl = i - dbase;   // < 64: within dc / dn
    const uint32_t bf = __shfl_sync(HM_FULL, sl < 32 ? dc.bytes_flags : dn.bytes_flags, sl & 31);
    const int32_t moff = __shfl_sync(HM_FULL, sl < 32 ? dc.moff : dn.moff, sl & 31);
    const int nc = (int)(bf >> 24);
    const bool fan_run = moff >= fan_base;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int j = lane + 32 * u;
      src[u] = j < nc ? (fan_run ? __ldg(fan + (moff - fan_base) + j) : moff + j) : 0;
    }
  };
  auto issue = [&](int i) {   // warp 0 of the pair; src holds piece i's sources
    if (i - dbase >= 32) {
      dc = dn;
      dbase += 32;
      dn = dbase + 32 + lane < n ? cps[p0 + dbase + 32 + lane] : zero;
    }
    const int sl = i - dbase;
    const uint32_t off16 = __shfl_sync(HM_FULL, dc.off16, sl), bf = __shfl_sync(HM_FULL, dc.bytes_flags, sl);
    const int32_t sp = __shfl_sync(HM_FULL, dc.split_part, sl);
    const int s = i % MP_NS;
    uint8_t* st = ring + (size_t)s * MP_STAGE;
    const uint32_t nc = bf >> 24, pb = pad16m(bf & 0xffffu);
    fence_proxy_async();
    if (lane == 0) {
      info[pair][s] = make_int4((int)((bf >> 16) & 0xffu), sp, 0, 0);
      mbar_expect_tx(&bars[s], pb);
      bulk_g2s_hint(st, pay + (uint64_t)off16 * 16u, pb, &bars[s], pol);
    }
    __syncwarp();
    // multiplier rows lane, lane + 32 by cp.async (one bulk copy per piece only)
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int j = lane + 32 * u;
      if (j < (int)nc) cp_row(smem_u32(st + STAGE_BYTES + j * MP_TP), vec + (int64_t)src[u] * RP);
    }
    cp_arrive(&bars[s]);
    if (i + 1 < n) sources(i + 1);
  };
  if (wi == 0) {
    if (lane == 0) {
      for (int s = 0; s < MP_NS; ++s) mbar_init(&bars[s], 1 + 32);   // expect-tx arrival + 32 cp.async arrivals
      mbar_init_fence();
    }
    __syncwarp();
    sources(0);
    for (int i = 0; i < MP_NS && i < n; ++i) issue(i);
  }
  pair_sync(bid);   // the barriers are initialised before warp 1 waits on them
  const int g = lane >> 2, tq = lane & 3;
  float2 fhi[2][NT][2], flo[2][NT][2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        fhi[mt][nt][h] = make_float2(0.f, 0.f);
        flo[mt][nt][h] = make_float2(0.f, 0.f);
      }
  for (int i = 0; i < n; ++i) {
    const int s = i % MP_NS;
    const bool ok = mbar_wait(&bars[s], (uint32_t)((i / MP_NS) & 1));
    if (pair_any(bid, !ok)) {   // a copy did not arrive in time: wait (bounded) for those in flight, give up
      if (wi == 0 && lane == 0) {
        latch_error(err, 99);
        for (int j = i; j < n && j < i + MP_NS; ++j)
          mbar_wait(&bars[j % MP_NS], (uint32_t)((j / MP_NS) & 1), 50u);
      }
      return;
    }
    const uint32_t sa = smem_u32(ring + (size_t)s * MP_STAGE);
    PieceHdr H;
    {
      const uint4 a = lds128(sa), b = lds128(sa + 16);
      H.row0 = (int32_t)a.x;
      H.nrows = (uint16_t)(a.y & 0xffffu);
      H.flags = (uint16_t)(a.y >> 16);
      H.fb = (uint16_t)(a.z & 0xffffu);
      H.em = (uint16_t)(a.z >> 16);
      H.vin0 = (int32_t)a.w;
      H.ncols = (uint16_t)(b.x & 0xffffu);
      H.limbs = (uint16_t)(b.x >> 16);
      H.scale = F2{__uint_as_float(b.z), __uint_as_float(b.w)};
    }
    const int4 rinfo = info[pair][s];
    const int R = H.nrows;
    if (rinfo.x & PD_FIRST) {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            fhi[mt][nt][h] = make_float2(0.f, 0.f);
            flo[mt][nt][h] = make_float2(0.f, 0.f);
          }
    }
    if (32 * wi < R) {
      switch (H.fb) {
#define HM_MP(FF_, BB_) \
  case ((FF_) << 4) | (BB_): ms_piece<FF_, BB_>(sa, H, alpha_ff, wi, lane, fhi, flo); break;
        HM_FORMATS(HM_MP)
#undef HM_MP
        default:
          latch_error(err, 13);
      }
    }
    if (rinfo.x & PD_LAST) {
      const bool calpha = (H.flags & PH_CALPHA) != 0;
      const bool split = (rinfo.x & PD_SPLIT) != 0;
      const Split sp = split ? splits[rinfo.y >> 8] : Split{0, 1};
      bool emit = !split;
      if (split) {   // this part's rows, then the last part to arrive adds them all in part order
        F2* mine = fix + (size_t)(sp.slot0 + (rinfo.y & 0xff)) * CHUNK_ROWS * RP;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int row = 32 * wi + 4 * g + 2 * mt + h;
            if (row < R) {
#pragma unroll
              for (int nt = 0; nt < NT; ++nt) {
                const int k = 8 * nt + 2 * tq;
                *reinterpret_cast<float4*>(mine + row * RP + k) =
                    make_float4(fhi[mt][nt][h].x, flo[mt][nt][h].x, fhi[mt][nt][h].y, flo[mt][nt][h].y);
              }
            }
          }
        pair_sync(bid);   // both warps' rows before warp 0's release
        if (wi == 0 && lane == 0) s_last[pair] = atom_add_acq_rel(&fixcnt[rinfo.y >> 8], 1) == sp.nparts - 1;
        pair_sync(bid);   // the acquire before the parts are read
        emit = s_last[pair] != 0;
      }
      if (emit) {
        if (split) {
#pragma unroll
          for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                fhi[mt][nt][h] = make_float2(0.f, 0.f);
                flo[mt][nt][h] = make_float2(0.f, 0.f);
              }
          for (int part = 0; part < sp.nparts; ++part) {
            const F2* src = fix + (size_t)(sp.slot0 + part) * CHUNK_ROWS * RP;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int row = 32 * wi + 4 * g + 2 * mt + h;
                if (row < R) {
#pragma unroll
                  for (int nt = 0; nt < NT; ++nt) {
                    const float4 v = __ldcg(reinterpret_cast<const float4*>(src + row * RP + 8 * nt + 2 * tq));
                    const FF a = ff_add(FF{fhi[mt][nt][h].x, flo[mt][nt][h].x}, FF{v.x, v.y});
                    const FF b = ff_add(FF{fhi[mt][nt][h].y, flo[mt][nt][h].y}, FF{v.z, v.w});
                    fhi[mt][nt][h] = make_float2(a.hi, b.hi);
                    flo[mt][nt][h] = make_float2(a.lo, b.lo);
                  }
                }
              }
          }
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int row = 32 * wi + 4 * g + 2 * mt + h;
            if (row >= R) continue;
            if constexpr (MODE == MODE_Y) {
              const int o = __ldg(perm + H.row0 + row);
              double yo[NT][2];
#pragma unroll
              for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                  const int k = 8 * nt + 2 * tq + c;
                  yo[nt][c] = (beta != 0.0 && k < r) ? y[o + (int64_t)k * ldy] : 0.0;
                }
#pragma unroll
              for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                  const int k = 8 * nt + 2 * tq + c;
                  if (k < r) {
                    const double val = ff_to_d(FF{c ? fhi[mt][nt][h].y : fhi[mt][nt][h].x,
                                                  c ? flo[mt][nt][h].y : flo[mt][nt][h].x});
                    y[o + (int64_t)k * ldy] = (beta == 0.0) ? val : fma(beta, yo[nt][c], val);
                  }
                }
            } else {   // coefficient panels: float-float updates, one rounding to FP32
              const int gg = H.row0 + row;
              const F2 rsc = rowscale ? rowscale[gg] : F2{1.f, 0.f};
#pragma unroll
              for (int nt = 0; nt < NT; ++nt) {
                const int k0 = 8 * nt + 2 * tq;
                const float2 old = (MODE == MODE_VEC_ADD) ? *reinterpret_cast<const float2*>(vout + (int64_t)gg * RP + k0)
                                                          : make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 2; ++c)
                  if (k0 + c < r) {
                    FF v = {c ? fhi[mt][nt][h].y : fhi[mt][nt][h].x, c ? flo[mt][nt][h].y : flo[mt][nt][h].x};
                    if constexpr (MODE == MODE_VEC_ADD) v = ff_add_f(v, c ? old.y : old.x);
                    if (rowscale) v = ff_mul(v, FF{rsc.hi, rsc.lo});
                    if (calpha) v = ff_mul(v, FF{alpha_ff.hi, alpha_ff.lo});
                    vout[(int64_t)gg * RP + k0 + c] = v.hi + v.lo;
                  }
              }
            }
          }
      }
      if (split && emit && wi == 0 && lane == 0) fixcnt[rinfo.y >> 8] = 0;
    }
    pair_sync(bid);   // both warps are done with stage s
    if (wi == 0 && i + MP_NS < n) issue(i + MP_NS);
  }
}

// ---------------------------------------------------------------- column dots, FP32 pipes
// out (nc x RP) = A^T (nc x R) X (R x RP) with one FP32 FMA per product, one
// warp per range of pieces (its own ring of CW_NS stages, pieces only).  Lane
// (tq = lane / 8, g = lane % 8) holds the input rows 8 g .. 8 g + 7 of the
// segment for the right-hand sides 8 tq .. 8 tq + 7 in registers (read from
// the panel when the segment changes); per column it decodes its 8 codes,
// forms the 8 partial dots over its rows (FFMA2) and a reduce-scatter over the
// 8 lanes g leaves lane g with the column's total for right-hand side 8 tq + g
// (each column sums its <= 64 rows in FP32, as the single-RHS kernel).
constexpr int CW_WARPS = 16;
constexpr int CW_NS = 2;
constexpr size_t CW_SMEM = (size_t)CW_WARPS * CW_NS * STAGE_BYTES + (size_t)CW_WARPS * CW_NS * 8;
static_assert(CW_SMEM <= 227 * 1024, "column-dot warps per block");

// Reduce-scatter of 8 values over the 8 lanes q = lane bits 0..2 (fixed
// pattern): returns the lanes' total of value q.
__device__ __forceinline__ float rs8(float (&p)[8], int q) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const bool up = (q & 4) != 0;
    const float send = up ? p[k] : p[k + 4], keep = up ? p[k + 4] : p[k];
    p[k] = keep + __shfl_xor_sync(HM_FULL, send, 4);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const bool up = (q & 2) != 0;
    const float send = up ? p[k] : p[k + 2], keep = up ? p[k + 2] : p[k];
    p[k] = keep + __shfl_xor_sync(HM_FULL, send, 2);
  }
  const bool up = (q & 1) != 0;
  const float send = up ? p[0] : p[1], keep = up ? p[1] : p[0];
  return keep + __shfl_xor_sync(HM_FULL, send, 1);
}

template <int F, int B>
__device__ __forceinline__ void cw_piece(uint32_t sa, int R, int nc, int flags, const float2 (&xr)[8][4], int lane,
                                         F2 alpha, float* __restrict__ partial, float* __restrict__ vout) {
  const int tq = lane >> 3, g = lane & 7;
  const bool fin = (flags & ITEM_FINAL) != 0;
  const int Rp = (R + 15) & ~15;   // rows R .. Rp - 1 hold zero codes
  const uint32_t stride = (uint32_t)Rp * B;
  const uint32_t cm = sa + (uint32_t)sizeof(CPieceHdr);
  const uint32_t scl = cm + 8u * nc;
  const uint32_t cb = cm + (fin ? 16u : 8u) * nc + (uint32_t)(8 * g * B);
  const bool rows_on = 8 * g < Rp;
  const FF fa = {alpha.hi, alpha.lo};
#pragma unroll 2
  for (int j = 0; j < nc; ++j) {
    int e = 0, m = 0;
    if constexpr (F == 2) {
      const uint32_t em = lds32(cm + 8u * j) & 0xffffu;
      e = em & 0xff;
      m = em >> 8;
    }
    float2 h2[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (rows_on) decode8p<F, B>(cb + (uint32_t)j * stride, e, m, h2);
    float2 p2[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float v = (u & 1) ? h2[u >> 1].y : h2[u >> 1].x;
      const float2 vv = make_float2(v, v);
#pragma unroll
      for (int k = 0; k < 4; ++k) p2[k] = __ffma2_rn(vv, xr[u][k], p2[k]);
    }
    float p[8] = {p2[0].x, p2[0].y, p2[1].x, p2[1].y, p2[2].x, p2[2].y, p2[3].x, p2[3].y};
    const float tot = rs8(p, g);
    const int32_t out = (int32_t)lds32(cm + 8u * j + 4u);
    const int64_t o = (int64_t)out * RP + 8 * tq + g;
    if (fin) {
      const uint2 f = lds64(scl + 8u * j);
      FF sc = {__uint_as_float(f.x), __uint_as_float(f.y)};
      if (flags & ITEM_ALPHA) sc = ff_mul(sc, fa);
      const FF v = ff_mul(FF{tot, 0.f}, sc);
      vout[o] = v.hi + v.lo;
    } else {
      partial[o] = tot;
    }
  }
}

__global__ void __launch_bounds__(CW_WARPS * 32, 1)
    k_cdot_ws(const ItemCopy* __restrict__ cps, const int32_t* __restrict__ wbeg, int nrange,
              const uint8_t* __restrict__ pay, const float* __restrict__ vec, F2 alpha, float* __restrict__ partial,
              float* __restrict__ vout, int* err) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * CW_WARPS + warp;
  if (gw >= nrange) return;
  const int p0 = wbeg[gw], n = wbeg[gw + 1] - p0;
  if (n <= 0) return;
  uint8_t* ring = smem + (size_t)warp * CW_NS * STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)CW_WARPS * CW_NS * STAGE_BYTES) + warp * CW_NS;
  const uint64_t pol = policy_evict_first();
  const ItemCopy zero{0, 0, -1, 0};
  ItemCopy dc = lane < n ? cps[p0 + lane] : zero;
  ItemCopy dn = 32 + lane < n ? cps[p0 + 32 + lane] : zero;
  int dbase = 0;
  auto issue = [&](int i) {   // all lanes
    if (i - dbase >= 32) {
      dc = dn;
      dbase += 32;
      dn = dbase + 32 + lane < n ? cps[p0 + dbase + 32 + lane] : zero;
    }
    const int sl = i - dbase;
    const uint32_t off16 = __shfl_sync(HM_FULL, dc.off16, sl), bytes = __shfl_sync(HM_FULL, dc.bytes, sl);
    if (lane == 0) {
      const int s = i % CW_NS;
      const uint32_t pb = pad16m(bytes);
      fence_proxy_async();
      mbar_expect_tx(&bars[s], pb);
      bulk_g2s_hint(ring + (size_t)s * STAGE_BYTES, pay + (uint64_t)off16 * 16u, pb, &bars[s], pol);
    }
  };
  if (lane == 0) {
    for (int s = 0; s < CW_NS; ++s) mbar_init(&bars[s], 1);
    mbar_init_fence();
  }
  __syncwarp();
  for (int i = 0; i < CW_NS && i < n; ++i) issue(i);
  const int tq = lane >> 3, g = lane & 7;
  float2 xr[8][4];
  int32_t xv = -1, xn = -1;
  for (int i = 0; i < n; ++i) {
    const int s = i % CW_NS;
    if (!mbar_wait(&bars[s], (uint32_t)((i / CW_NS) & 1))) {   // wait (bounded) for the copies in flight, give up
      if (lane == 0) {
        latch_error(err, 99);
        for (int j = i; j < n && j < i + CW_NS; ++j)
          mbar_wait(&bars[j % CW_NS], (uint32_t)((j / CW_NS) & 1), 50u);
      }
      return;
    }
    const uint32_t sa = smem_u32(ring + (size_t)s * STAGE_BYTES);
    const uint4 hw = lds128(sa);   // CPieceHdr
    const int32_t hvin = (int32_t)hw.x;
    const int R = (int)(hw.y & 0xffffu), nc = (int)(hw.y >> 16);
    const uint32_t fb = hw.z & 0xffffu, flags = hw.z >> 16;
    if (hvin != xv || R != xn) {   // the input rows of a new segment
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int row = 8 * g + u;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (row < R) {
          const float4* src = reinterpret_cast<const float4*>(vec + (int64_t)(hvin + row) * RP + 8 * tq);
          a = __ldg(src);
          b = __ldg(src + 1);
        }
        xr[u][0] = make_float2(a.x, a.y);
        xr[u][1] = make_float2(a.z, a.w);
        xr[u][2] = make_float2(b.x, b.y);
        xr[u][3] = make_float2(b.z, b.w);
      }
      xv = hvin;
      xn = R;
    }
    switch (fb) {
#define HM_CW(FF_, BB_) \
  case ((FF_) << 4) | (BB_): cw_piece<FF_, BB_>(sa, R, nc, (int)flags, xr, lane, alpha, partial, vout); break;
      HM_FORMATS(HM_CW)
#undef HM_CW
      default:
        latch_error(err, 15);
    }
    __syncwarp();
    if (i + CW_NS < n) issue(i + CW_NS);
  }
}

// ---------------------------------------------------------------- launchers
cudaError_t mr_init() {
  cudaError_t e = cudaFuncSetAttribute(k_cdot_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CW_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_ms<MODE_Y>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MP_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_ms<MODE_VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MP_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_ms<MODE_VEC_ADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MP_SMEM);
  return e;
}

cudaError_t launch_gather_mr(const double* x, int64_t ldx, int r, const int32_t* perm, int n, float* v,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t tot = (int64_t)n * RP;
  k_gather_mr<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(x, ldx, r, perm, n, v);
  return cudaGetLastError();
}

cudaError_t launch_gsum_mr(const GsumOut* outs, int nouts, const F2* pscale, const float* partial, F2 alpha, float* v,
                           cudaStream_t st) {
  if (nouts <= 0) return cudaSuccess;
  const int64_t tot = (int64_t)nouts * RP;
  k_gsum_mr<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(outs, nouts, pscale, partial, alpha, v);
  return cudaGetLastError();
}

// nblk ranges, one per warp
cudaError_t launch_cdot_ws(const ItemCopy* items, const int32_t* wbeg, int nblk, const uint8_t* pay, const float* vec,
                           F2 alpha, float* partial, float* vout, int* err, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  k_cdot_ws<<<(unsigned)((nblk + CW_WARPS - 1) / CW_WARPS), CW_WARPS * 32, CW_SMEM, st>>>(items, wbeg, nblk, pay, vec,
                                                                                           alpha, partial, vout, err);
  return cudaGetLastError();
}

// nblk ranges, one per warp pair; chunks of at most MP_ROWS rows
cudaError_t launch_rgemv_ms(int mode, const PieceCopy* pieces, const int32_t* wbeg, int nblk, const uint8_t* pay,
                            const float* vec, double alpha, F2 alpha_ff, double beta, double* y, int64_t ldy, int r,
                            const int32_t* perm, float* vout, const F2* rowscale, F2* fix, int32_t* fixcnt,
                            const Split* splits, const int32_t* fan, int32_t fan_base, int* err, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((nblk + MP_PAIRS - 1) / MP_PAIRS);
#define HM_MSG(M)                                                                                            \
  k_rgemv_ms<M><<<grid, MP_THREADS, MP_SMEM, st>>>(pieces, wbeg, nblk, pay, vec, alpha, alpha_ff, beta, y, ldy, r, \
                                                   perm, vout, rowscale, fix, fixcnt, splits, fan, fan_base, err)
  if (mode == MODE_Y)
    HM_MSG(MODE_Y);
  else if (mode == MODE_VEC)
    HM_MSG(MODE_VEC);
  else
    HM_MSG(MODE_VEC_ADD);
#undef HM_MSG
  return cudaGetLastError();
}

}  // namespace hm
