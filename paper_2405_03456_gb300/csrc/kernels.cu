// sm_103a kernels of libhm: on-the-fly decompression (Sec. 4.1, Alg. 8) fused
// into the column-dot and row-chunk products of the H / UH / H^2 matvec (Sec. 3).
//
// Both product kernels are streaming kernels: each warp owns a contiguous
// range of the launch's packed units (about equal bytes per warp) and pulls
// them through its own ring of shared-memory stages with bulk copies
// (cp.async.bulk, completion on an mbarrier), so every warp keeps several KB
// in flight while it decodes the unit that has landed.  Units carry inline
// headers (formats, output indices, column metadata): the only global reads
// besides the payload are the copy descriptors (prefetched 32 at a time) and
// the multipliers (gathered one unit ahead).
// Race freedom (Sec. 3.1, Alg. 3): every output row belongs to exactly one
// chunk; a chunk is reduced by one warp, or, when it straddles warp ranges, by
// whichever of its parts finishes last, adding the parts in a fixed order.  No
// floating-point atomics: results are bitwise reproducible.
#include <cstdint>
#include <cuda_runtime.h>

#include "decode.cuh"

namespace hm {

constexpr int A_XOFF = STAGE_BYTES;                 // x segment inside a column-dot stage
constexpr int A_STAGE = A_XOFF + SEG_ROWS * 8 + 16; // 4624 bytes
constexpr int C_MOFF = STAGE_BYTES;                 // multipliers inside a row-chunk stage
constexpr int C_STAGE = C_MOFF + PIECE_MAX_COLS * 8 + 16;
constexpr int C_INFO = 16;                          // per-stage record (range flags, split / part, multiplier parity)
constexpr int SMEM_TAIL = 128;                      // lane over-reads past the last stage

__device__ __forceinline__ uint32_t pad16u(uint32_t x) { return (x + 15u) & ~15u; }

// After a bounded wait gave up: wait (bounded) for the copies still in flight
// into this warp's stages [i, issued) so that none lands after the block exits.
template <int NS>
__device__ void drain(uint64_t* bars, int i, int issued, uint32_t it0 = 0) {
  for (int j = i; j < issued; ++j) {
    const uint32_t u = it0 + (uint32_t)j;
    mbar_wait(&bars[u % NS], (u / NS) & 1u, 50u);
  }
}

// Programmatic dependent launch: a kernel lets the next one in the stream start
// at once (its blocks take SM resources as they free up and run their prologue),
// and waits for the previous one (completed, memory visible) before it reads
// anything that kernel wrote.  Both are no-ops for ordinary launches.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------- column dots (phase A)
// (s, c) += (s2, c2) for Dot2 pairs (TwoSum of the leading parts).
template <int TIER>
__device__ __forceinline__ void pair_add(float& s, float& c, float s2, float c2) {
  if constexpr (TIER == TIER_F32) {
    s += s2;
  } else {
    float t, e;
    two_sum(s, s2, t, e);
    s = t;
    c += c2 + e;
  }
}

// One halving step of a reduce-scatter over lanes: C values per lane, the
// lane keeps the upper half (if `up`) or the lower half and adds the partner's
// (lane ^ mask) copy of it.
template <int TIER, int C>
__device__ __forceinline__ void rscatter_step(float (&p)[8], float (&pc)[8], bool up, int mask) {
  constexpr int H = C / 2;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const float send = up ? p[k] : p[k + H];
    const float keep = up ? p[k + H] : p[k];
    const float keepc = up ? pc[k + H] : pc[k];
    const float got = __shfl_xor_sync(HM_FULL, send, mask);
    float gotc = 0.f;
    if constexpr (TIER == TIER_FF) gotc = __shfl_xor_sync(HM_FULL, up ? pc[k] : pc[k + H], mask);
    p[k] = keep;
    pc[k] = keepc;
    pair_add<TIER>(p[k], pc[k], got, gotc);
  }
}

// Reduce-scatter of 8 per-column partials over the L lanes q of a group (lane
// bits 0 .. log2 L - 1): afterwards lane q holds in p[0 .. 8/L) the group's
// totals of columns q * 8/L + k.  Fixed exchange pattern (deterministic).
template <int TIER, int L>
__device__ __forceinline__ void reduce_scatter8(float (&p)[8], float (&pc)[8], int q) {
  if constexpr (L == 8) {
    rscatter_step<TIER, 8>(p, pc, (q & 4) != 0, 4);
    rscatter_step<TIER, 4>(p, pc, (q & 2) != 0, 2);
    rscatter_step<TIER, 2>(p, pc, (q & 1) != 0, 1);
  } else {
    static_assert(L == 4, "lanes per column");
    rscatter_step<TIER, 8>(p, pc, (q & 2) != 0, 2);
    rscatter_step<TIER, 4>(p, pc, (q & 1) != 0, 1);
  }
}

// One column-dot piece at shared address sa.  A column's <= 64 rows are
// spread over LPC = 64 / RL lanes of RL rows each; the warp's NG = 32 / LPC
// lane groups take the columns g, g + NG, ... (x rows in registers).  The
// column loop is rolled: each step shifts the partials down one register, so
// after 8 steps p[t] holds column g + NG t of this round; a round covers
// 8 NG columns and ends with a reduce-scatter over the LPC lanes.
template <int TIER, int F, int B, int RL>
__device__ __forceinline__ void cs_piece(uint32_t sa, int R, int nc, int flags, const float (&xh)[RL],
                                         const float (&xl)[RL], int lane, F2 alpha, F2* __restrict__ partial,
                                         float2* __restrict__ vout) {
  constexpr int LPC = SEG_ROWS / RL, NG = 32 / LPC, KO = 8 / LPC;
  const int g = lane / LPC, q = lane % LPC;
  const uint32_t stride = (((uint32_t)R + 15u) & ~15u) * B;
  const bool fin = (flags & ITEM_FINAL) != 0;
  const uint32_t cm = sa + (uint32_t)sizeof(CPieceHdr);          // CColMeta[nc]
  const uint32_t sc = cm + 8u * nc;                                // F2[nc] (final only)
  const uint32_t cb = cm + (fin ? 16u : 8u) * nc + (uint32_t)(RL * q * B);
  const bool rows_on = RL * q < R;
  for (int j0 = 0; j0 < nc; j0 += 8 * NG) {
    float p[8], pc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      p[t] = 0.f;
      pc[t] = 0.f;
    }
#pragma unroll 1
    for (int t = 0; t < 8; ++t) {
      const int j = j0 + g + NG * t;
      float a = 0.f, ac = 0.f;
      if (j < nc && rows_on) {
        int e = 0, m = 0;
        if constexpr (F == 2) {
          const uint32_t em = lds32(cm + 8u * j) & 0xffffu;
          e = em & 0xff;
          m = em >> 8;
        }
        float2 a2 = make_float2(0.f, 0.f), ac2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int hb = 0; hb < RL / RPL; ++hb) {
          float h[8], l[8];
          decode8s<TIER, F, B>(cb + (uint32_t)j * stride + (uint32_t)(hb * RPL * B), e, m, h, l);
#pragma unroll
          for (int u = 0; u < 8; u += 2) {
            if constexpr (TIER == TIER_F32) {
              a = fmaf(h[u], xh[hb * RPL + u], a);
              a = fmaf(h[u + 1], xh[hb * RPL + u + 1], a);
            } else {
              dot2_2(a2, ac2, make_float2(h[u], h[u + 1]), make_float2(l[u], l[u + 1]),
                     make_float2(xh[hb * RPL + u], xh[hb * RPL + u + 1]),
                     make_float2(xl[hb * RPL + u], xl[hb * RPL + u + 1]));
            }
          }
        }
        if constexpr (TIER == TIER_FF) {   // even + odd rows (TwoSum of the leading parts)
          a = a2.x;
          ac = ac2.x;
          pair_add<TIER>(a, ac, a2.y, ac2.y);
        }
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        p[k] = p[k + 1];
        pc[k] = pc[k + 1];
      }
      p[7] = a;
      pc[7] = ac;
    }
    reduce_scatter8<TIER, LPC>(p, pc, q);
#pragma unroll
    for (int k = 0; k < KO; ++k) {
      const int j = j0 + g + NG * (q * KO + k);
      if (j < nc) {
        const float s = p[k], c = pc[k];
        const float h = s + c;
        FF v = {h, c - (h - s)};
        const int32_t out = (int32_t)lds32(cm + 8u * j + 4u);
        if (fin) {
          const uint2 f = lds64(sc + 8u * j);
          v = ff_mul(v, FF{__uint_as_float(f.x), __uint_as_float(f.y)});
          if (flags & ITEM_ALPHA) v = ff_mul(v, FF{alpha.hi, alpha.lo});
          vout[out] = make_float2(v.hi, v.lo);
        } else {
          partial[out] = F2{v.hi, v.lo};
        }
      }
    }
  }
}

// FP32-tier column-dot piece: lanes (g, q) = (lane / 8, lane % 8) take rows
// 8q .. 8q+7 of the columns g, g + 4, ...; two columns per step (independent
// decodes), products summed in FP32 pairs; the 4 steps of a round are unrolled
// so that p[t] holds column g + 4t; a round of 32 columns ends with the
// reduce-scatter over the 8 lanes.  Steps past the last column are skipped as a
// whole; a ragged step masks its results.
template <int F, int B>
__device__ __forceinline__ void cs_piece_f32(uint32_t sa, int R, int nc, int flags, const float2 (&x2)[4], int lane,
                                             F2 alpha, F2* __restrict__ partial, float2* __restrict__ vout) {
  constexpr int NG = 4;
  const int g = lane >> 3, q = lane & 7;
  const uint32_t stride = (((uint32_t)R + 15u) & ~15u) * B;
  const bool fin = (flags & ITEM_FINAL) != 0;
  const uint32_t cm = sa + (uint32_t)sizeof(CPieceHdr);          // CColMeta[nc]
  const uint32_t sc = cm + 8u * nc;                                // F2[nc] (final only)
  const uint32_t cb = cm + (fin ? 16u : 8u) * nc + (uint32_t)(RPL * q * B);
  const bool rows_on = RPL * q < R;
  for (int j0 = 0; j0 < nc; j0 += 8 * NG) {
    float p[8], pc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      p[t] = 0.f;
      pc[t] = 0.f;
    }
    const int tmax = (nc - j0 + NG - 1) / NG;   // steps holding a column (same for the warp)
#pragma unroll
    for (int t = 0; t < 8; t += 2) {
      float r[2] = {0.f, 0.f};
      if (t < tmax) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = j0 + g + NG * (t + h);
          const bool v = j < nc && rows_on;
          const int jj = v ? j : 0;
          int e = 0, m = 0;
          if constexpr (F == 2) {
            const uint32_t em = lds32(cm + 8u * jj) & 0xffffu;
            e = em & 0xff;
            m = em >> 8;
          }
          float2 h2[4];
          decode8p<F, B>(cb + (uint32_t)jj * stride, e, m, h2);
          float2 a2 = __fmul2_rn(h2[0], x2[0]);
          a2 = __ffma2_rn(h2[1], x2[1], a2);
          a2 = __ffma2_rn(h2[2], x2[2], a2);
          a2 = __ffma2_rn(h2[3], x2[3], a2);
          r[h] = v ? a2.x + a2.y : 0.f;
        }
      }
      p[t] = r[0];
      p[t + 1] = r[1];
    }
    reduce_scatter8<TIER_F32, 8>(p, pc, q);
    const int j = j0 + g + NG * q;
    if (j < nc) {
      FF v = {p[0], 0.f};
      const int32_t out = (int32_t)lds32(cm + 8u * j + 4u);
      if (fin) {
        const uint2 f = lds64(sc + 8u * j);
        v = ff_mul(v, FF{__uint_as_float(f.x), __uint_as_float(f.y)});
        if (flags & ITEM_ALPHA) v = ff_mul(v, FF{alpha.hi, alpha.lo});
        vout[out] = make_float2(v.hi, v.lo);
      } else {
        partial[out] = F2{v.hi, v.lo};
      }
    }
  }
}

// Arguments of the column-dot products shared by every range of a launch.
struct CsArgs {
  const ItemCopy* cps;
  const uint8_t* pay;
  const float2* vec;
  F2 alpha;
  F2* partial;
  float2* vout;
  int* err;
};

// One warp's range of column-dot pieces [p0, p0 + n): a ring of NS shared-memory
// stages (SSTR bytes apart) filled by bulk copies (piece + its input segment
// when it changes), decoded and reduced.  it counts the stages this warp has
// used before (their mbarrier phases) and is advanced.  Returns false if a
// copy did not arrive in time (error latched).
template <int TIER, int NS, int SSTR>
__device__ __forceinline__ bool cs_range(const CsArgs& A, int p0, int n, uint8_t* ring, uint64_t* bars, int lane,
                                         uint32_t& it) {
  const uint32_t sring = smem_u32(ring);
  const uint32_t it0 = it;
  // copy descriptors, 32 per batch: lane l holds entry dbase + l (dc) and dbase + 32 + l (dn)
  const ItemCopy zero{0, 0, -1, 0};
  ItemCopy dc = lane < n ? A.cps[p0 + lane] : zero;
  ItemCopy dn = 32 + lane < n ? A.cps[p0 + 32 + lane] : zero;
  int dbase = 0, issued = 0;
  const uint64_t pol = policy_evict_first();
  int32_t last_vin = -1, last_rows = -1;   // input segment of the last issued piece
  auto issue = [&](int i) {   // all lanes; copies piece i (and its input segment if new) into stage (it0 + i) % NS
    if (i - dbase >= 32) {
      dc = dn;
      dbase += 32;
      dn = dbase + 32 + lane < n ? A.cps[p0 + dbase + 32 + lane] : zero;
    }
    const int sl = i - dbase;
    const uint32_t off16 = __shfl_sync(HM_FULL, dc.off16, sl);
    const uint32_t bytes = __shfl_sync(HM_FULL, dc.bytes, sl);
    const int32_t vin = __shfl_sync(HM_FULL, dc.vin, sl);
    const int32_t nrows = __shfl_sync(HM_FULL, dc.nrows, sl);
    const bool newx = vin != last_vin || nrows != last_rows;
    last_vin = vin;
    last_rows = nrows;
    if (lane == 0) {
      const uint32_t st_i = (it0 + (uint32_t)i) % NS;
      uint8_t* st = ring + st_i * SSTR;
      uint64_t* bar = &bars[st_i];
      const uint32_t pb = pad16u(bytes);
      const int64_t x0 = (int64_t)vin & ~int64_t(1);
      const uint32_t xb = newx ? pad16u((uint32_t)((vin - x0) + nrows) * 8u) : 0u;
      fence_proxy_async();
      mbar_expect_tx(bar, pb + xb);
      bulk_g2s_hint(st, A.pay + (uint64_t)off16 * 16u, pb, bar, pol);
      if (newx) bulk_g2s(st + A_XOFF, A.vec + x0, xb, bar);
    }
    issued = i + 1;
  };
  for (int i = 0; i < NS && i < n; ++i) issue(i);
  constexpr int RL = RPL;   // rows per lane
  float xh[RL], xl[RL];
  int32_t xv = -1, xr = -1;
  for (int i = 0; i < n; ++i) {
    const uint32_t u = it0 + (uint32_t)i;
    const uint32_t s = u % NS;
    if (!mbar_wait(&bars[s], (u / NS) & 1u)) {
      latch_error(A.err, 99);
      drain<NS>(bars, i + 1, issued, it0);
      it = it0 + (uint32_t)issued;
      return false;
    }
    const uint32_t sa = sring + s * (uint32_t)SSTR;
    const uint4 hw = lds128(sa);                       // CPieceHdr
    const int32_t hvin = (int32_t)hw.x;
    const int R = (int)(hw.y & 0xffffu), nc = (int)(hw.y >> 16);
    const uint32_t fb = hw.z & 0xffffu, flags = hw.z >> 16;
    if (hvin != xv || R != xr) {   // a new input segment came with this piece
      const uint32_t xa = sa + A_XOFF + 8u * (uint32_t)(hvin & 1);
      const int q = lane % (SEG_ROWS / RL);
#pragma unroll
      for (int k = 0; k < RL; ++k) {
        const int r = RL * q + k;
        uint2 v = make_uint2(0u, 0u);
        if (r < R) v = lds64(xa + 8u * r);
        xh[k] = __uint_as_float(v.x);
        xl[k] = __uint_as_float(v.y);
      }
      xv = hvin;
      xr = R;
    }
    if constexpr (TIER == TIER_F32) {
      const float2 x2[4] = {make_float2(xh[0], xh[1]), make_float2(xh[2], xh[3]), make_float2(xh[4], xh[5]),
                            make_float2(xh[6], xh[7])};
      switch (fb) {
#define HM_CS(FF_, BB_) \
  case ((FF_) << 4) | (BB_): cs_piece_f32<FF_, BB_>(sa, R, nc, (int)flags, x2, lane, A.alpha, A.partial, A.vout); break;
        HM_FORMATS(HM_CS)
#undef HM_CS
        default:
          latch_error(A.err, 1);
      }
    } else {
      switch (fb) {
#define HM_CS(FF_, BB_) \
  case ((FF_) << 4) | (BB_): cs_piece<TIER, FF_, BB_, RL>(sa, R, nc, (int)flags, xh, xl, lane, A.alpha, A.partial, A.vout); break;
        HM_FORMATS(HM_CS)
#undef HM_CS
        default:
          latch_error(A.err, 1);
      }
    }
    __syncwarp();
    if (issued < n) issue(issued);
  }
  it = it0 + (uint32_t)n;
  return true;
}

template <int TIER, int NW, int NS>
__global__ void __launch_bounds__(NW * 32, 1)
    k_cstream(const ItemCopy* __restrict__ cps, const int32_t* __restrict__ wbeg, int nwt,
              const uint8_t* __restrict__ pay, const float2* __restrict__ vec, F2 alpha,
              F2* __restrict__ partial, float2* __restrict__ vout, int* err) {
  extern __shared__ __align__(128) uint8_t smem[];
  pdl_trigger();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * NW + warp;
  if (gw >= nwt) return;
  const int p0 = wbeg[gw], n = wbeg[gw + 1] - p0;
  if (n <= 0) return;
  uint8_t* ring = smem + (size_t)warp * NS * A_STAGE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)NW * NS * A_STAGE) + warp * NS;
  if (lane == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    mbar_init_fence();
  }
  __syncwarp();
  pdl_wait();   // the input segments come from the previous kernel
  const CsArgs A{cps, pay, vec, alpha, partial, vout, err};
  uint32_t it = 0;
  cs_range<TIER, NS, A_STAGE>(A, p0, n, ring, bars, lane, it);
}

// ---------------------------------------------------------------- row chunks (phase C)
// Lane split of a row-chunk piece: G = ceil(R / 8) lanes per column, S = 32 / G
// column slots, lane = slot G + q.  The divisions by the runtime G go through a
// table: slot = (lane * ceil(1024 / G)) >> 10 is exact for lane < 1024 / G,
// which holds for lane < 32 and G <= 16.
__constant__ uint16_t c_div1024[17] = {0,    1024, 512, 342, 256, 205, 171, 147, 128,
                                       114,  103,  94,  86,  79,  74,  69,  64};
__constant__ uint8_t c_slots[17] = {0, 32, 16, 10, 8, 6, 5, 4, 4, 3, 3, 2, 2, 2, 2, 2, 2};
__device__ __forceinline__ void lane_split(int R, int lane, int& G, int& S, int& slot, int& q) {
  G = (R + RPL - 1) / RPL;
  S = c_slots[G];
  slot = (lane * (int)c_div1024[G]) >> 10;
  q = lane - slot * G;
}

// Sum of the piece's columns into this lane's 8 rows: lanes (slot, q) take
// rows 8q .. 8q+7 of the columns slot, slot + S, ...; FP32 sums (or Dot2
// pairs) per piece, folded into the float-float row sums (row pairs
// (2k, 2k+1): hi[k], lo[k]) at the end.
template <int TIER, int F, int B>
__device__ __forceinline__ void rs_piece(uint32_t sa, const PieceHdr& H, uint32_t tbl, F2 alpha_ff, int lane,
                                         float2 (&ahi)[4], float2 (&alo)[4]) {
  const int R = H.nrows;
  int G, S, slot, q;
  lane_split(R, lane, G, S, slot, q);
  const bool tile = (H.flags & PH_TILE) != 0;
  const uint32_t stride = pad8u((uint32_t)R * B);
  const uint32_t cm = sa + (uint32_t)sizeof(PieceHdr);   // merged pieces: uint16 em[ncols]
  const uint32_t cb = cm + (tile ? 0u : pad8u(2u * H.ncols)) + (uint32_t)(RPL * q * B);
  const int e_t = H.em & 0xff, m_t = H.em >> 8;
  FF sc = {1.f, 0.f};
  if (tile) {
    sc = FF{H.scale.hi, H.scale.lo};
    if (H.flags & PH_TALPHA) sc = ff_mul(sc, FF{alpha_ff.hi, alpha_ff.lo});
  }
  const int nc = slot < S ? H.ncols : 0;
  if constexpr (TIER == TIER_F32) {
    float2 s2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) s2[k] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int j = slot; j < nc; j += S) {
      const float vh = __uint_as_float(lds32(tbl + 8u * j)) * sc.hi;
      int e = e_t, m = m_t;
      if constexpr (F == 2) {
        if (!tile) {
          const uint32_t em = lds32((cm + 2u * j) & ~3u) >> (16u * (j & 1));
          e = em & 0xff;
          m = (em >> 8) & 0xff;
        }
      }
      float2 h2[4];
      decode8p<F, B>(cb + (uint32_t)j * stride, e, m, h2);
      const float2 v2 = make_float2(vh, vh);
#pragma unroll
      for (int k = 0; k < 4; ++k) s2[k] = __ffma2_rn(h2[k], v2, s2[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) ff_add_f2(ahi[k], alo[k], s2[k]);
  } else {
    // float-float tier: Dot2 on row pairs (2k, 2k+1)
    float2 s2[4], c2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      s2[k] = make_float2(0.f, 0.f);
      c2[k] = make_float2(0.f, 0.f);
    }
#pragma unroll 2
    for (int j = slot; j < nc; j += S) {
      const uint2 vb = lds64(tbl + 8u * j);
      float vh = __uint_as_float(vb.x), vl = __uint_as_float(vb.y);
      int e = e_t, m = m_t;
      if (tile) {
        const FF r = ff_mul(FF{vh, vl}, sc);
        vh = r.hi;
        vl = r.lo;
      } else if constexpr (F == 2) {
        const uint32_t em = lds32((cm + 2u * j) & ~3u) >> (16u * (j & 1));
        e = em & 0xff;
        m = (em >> 8) & 0xff;
      }
      float h[8], l[8];
      decode8s<TIER, F, B>(cb + (uint32_t)j * stride, e, m, h, l);
      const float2 vh2 = make_float2(vh, vh), vl2 = make_float2(vl, vl);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        dot2_2(s2[k], c2[k], make_float2(h[2 * k], h[2 * k + 1]), make_float2(l[2 * k], l[2 * k + 1]), vh2, vl2);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) ff_add_dot2(ahi[k], alo[k], s2[k], c2[k]);
  }
}

// Float-float row sums of a lane (RL rows), passed by value to the emit path.
template <int RL>
struct AccR {
  FF v[RL];
};

// Write the finished rows g0 .. g0 + nr - 1 of a chunk (nr <= RL; a lane's rows).
// Every global load the rows need (y through perm, the old coefficients, the row
// scales) is issued before the first store, so the lane waits for one round trip
// instead of one per row.  Coefficient vectors stay in float-float arithmetic
// (FP64 instructions are scarce on this GPU); y takes the FP64 sum hi + lo.
template <int MODE, int RL>
__device__ __forceinline__ void rs_store_rows(const AccR<RL>& acc, int g0, int nr, F2 alpha_ff, double beta,
                                              double* __restrict__ y, const int32_t* __restrict__ perm,
                                              float2* __restrict__ vout, const F2* __restrict__ rowscale,
                                              bool calpha) {
  if constexpr (MODE == MODE_Y) {
    int o[RL];
#pragma unroll
    for (int u = 0; u < RL; ++u) o[u] = u < nr ? __ldg(perm + g0 + u) : 0;
    double yo[RL];
#pragma unroll
    for (int u = 0; u < RL; ++u) yo[u] = (u < nr && beta != 0.0) ? y[o[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < RL; ++u) {
      if (u < nr) {
        const double val = ff_to_d(acc.v[u]);
        y[o[u]] = (beta == 0.0) ? val : fma(beta, yo[u], val);
      }
    }
  } else {
    float2 old[RL], sc[RL];
#pragma unroll
    for (int u = 0; u < RL; ++u) {
      old[u] = (MODE == MODE_VEC_ADD && u < nr) ? __ldcg(vout + g0 + u) : make_float2(0.f, 0.f);
      sc[u] = (rowscale && u < nr) ? __ldg(reinterpret_cast<const float2*>(rowscale + g0 + u)) : make_float2(1.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < RL; ++u) {
      if (u < nr) {
        FF v = acc.v[u];
        if constexpr (MODE == MODE_VEC_ADD) v = ff_add(v, FF{old[u].x, old[u].y});
        if (rowscale) v = ff_mul(v, FF{sc[u].x, sc[u].y});
        if (calpha) v = ff_mul(v, FF{alpha_ff.hi, alpha_ff.lo});
        vout[g0 + u] = make_float2(v.hi, v.lo);
      }
    }
  }
}

// End of a warp's part of a chunk (hflags: piece header flags, bit 16 set when
// the chunk is shared by several warps): reduce the column slots (fixed order), then
// emit the rows, directly or through the fix-up of a chunk shared by warps (the
// last part to arrive sums all parts in part order, so the result does not
// depend on which warp finishes last).
// Out of line: it runs once per part and keeps the piece loop compact.
template <int MODE, int RL>
__device__ __noinline__ bool rs_emit(AccR<RL> acc, int row0, int R, int hflags, int split, int pidx, int lane,
                                     F2 alpha_ff, double beta, double* __restrict__ y,
                                     const int32_t* __restrict__ perm, float2* __restrict__ vout,
                                     const F2* __restrict__ rowscale, F2* __restrict__ fix,
                                     int32_t* __restrict__ fixcnt, const Split* __restrict__ splits) {
  static_assert(RL == RPL, "lanes hold RPL rows");
  int G, S, slot, q;
  lane_split(R, lane, G, S, slot, q);
  // pairwise tree over the S column slots (slot s takes s + off when s is a
  // multiple of 2 off): log2 S shuffle rounds, all rows of a round in flight
  for (int off = 1; off < S; off <<= 1) {
    float hi[RL], lo[RL];
#pragma unroll
    for (int u = 0; u < RL; ++u) {
      hi[u] = __shfl_down_sync(HM_FULL, acc.v[u].hi, off * G);
      lo[u] = __shfl_down_sync(HM_FULL, acc.v[u].lo, off * G);
    }
    if ((slot & (2 * off - 1)) == 0 && slot + off < S) {
#pragma unroll
      for (int u = 0; u < RL; ++u) acc.v[u] = ff_add(acc.v[u], FF{hi[u], lo[u]});
    }
  }
  const bool mine = lane < G;   // slot 0 lanes hold the chunk's rows RL q .. RL q + RL-1
  const int nr = mine ? min(RL, R - RL * q) : 0;
  const bool calpha = (hflags & PH_CALPHA) != 0;
  if (!(hflags & 0x10000)) {   // not shared with other warps
    if (nr > 0) rs_store_rows<MODE, RL>(acc, row0 + RL * q, nr, alpha_ff, beta, y, perm, vout, rowscale, calpha);
    return true;
  }
  const Split sp = splits[split];
  F2* mypart = fix + (size_t)(sp.slot0 + pidx) * CHUNK_ROWS + RL * q;   // split, pidx: from the piece's split / part word
#pragma unroll
  for (int u = 0; u < RL; ++u)
    if (u < nr) mypart[u] = F2{acc.v[u].hi, acc.v[u].lo};
  __syncwarp();   // the part's rows before lane 0's release
  int last = 0;
  if (lane == 0) last = atom_add_acq_rel(&fixcnt[split], 1) == sp.nparts - 1;
  last = __shfl_sync(HM_FULL, last, 0);
  if (!last) return false;
  __syncwarp();   // lane 0's acquire before the lanes read the other parts
  if (nr > 0) {
#pragma unroll
    for (int u = 0; u < RL; ++u) acc.v[u] = FF{0.f, 0.f};
    const F2* base = fix + (size_t)sp.slot0 * CHUNK_ROWS + RL * q;
    for (int k = 0; k < sp.nparts; ++k) {   // the rows of one part: independent loads, then the sums
      float2 v[RL];
#pragma unroll
      for (int u = 0; u < RL; ++u)
        v[u] = u < nr ? __ldcg(reinterpret_cast<const float2*>(base + (size_t)k * CHUNK_ROWS + u))
                      : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < RL; ++u) acc.v[u] = ff_add(acc.v[u], FF{v[u].x, v[u].y});
    }
    rs_store_rows<MODE, RL>(acc, row0 + RL * q, nr, alpha_ff, beta, y, perm, vout, rowscale, calpha);
  }
  if (lane == 0) fixcnt[split] = 0;   // ready for the next product
  return true;
}

// Arguments of the row-chunk products shared by every range of a launch.
struct RsArgs {
  const PieceCopy* cps;
  const uint8_t* pay;
  const float2* vec;
  double alpha;
  F2 alpha_ff;
  double beta;
  double* y;
  const int32_t* perm;
  float2* vout;
  const F2* rowscale;
  F2* fix;
  int32_t* fixcnt;
  const Split* splits;
  int* err;
};

// Dataflow state of a persistent launch: per-piece dependencies, versions of
// the coefficient chunks, and an abort word (set on the first timeout, so that
// every other wait gives up at once).
struct DfArgs {
  const SeqDep* deps;
  unsigned* ver;
  int* abort;
  unsigned* claim;   // per phase: ranges handed out so far
};

// Wait (lane 0, bounded) until chunk c has reached version v; acquire.
__device__ __forceinline__ bool wait_version(const DfArgs& D, int c, int v) {
  if (c < 0 || v <= 0) return true;
  for (uint32_t i = 0; i < (1u << 22); ++i) {   // each try is an L2 round trip: about 2 s in all
    unsigned x;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(x) : "l"(D.ver + c) : "memory");
    if ((int)x >= v) return true;
    if ((i & 255u) == 255u && *(volatile int*)D.abort) return false;
  }
  atomicExch(D.abort, 1);
  return false;
}

// One warp's range of row-chunk pieces [p0, p0 + n): a ring of NS shared-memory
// stages filled by bulk copies (piece + its multiplier run), decoded and summed
// into float-float row sums, emitted at the end of each chunk.  it counts the
// stages this warp has used before (their mbarrier phases), and is advanced.
// DF (persistent launches): a piece's payload is copied at once, its
// multipliers only after the chunks it depends on have reached their versions;
// every emit of a coefficient chunk then publishes the next version.
// Returns false if a copy or a dependency did not arrive in time (error latched).
template <int TIER, int MODE, int NS, bool DF = false>
__device__ __forceinline__ bool rs_range(const RsArgs& A, int p0, int n, uint8_t* ring, int4* info,
                                         uint64_t* bars, int lane, uint32_t& it, const DfArgs* D = nullptr) {
  const uint32_t sring = smem_u32(ring);
  const PieceCopy zero{0, 0, 0, -1};
  PieceCopy dc = lane < n ? A.cps[p0 + lane] : zero;
  PieceCopy dn = 32 + lane < n ? A.cps[p0 + 32 + lane] : zero;
  int dbase = 0, issued = 0;
  const uint64_t pol = policy_evict_first();
  const uint32_t it0 = it;
  auto issue = [&](int i) {   // all lanes; copies piece i and its multipliers into stage (it0 + i) % NS
    if (i - dbase >= 32) {
      dc = dn;
      dbase += 32;
      dn = dbase + 32 + lane < n ? A.cps[p0 + dbase + 32 + lane] : zero;
    }
    const int sl = i - dbase;
    const uint32_t off16 = __shfl_sync(HM_FULL, dc.off16, sl);
    const uint32_t bf = __shfl_sync(HM_FULL, dc.bytes_flags, sl);
    const int32_t moff = __shfl_sync(HM_FULL, dc.moff, sl);
    const int32_t sp = __shfl_sync(HM_FULL, dc.split_part, sl);
    if (lane == 0) {
      const uint32_t st_i = (it0 + (uint32_t)i) % NS;
      uint8_t* st = ring + st_i * C_STAGE;
      uint64_t* bar = &bars[st_i];
      const uint32_t nc = bf >> 24;
      const uint32_t pb = pad16u(bf & 0xffffu);
      const int64_t m0 = (int64_t)moff & ~int64_t(1);
      const uint32_t mb = nc ? pad16u((uint32_t)((moff - m0) + nc) * 8u) : 0u;
      int ce = -1;
      fence_proxy_async();
      mbar_expect_tx(bar, pb + mb);
      bulk_g2s_hint(st, A.pay + (uint64_t)off16 * 16u, pb, bar, pol);
      if constexpr (DF) {
        const SeqDep d = D->deps[p0 + i];
        ce = d.c1;
        if (!(wait_version(*D, d.c0, d.v0) && wait_version(*D, d.c1, d.v1))) latch_error(A.err, 99);
        asm volatile("fence.proxy.async.global;" ::: "memory");   // the multipliers were written by other SMs
      }
      info[st_i] = make_int4((int)((bf >> 16) & 0xffu), sp, moff & 1, ce);
      if (mb) bulk_g2s(st + C_MOFF, A.vec + m0, mb, bar);   // issued even after a failed wait: the stage completes
    }
    if constexpr (DF) __syncwarp();   // lane 0's acquires before the lanes' reads of this piece's chunk
    issued = i + 1;
  };
  for (int i = 0; i < NS && i < n; ++i) issue(i);
  constexpr int RL = RPL;   // rows per lane
  float2 ahi[4], alo[4];     // float-float row sums, rows (2k, 2k+1)
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ahi[k] = make_float2(0.f, 0.f);
    alo[k] = make_float2(0.f, 0.f);
  }
  for (int i = 0; i < n; ++i) {
    const uint32_t u = it0 + (uint32_t)i;
    const uint32_t s = u % NS;
    if (!mbar_wait(&bars[s], (u / NS) & 1u)) {
      latch_error(A.err, 99);
      if constexpr (DF) {
        if (lane == 0) atomicExch(D->abort, 1);
      }
      drain<NS>(bars, i + 1, issued, it0);
      it = it0 + (uint32_t)issued;
      return false;
    }
    const uint32_t sa = sring + s * (uint32_t)C_STAGE;
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
      H.scale = F2{__uint_as_float(b.z), __uint_as_float(b.w)};
    }
    const int4 rinfo = info[s];   // range flags, split / part, multiplier parity of this piece
    if (rinfo.x & PD_FIRST) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ahi[k] = make_float2(0.f, 0.f);
        alo[k] = make_float2(0.f, 0.f);
      }
    }
    const uint32_t tbl = sa + C_MOFF + 8u * (uint32_t)rinfo.z;
    switch (H.fb) {
#define HM_RS(FF_, BB_) \
  case ((FF_) << 4) | (BB_): rs_piece<TIER, FF_, BB_>(sa, H, tbl, A.alpha_ff, lane, ahi, alo); break;
      HM_FORMATS(HM_RS)
#undef HM_RS
      default:
        latch_error(A.err, 2);
    }
    if (rinfo.x & PD_LAST) {
      AccR<RL> a8;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        a8.v[2 * k] = FF{ahi[k].x, alo[k].x};
        a8.v[2 * k + 1] = FF{ahi[k].y, alo[k].y};
      }
      const bool wrote =
          rs_emit<MODE, RL>(a8, H.row0, H.nrows, H.flags | ((rinfo.x & PD_SPLIT) ? 0x10000 : 0), rinfo.y >> 8,
                            rinfo.y & 0xff, lane, A.alpha_ff, A.beta, A.y, A.perm, A.vout, A.rowscale, A.fix,
                            A.fixcnt, A.splits);
      if constexpr (DF) {
        if (wrote && rinfo.w >= 0) {   // publish the chunk's next version after all lanes' stores
          __syncwarp();
          if (lane == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(D->ver + rinfo.w) : "memory");
        }
      }
    }
    __syncwarp();
    if (issued < n) issue(issued);
  }
  it = it0 + (uint32_t)n;
  return true;
}

template <int NW, int NS>
__device__ __forceinline__ void rs_ring_init(uint8_t*& ring, int4*& info, uint64_t*& bars, int warp, int lane) {
  extern __shared__ __align__(128) uint8_t smem[];
  ring = smem + (size_t)warp * NS * C_STAGE;
  info = reinterpret_cast<int4*>(smem + (size_t)NW * NS * C_STAGE) + warp * NS;
  bars = reinterpret_cast<uint64_t*>(smem + (size_t)NW * NS * (C_STAGE + C_INFO)) + warp * NS;
  if (lane == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    mbar_init_fence();
  }
  __syncwarp();
}

template <int TIER, int MODE, int NW, int NS>
__global__ void __launch_bounds__(NW * 32, 1)
    k_rstream(RsArgs A, const int32_t* __restrict__ wbeg, int nwt) {
  pdl_trigger();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * NW + warp;
  if (gw >= nwt) return;
  const int p0 = wbeg[gw], n = wbeg[gw + 1] - p0;
  if (n <= 0) return;
  uint8_t* ring;
  int4* info;
  uint64_t* bars;
  rs_ring_init<NW, NS>(ring, info, bars, warp, lane);
  pdl_wait();   // multipliers and outputs depend on the previous kernels
  uint32_t it = 0;
  rs_range<TIER, MODE, NS>(A, p0, n, ring, info, bars, lane, it);
}

// ---------------------------------------------------------------- persistent phases
// A run of row-chunk launches (the levels of the sweeps, the couplings) as the
// phases of one cooperative launch (all warps resident): the warp ranges of a
// phase are handed out in order from a counter to whichever warp is free (a
// warp takes phase p + 1 ranges once phase p has none left), and each piece
// waits only for the coefficient chunks it reads (versions published by the
// emits of earlier phases), so the levels of different subtrees overlap and a
// warp held up by a dependency does not hold up the ranges behind it.  A warp
// holds one range at a time and only waits for chunks of earlier phases, which
// are held by running warps: no cycle.
template <int TIER, int NW, int NS>
__global__ void __launch_bounds__(NW * 32, 1)
    k_rseq(RsArgs A, const SeqPhase* __restrict__ ph, int nph, const int32_t* __restrict__ wbeg,
           const F2* __restrict__ rowscale, DfArgs D) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t* ring;
  int4* info;
  uint64_t* bars;
  rs_ring_init<NW, NS>(ring, info, bars, warp, lane);
  uint32_t it = 0;
  for (int p = 0; p < nph; ++p) {
    const SeqPhase P = ph[p];
    RsArgs B = A;
    B.rowscale = P.rowscale ? rowscale : nullptr;
    for (;;) {   // ranges of this phase are handed out in order to whichever warp is free
      int r = 0;
      if (lane == 0) r = (int)atomicAdd(D.claim + p, 1u);
      r = __shfl_sync(HM_FULL, r, 0);
      if (r >= P.nw) break;
      const int p0 = wbeg[P.woff + r], n = wbeg[P.woff + r + 1] - p0;
      if (n <= 0) continue;
      bool ok;
      if (P.mode == MODE_Y)
        ok = rs_range<TIER, MODE_Y, NS, true>(B, p0, n, ring, info, bars, lane, it, &D);
      else if (P.mode == MODE_VEC)
        ok = rs_range<TIER, MODE_VEC, NS, true>(B, p0, n, ring, info, bars, lane, it, &D);
      else
        ok = rs_range<TIER, MODE_VEC_ADD, NS, true>(B, p0, n, ring, info, bars, lane, it, &D);
      if (!ok) return;
    }
  }
}

// ---------------------------------------------------------------- multiplier fan-out
// Slot i of a row-chunk launch's multiplier runs takes coefficient v[src[i]].
// FAN_PER slots per thread, all index loads, then all gathers, then all stores
// (few waves of threads, several loads in flight per thread).
constexpr int FAN_PER = 4;
// Slots [base, base + FAN_PER * stride) of thread `base`: the fan-out work of one thread.
__device__ __forceinline__ void fanout_one(const int32_t* __restrict__ src, int n, float2* __restrict__ dst,
                                           const float2* __restrict__ vec, int base, int stride) {
  int ix[FAN_PER];
#pragma unroll
  for (int k = 0; k < FAN_PER; ++k) {
    const int i = base + k * stride;
    ix[k] = i < n ? __ldg(src + i) : -1;
  }
  float2 v[FAN_PER];
#pragma unroll
  for (int k = 0; k < FAN_PER; ++k) v[k] = ix[k] >= 0 ? vec[ix[k]] : make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < FAN_PER; ++k)
    if (ix[k] >= 0) dst[base + k * stride] = v[k];
}

__global__ void k_fanout(const int32_t* __restrict__ src, int n, float2* __restrict__ dst,
                         const float2* __restrict__ vec) {
  pdl_trigger();
  pdl_wait();
  fanout_one(src, n, dst, vec, blockIdx.x * blockDim.x * FAN_PER + threadIdx.x, blockDim.x);
}

// ---------------------------------------------------------------- segment sums (phase A2)
// Segment sums: GS_LANES lanes per output; lane k sums the partials p0 + k,
// p0 + k + GS_LANES, ... (consecutive lanes read consecutive partials), then a
// fixed xor tree combines the lanes (deterministic order).
constexpr int GS_LANES = 4;
// Output t / GS_LANES, lane t % GS_LANES of its group (whole warps call this).
// fan_dst non-null: a folded fan-out -- the group also writes the output's
// slots fan_dst[O.pad .. O.pad + (O.flags >> 8)) (lane k: slots k, k + 8, ...;
// the first slot index is loaded beside the partials).
__device__ __forceinline__ void gsum_one(const GsumOut* __restrict__ outs, int nouts, const F2* __restrict__ pscale,
                                         const F2* __restrict__ partial, F2 alpha, float2* __restrict__ vout,
                                         const int32_t* __restrict__ fan_dst, int64_t t) {
  const int64_t i = t / GS_LANES;
  const int k = (int)(t % GS_LANES);
  const bool on = i < nouts;
  GsumOut O{};
  if (on) O = outs[i];
  const int nslot = fan_dst ? (O.flags >> 8) : 0;
  const int32_t slot0 = k < nslot ? fan_dst[O.pad + k] : -1;
  FF s = {0.f, 0.f};
  // (unrolled: several partials in flight per lane; the sum order is unchanged)
  if (O.flags & 2) {
#pragma unroll 4
    for (int p = O.p0 + k; p < O.p1; p += GS_LANES) {
      const F2 v = partial[p];
      const F2 w = pscale[O.ps + (p - O.p0)];
      s = ff_add(s, ff_mul(FF{v.hi, v.lo}, FF{w.hi, w.lo}));
    }
  } else {
#pragma unroll 4
    for (int p = O.p0 + k; p < O.p1; p += GS_LANES) {
      const F2 v = partial[p];
      s = ff_add(s, FF{v.hi, v.lo});
    }
  }
#pragma unroll
  for (int m = GS_LANES / 2; m >= 1; m >>= 1) {   // whole warps: every lane takes part
    const float hi = __shfl_xor_sync(HM_FULL, s.hi, m);
    const float lo = __shfl_xor_sync(HM_FULL, s.lo, m);
    s = (k & m) ? ff_add(FF{hi, lo}, s) : ff_add(s, FF{hi, lo});
  }
  if (!on) return;
  if (nslot == 0 && k != 0) return;
  // every lane of the group holds the same sum: lane 0 writes the coefficient,
  // the group its slots
  s = ff_mul(s, FF{O.scale.hi, O.scale.lo});
  if (O.flags & 1) s = ff_mul(s, FF{alpha.hi, alpha.lo});
  const float2 val = make_float2(s.hi, s.lo);
  if (k == 0) vout[O.out] = val;
  if (slot0 >= 0) vout[slot0] = val;
  for (int q = k + GS_LANES; q < nslot; q += GS_LANES) vout[fan_dst[O.pad + q]] = val;
}

// Copy entries of a folded fan-out: slot cdst[i] takes v[csrc[i]] (FAN_PER per
// thread: all index loads, then the gathers, then the stores).
__device__ __forceinline__ void fcopy_one(const int32_t* __restrict__ csrc, const int32_t* __restrict__ cdst, int n,
                                          float2* __restrict__ vec, int base, int stride) {
  int ix[FAN_PER], dx[FAN_PER];
#pragma unroll
  for (int q = 0; q < FAN_PER; ++q) {
    const int i = base + q * stride;
    ix[q] = i < n ? __ldg(csrc + i) : -1;
    dx[q] = i < n ? __ldg(cdst + i) : -1;
  }
  float2 v[FAN_PER];
#pragma unroll
  for (int q = 0; q < FAN_PER; ++q) v[q] = ix[q] >= 0 ? vec[ix[q]] : make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < FAN_PER; ++q)
    if (ix[q] >= 0) vec[dx[q]] = v[q];
}

// Blocks [0, gblocks) take the segment sums; the rest the copy entries of a
// folded fan-out (ncopy of them).
__global__ void k_gsum(const GsumOut* __restrict__ outs, int nouts, const F2* __restrict__ pscale,
                       const F2* __restrict__ partial, F2 alpha, float2* __restrict__ vout,
                       const int32_t* __restrict__ fan_dst, const int32_t* __restrict__ csrc,
                       const int32_t* __restrict__ cdst, int ncopy, int gblocks) {
  pdl_trigger();
  pdl_wait();
  if ((int)blockIdx.x < gblocks)
    gsum_one(outs, nouts, pscale, partial, alpha, vout, fan_dst, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  else
    fcopy_one(csrc, cdst, ncopy, vout, ((int)blockIdx.x - gblocks) * blockDim.x * FAN_PER + threadIdx.x, blockDim.x);
}

// ---------------------------------------------------------------- gather x
__global__ void k_gather(const double* __restrict__ x, const int32_t* __restrict__ perm, int n,
                         float2* __restrict__ xo) {
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  FF f = ff_from_d(x[perm[i]]);
  xo[i] = make_float2(f.hi, f.lo);
}

constexpr int SEQ_NW = RS_CFG_WARPS[SEQ_SHAPE], SEQ_NS = RS_CFG_STAGES[SEQ_SHAPE];   // persistent phases

// ---------------------------------------------------------------- the whole product as one launch
// All launches of a product (gather, column dots, segment sums, fan-outs, row
// chunks) as the phases of ONE cooperative launch of SEQ_NW warps per block,
// one block per SM.  Phases follow each other at grid barriers (every warp of
// every block takes part in each barrier, also after an error, so none can be
// left waiting); a run of row-chunk launches is one dataflow phase as in
// k_rseq.  The column-dot and row-chunk phases use the warp ranges of launch
// shape 0, so the result equals the per-launch path with shape 0 bit for bit.
struct ProgArgs {
  const ProgPhase* phases;
  int nphases;
  const double* x;
  const ItemCopy* items;
  const GsumOut* gouts;
  const F2* pscale;
  F2* partial;
  const int32_t* fan;
  const int32_t* wbeg;
  const SeqPhase* seqph;
  const SeqDep* deps;
  unsigned* state;     // [0]: barrier counter, [1]: abort word, then the runs' versions / abort / claims
  const F2* rowscale;
  const int32_t* fan_dst;       // folded fan-outs (segment-sum phases with aux = 1)
  const int32_t* fan_copy_src;
  const int32_t* fan_copy_dst;
};

// Grid barrier number b (0, 1, ...): the block's warps meet, thread 0 publishes
// the block's writes (gpu-scope fence) and waits (bounded) until every block
// has arrived; the warps then see every block's writes.  False after a timeout
// or an abort elsewhere (the abort word is set, every later wait gives up).
__device__ bool prog_barrier(unsigned* state, unsigned target) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(state, 1u);
    for (uint32_t i = 0;; ++i) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(state) : "memory");
      if (v >= target) break;
      if (*(volatile int*)(state + 1) || i >= (1u << 22)) {   // about 2 s of L2 round trips
        atomicExch(reinterpret_cast<int*>(state + 1), 1);
        ok = 0;
        break;
      }
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");   // later bulk copies read what other SMs wrote
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// The range loops of the phases, out of line: each keeps the register
// allocation it has in its own kernel instead of sharing one across all phases.
template <int TIER>
__device__ __noinline__ bool prog_cs(const CsArgs& C, int p0, int n, uint8_t* ring, uint64_t* bars, int lane,
                                     uint32_t& it) {
  return cs_range<TIER, SEQ_NS, C_STAGE>(C, p0, n, ring, bars, lane, it);
}

template <int TIER, int MODE, bool DF>
__device__ __noinline__ bool prog_rs(const RsArgs& B, int p0, int n, uint8_t* ring, int4* info, uint64_t* bars,
                                     int lane, uint32_t& it, const DfArgs* D) {
  return rs_range<TIER, MODE, SEQ_NS, DF>(B, p0, n, ring, info, bars, lane, it, D);
}

template <int TIER>
__global__ void __launch_bounds__(SEQ_NW * 32, 1) k_prog(RsArgs A, ProgArgs P) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * SEQ_NW + warp, nwarps = gridDim.x * SEQ_NW;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthreads = (int64_t)gridDim.x * blockDim.x;
  uint8_t* ring;
  int4* info;
  uint64_t* bars;
  rs_ring_init<SEQ_NW, SEQ_NS>(ring, info, bars, warp, lane);
  uint32_t it = 0;
  bool good = true;        // this warp has not hit a timeout
  unsigned nbar = 0;
  const CsArgs C{P.items, A.pay, A.vec, A.alpha_ff, P.partial, A.vout, A.err};
  for (int p = 0; p < P.nphases; ++p) {
    const ProgPhase Ph = P.phases[p];
    if (good && !*(volatile int*)(P.state + 1)) {
      switch (Ph.kind) {
        case PP_GATHER:
          for (int64_t i = gtid; i < Ph.n; i += nthreads) {
            const FF f = ff_from_d(P.x[A.perm[i]]);
            A.vout[i] = make_float2(f.hi, f.lo);
          }
          break;
        case PP_CDOT:
          for (int r = gw; r < Ph.n; r += nwarps) {
            const int p0 = P.wbeg[Ph.off + r], n = P.wbeg[Ph.off + r + 1] - p0;
            if (n > 0 && !prog_cs<TIER>(C, p0, n, ring, bars, lane, it)) good = false;
          }
          break;
        case PP_GSUM: {
          const int64_t total = (int64_t)Ph.n * GS_LANES;
          for (int64_t t0 = (int64_t)gw * 32; t0 < total; t0 += (int64_t)nwarps * 32)
            gsum_one(P.gouts + Ph.off, Ph.n, P.pscale, P.partial, A.alpha_ff, A.vout, Ph.aux ? P.fan_dst : nullptr,
                     t0 + lane);
          if (Ph.aux) {   // copy entries [mode, mode + nchunks) of the folded fan-out
            const int64_t per = (int64_t)blockDim.x * FAN_PER;
            for (int64_t c = blockIdx.x; c * per < Ph.nchunks; c += gridDim.x)
              fcopy_one(P.fan_copy_src + Ph.mode, P.fan_copy_dst + Ph.mode, Ph.nchunks, A.vout,
                        (int)(c * per) + threadIdx.x, blockDim.x);
          }
          break;
        }
        case PP_FANOUT: {
          const int64_t per = (int64_t)blockDim.x * FAN_PER;
          for (int64_t c = blockIdx.x; c * per < Ph.n; c += gridDim.x)
            fanout_one(P.fan + Ph.off, Ph.n, A.vout + Ph.aux + Ph.off, A.vec, (int)(c * per) + threadIdx.x,
                       blockDim.x);
          break;
        }
        case PP_RGEMV: {
          RsArgs B = A;
          B.rowscale = Ph.rowscale ? P.rowscale : nullptr;
          for (int r = gw; r < Ph.n && good; r += nwarps) {
            const int p0 = P.wbeg[Ph.off + r], n = P.wbeg[Ph.off + r + 1] - p0;
            if (n <= 0) continue;
            bool ok;
            if (Ph.mode == MODE_Y)
              ok = prog_rs<TIER, MODE_Y, false>(B, p0, n, ring, info, bars, lane, it, nullptr);
            else if (Ph.mode == MODE_VEC)
              ok = prog_rs<TIER, MODE_VEC, false>(B, p0, n, ring, info, bars, lane, it, nullptr);
            else
              ok = prog_rs<TIER, MODE_VEC_ADD, false>(B, p0, n, ring, info, bars, lane, it, nullptr);
            good = good && ok;
          }
          break;
        }
        case PP_RUN: {
          unsigned* st = P.state + Ph.aux;
          const DfArgs D{P.deps, st, reinterpret_cast<int*>(st + Ph.nchunks), st + Ph.nchunks + 1};
          for (int q = 0; q < Ph.n && good; ++q) {
            const SeqPhase S = P.seqph[Ph.off + q];
            RsArgs B = A;
            B.rowscale = S.rowscale ? P.rowscale : nullptr;
            for (;;) {   // ranges of this phase are handed out in order to whichever warp is free
              int r = 0;
              if (lane == 0) r = (int)atomicAdd(D.claim + q, 1u);
              r = __shfl_sync(HM_FULL, r, 0);
              if (r >= S.nw) break;
              const int p0 = P.wbeg[S.woff + r], n = P.wbeg[S.woff + r + 1] - p0;
              if (n <= 0) continue;
              bool ok;
              if (S.mode == MODE_Y)
                ok = prog_rs<TIER, MODE_Y, true>(B, p0, n, ring, info, bars, lane, it, &D);
              else if (S.mode == MODE_VEC)
                ok = prog_rs<TIER, MODE_VEC, true>(B, p0, n, ring, info, bars, lane, it, &D);
              else
                ok = prog_rs<TIER, MODE_VEC_ADD, true>(B, p0, n, ring, info, bars, lane, it, &D);
              if (!ok) {
                good = false;
                break;
              }
            }
          }
          break;
        }
        default:
          latch_error(A.err, 2);
      }
    }
    if (!good && lane == 0) atomicExch(reinterpret_cast<int*>(P.state + 1), 1);
    if (p + 1 < P.nphases && !prog_barrier(P.state, ++nbar * gridDim.x)) good = false;
  }
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

// ---------------------------------------------------------------- decoder check over the resident payload
// One task: 8 consecutive codes of one packed column (a lane's share in the
// product kernels), decoded by the same template instances the product kernels
// run -- decode8p (FP32 tier: column dots, row chunks, multi-RHS) or
// decode8s<TIER_FF> (float-float tier) -- from a per-thread shared-memory copy
// of the 8 B bytes, exactly as the kernels read them from their stages.
template <int TIER>
__global__ void k_decode_debug(const DbgTask* __restrict__ tasks, int64_t ntask, const uint8_t* __restrict__ pay,
                               float2* __restrict__ out, int* err) {
  __shared__ __align__(16) uint64_t buf[256 * 8];
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntask) return;
  const DbgTask T = tasks[t];
  const int fb = (int)(T.fbem & 0xffu), B = fb & 15;
  const int e = (int)((T.fbem >> 16) & 0xffu), m = (int)(T.fbem >> 24);
  const uint64_t* src = reinterpret_cast<const uint64_t*>(pay + T.off);
  uint64_t* dst = buf + threadIdx.x * 8;
  for (int i = 0; i < B && i < 8; ++i) dst[i] = src[i];
  const uint32_t a = smem_u32(dst);
  float h[8], l[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    h[u] = 0.f;
    l[u] = 0.f;
  }
  bool ok = true;
  if constexpr (TIER == TIER_F32) {
    float2 h2[4];
    switch (fb) {
#define HM_DD(FF_, BB_) \
  case ((FF_) << 4) | (BB_): decode8p<FF_, BB_>(a, e, m, h2); break;
      HM_FORMATS(HM_DD)
#undef HM_DD
      default:
        ok = false;
    }
    if (ok) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        h[2 * k] = h2[k].x;
        h[2 * k + 1] = h2[k].y;
      }
    }
  } else {
    switch (fb) {
#define HM_DD(FF_, BB_) \
  case ((FF_) << 4) | (BB_): decode8s<TIER_FF, FF_, BB_>(a, e, m, h, l); break;
      HM_FORMATS(HM_DD)
#undef HM_DD
      default:
        ok = false;
    }
  }
  if (!ok) {
    latch_error(err, 1);
    return;
  }
#pragma unroll
  for (int u = 0; u < 8; ++u)
    if (u < T.nr) out[T.out + u] = make_float2(h[u], l[u]);
}

// ---------------------------------------------------------------- launchers
// Launch with programmatic stream serialization (see pdl_trigger / pdl_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}
template <int NW, int NS>
constexpr size_t cs_smem() {
  return (size_t)NW * NS * (A_STAGE + 8) + SMEM_TAIL;
}
template <int NW, int NS>
constexpr size_t rs_smem() {
  return (size_t)NW * NS * (C_STAGE + C_INFO + 8) + SMEM_TAIL;
}
#define HM_CS_CFGS(X) X(0, 16, 2) X(1, 10, 3) X(2, 7, 4)
#define HM_RS_CFGS(X) X(0, 16, 2) X(1, 11, 3) X(2, 8, 4)
#define HM_CHK_CS(I, NW, NS)                                                                      \
  static_assert(CS_CFG_WARPS[I] == NW && CS_CFG_STAGES[I] == NS, "column-dot launch shapes");     \
  static_assert(cs_smem<NW, NS>() <= 227 * 1024, "shared memory per block");
#define HM_CHK_RS(I, NW, NS)                                                                      \
  static_assert(RS_CFG_WARPS[I] == NW && RS_CFG_STAGES[I] == NS, "row-chunk launch shapes");      \
  static_assert(rs_smem<NW, NS>() <= 227 * 1024, "shared memory per block");
HM_CS_CFGS(HM_CHK_CS)
HM_RS_CFGS(HM_CHK_RS)
#undef HM_CHK_CS
#undef HM_CHK_RS

cudaError_t kernels_init() {
  cudaError_t e = cudaSuccess;
#define HM_ATTR(K, SM) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SM));
#define HM_INIT_CS(I, NW, NS)                                                \
  HM_ATTR((k_cstream<TIER_F32, NW, NS>), (cs_smem<NW, NS>()))                \
  HM_ATTR((k_cstream<TIER_FF, NW, NS>), (cs_smem<NW, NS>()))
#define HM_INIT(I, NW, NS)                                                   \
  HM_ATTR((k_rstream<TIER_F32, MODE_Y, NW, NS>), (rs_smem<NW, NS>()))        \
  HM_ATTR((k_rstream<TIER_F32, MODE_VEC, NW, NS>), (rs_smem<NW, NS>()))      \
  HM_ATTR((k_rstream<TIER_F32, MODE_VEC_ADD, NW, NS>), (rs_smem<NW, NS>()))  \
  HM_ATTR((k_rstream<TIER_FF, MODE_Y, NW, NS>), (rs_smem<NW, NS>()))         \
  HM_ATTR((k_rstream<TIER_FF, MODE_VEC, NW, NS>), (rs_smem<NW, NS>()))       \
  HM_ATTR((k_rstream<TIER_FF, MODE_VEC_ADD, NW, NS>), (rs_smem<NW, NS>()))
  HM_CS_CFGS(HM_INIT_CS)
  HM_RS_CFGS(HM_INIT)
  HM_ATTR((k_rseq<TIER_F32, SEQ_NW, SEQ_NS>), (rs_smem<SEQ_NW, SEQ_NS>()))
  HM_ATTR((k_rseq<TIER_FF, SEQ_NW, SEQ_NS>), (rs_smem<SEQ_NW, SEQ_NS>()))
  HM_ATTR((k_prog<TIER_F32>), (rs_smem<SEQ_NW, SEQ_NS>()))
  HM_ATTR((k_prog<TIER_FF>), (rs_smem<SEQ_NW, SEQ_NS>()))
#undef HM_INIT_CS
#undef HM_INIT
#undef HM_ATTR
  return e;
}

cudaError_t launch_gather(const double* x, const int32_t* perm, int n, float2* xo, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<(n + 255) / 256, 256, 0, st>>>(x, perm, n, xo);
  return cudaGetLastError();
}

template <int NW, int NS>
cudaError_t cdot_shape(int tier, const ItemCopy* items, const int32_t* wbeg, int nw, const uint8_t* pay, const float2* vec,
                F2 alpha, F2* partial, float2* vout, int* err, cudaStream_t st) {
  const int grid = (nw + NW - 1) / NW;
  if (tier == TIER_F32)
    return launch_pdl(k_cstream<TIER_F32, NW, NS>, grid, NW * 32, cs_smem<NW, NS>(), st, items, wbeg, nw, pay, vec,
                      alpha, partial, vout, err);
  return launch_pdl(k_cstream<TIER_FF, NW, NS>, grid, NW * 32, cs_smem<NW, NS>(), st, items, wbeg, nw, pay, vec,
                    alpha, partial, vout, err);
}

cudaError_t launch_cdot(int tier, int cfg, const ItemCopy* items, const int32_t* wbeg, int nw, const uint8_t* pay,
                        const float2* vec, F2 alpha, F2* partial, float2* vout, int* err, cudaStream_t st) {
  if (nw <= 0) return cudaSuccess;
  switch (cfg) {
#define HM_L(I, NW, NS)                                                                            \
  case I: {                                                                                        \
    const cudaError_t e = cdot_shape<NW, NS>(tier, items, wbeg, nw, pay, vec, alpha, partial, vout, err, st); \
    if (e != cudaSuccess) return e;                                                                \
    break;                                                                                         \
  }
    HM_CS_CFGS(HM_L)
#undef HM_L
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fanout(const int32_t* src, int n, float2* dst, const float2* vec, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const cudaError_t e = launch_pdl(k_fanout, (unsigned)((n + 256 * FAN_PER - 1) / (256 * FAN_PER)), 256, 0, st, src,
                                   n, dst, vec);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_gsum(const GsumOut* outs, int nouts, const F2* pscale, const F2* partial, F2 alpha, float2* vout,
                        const int32_t* fan_dst, const int32_t* csrc, const int32_t* cdst, int ncopy, cudaStream_t st) {
  if (nouts <= 0 && ncopy <= 0) return cudaSuccess;
  const int64_t threads = (int64_t)nouts * GS_LANES;
  const int gblocks = (int)((threads + 255) / 256), cblocks = (ncopy + 256 * FAN_PER - 1) / (256 * FAN_PER);
  const cudaError_t e = launch_pdl(k_gsum, (unsigned)(gblocks + cblocks), 256, 0, st, outs, nouts, pscale, partial,
                                   alpha, vout, fan_dst, csrc, cdst, ncopy, gblocks);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int NW, int NS>
cudaError_t rgemv_shape(int tier, int mode, const PieceCopy* pieces, const int32_t* wbeg, int nw, const uint8_t* pay,
                 const float2* vec, double alpha, F2 alpha_ff, double beta, double* y, const int32_t* perm,
                 float2* vout, const F2* rowscale, F2* fix, int32_t* fixcnt, const Split* splits, int* err,
                 cudaStream_t st) {
  const int grid = (nw + NW - 1) / NW;
  const RsArgs A{pieces, pay, vec, alpha, alpha_ff, beta, y, perm, vout, rowscale, fix, fixcnt, splits, err};
#define HM_RG(T, M) launch_pdl(k_rstream<T, M, NW, NS>, grid, NW * 32, rs_smem<NW, NS>(), st, A, wbeg, nw)
  if (tier == TIER_F32) {
    if (mode == MODE_Y) return HM_RG(TIER_F32, MODE_Y);
    if (mode == MODE_VEC) return HM_RG(TIER_F32, MODE_VEC);
    return HM_RG(TIER_F32, MODE_VEC_ADD);
  }
  if (mode == MODE_Y) return HM_RG(TIER_FF, MODE_Y);
  if (mode == MODE_VEC) return HM_RG(TIER_FF, MODE_VEC);
  return HM_RG(TIER_FF, MODE_VEC_ADD);
#undef HM_RG
}

cudaError_t launch_rgemv(int tier, int mode, int cfg, const PieceCopy* pieces, const int32_t* wbeg, int nw,
                         const uint8_t* pay, const float2* vec, double alpha, F2 alpha_ff, double beta, double* y,
                         const int32_t* perm, float2* vout, const F2* rowscale, F2* fix, int32_t* fixcnt,
                         const Split* splits, int* err, cudaStream_t st) {
  if (nw <= 0) return cudaSuccess;
  switch (cfg) {
#define HM_L(I, NW, NS)                                                                                    \
  case I: {                                                                                                \
    const cudaError_t e = rgemv_shape<NW, NS>(tier, mode, pieces, wbeg, nw, pay, vec, alpha, alpha_ff, beta, y, \
                                              perm, vout, rowscale, fix, fixcnt, splits, err, st);           \
    if (e != cudaSuccess) return e;                                                                        \
    break;                                                                                                 \
  }
    HM_RS_CFGS(HM_L)
#undef HM_L
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// A run of row-chunk launches as one cooperative launch of nblk blocks (one
// per SM) of the persistent shape; the chunk versions, the abort word and the
// per-phase range counters (ver[0 .. nchunks + nph]) are zeroed first.
cudaError_t launch_rseq(int tier, int nblk, const SeqPhase* phases, int nph, const PieceCopy* pieces,
                        const int32_t* wbeg, const uint8_t* pay, float2* vec, double alpha, F2 alpha_ff, double beta,
                        double* y, const int32_t* perm, const F2* rowscale, F2* fix, int32_t* fixcnt,
                        const Split* splits, const SeqDep* deps, unsigned* ver, int nchunks, int* err,
                        cudaStream_t st) {
  if (nph <= 0 || nblk <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(ver, 0, (size_t)(nchunks + 1 + nph) * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const RsArgs A{pieces, pay, vec, alpha, alpha_ff, beta, y, perm, vec, nullptr, fix, fixcnt, splits, err};
  const DfArgs D{deps, ver, reinterpret_cast<int*>(ver + nchunks), ver + nchunks + 1};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nblk);
  cfg.blockDim = dim3(SEQ_NW * 32);
  cfg.dynamicSmemBytes = rs_smem<SEQ_NW, SEQ_NS>();
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (tier == TIER_F32)
    e = cudaLaunchKernelEx(&cfg, k_rseq<TIER_F32, SEQ_NW, SEQ_NS>, A, phases, nph, wbeg, rowscale, D);
  else
    e = cudaLaunchKernelEx(&cfg, k_rseq<TIER_FF, SEQ_NW, SEQ_NS>, A, phases, nph, wbeg, rowscale, D);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// The whole product as one cooperative launch of nblk blocks (one per SM); the
// barrier counter, abort word and the runs' state (nstate words) are zeroed first.
cudaError_t launch_prog(int tier, int nblk, const ProgPhase* phases, int nphases, const double* x,
                        const ItemCopy* items, const GsumOut* gouts, const F2* pscale, F2* partial,
                        const int32_t* fan, const PieceCopy* pieces, const int32_t* wbeg, const SeqPhase* seqph,
                        const SeqDep* deps, unsigned* state, int nstate, const uint8_t* pay, float2* vec,
                        double alpha, double beta, double* y, const int32_t* perm, const F2* rowscale, F2* fix,
                        int32_t* fixcnt, const Split* splits, const int32_t* fan_dst, const int32_t* fan_copy_src,
                        const int32_t* fan_copy_dst, int* err, cudaStream_t st) {
  if (nphases <= 0 || nblk <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(state, 0, (size_t)nstate * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const F2 aff{(float)alpha, (float)(alpha - (double)(float)alpha)};
  const RsArgs A{pieces, pay, vec, alpha, aff, beta, y, perm, vec, nullptr, fix, fixcnt, splits, err};
  const ProgArgs P{phases, nphases, x,        items,   gouts,        pscale,      partial,
                   fan,    wbeg,    seqph,    deps,    state,        rowscale,    fan_dst,
                   fan_copy_src, fan_copy_dst};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nblk);
  cfg.blockDim = dim3(SEQ_NW * 32);
  cfg.dynamicSmemBytes = rs_smem<SEQ_NW, SEQ_NS>();
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (tier == TIER_F32)
    e = cudaLaunchKernelEx(&cfg, k_prog<TIER_F32>, A, P);
  else
    e = cudaLaunchKernelEx(&cfg, k_prog<TIER_FF>, A, P);
  return e != cudaSuccess ? e : cudaGetLastError();
}

int prog_max_blocks() {
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prog<TIER_F32>, SEQ_NW * 32,
                                                    rs_smem<SEQ_NW, SEQ_NS>()) != cudaSuccess)
    return 0;
  return per_sm * nsm;
}

// Blocks of the persistent launch that fit on the device at once (0 if none).
int rseq_max_blocks() {
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rseq<TIER_F32, SEQ_NW, SEQ_NS>, SEQ_NW * 32,
                                                    rs_smem<SEQ_NW, SEQ_NS>()) != cudaSuccess)
    return 0;
  return per_sm * nsm;
}

cudaError_t launch_decode(const uint8_t* p, int64_t n, int B, int fmt, int e, int m, double vmin,
                          double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_decode<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, n, B, fmt, e, m, vmin, out);
  return cudaGetLastError();
}

cudaError_t launch_decode_debug(int tier, const DbgTask* tasks, int64_t ntask, const uint8_t* pay, float2* out,
                                int* err, cudaStream_t st) {
  if (ntask <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((ntask + 255) / 256);
  if (tier == TIER_F32)
    k_decode_debug<TIER_F32><<<grid, 256, 0, st>>>(tasks, ntask, pay, out, err);
  else
    k_decode_debug<TIER_FF><<<grid, 256, 0, st>>>(tasks, ntask, pay, out, err);
  return cudaGetLastError();
}

}  // namespace hm
