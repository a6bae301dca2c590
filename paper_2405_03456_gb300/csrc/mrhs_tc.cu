// Multi-RHS row-chunk products on the 5th-generation tensor cores (tcgen05,
// FP32 tier): y (or a coefficient panel) := the chunk rows of A times the
// multiplier panel T, for panels of RP right-hand sides.
//
// One CTA owns MP_PAIRS consecutive ranges of pieces; its warps have fixed roles and hand work on
// through mbarriers (no block-wide barrier in the loop):
//  * warp 0 streams every piece (one bulk copy) and its multiplier rows (RP
//    values each, taken from the coefficient they stand for; 16-byte cp.async)
//    into a ring of TC_NS stages;
//  * 8 decode warps cut the piece's values ONCE into three exact BF16 limbs by
//    truncation (shared-memory limb tiles, MN-major canonical layout, no
//    swizzle) and the multipliers (times the tile scale) the same way, into one
//    of two tile buffers;
//  * warp 1 (one thread) issues the tcgen05.mma chains of a piece (M = 128
//    chunk rows, N = RP, K = 16 per instruction): the limb-order-0 product into
//    one TMEM accumulator, the products of orders 1 and 2 into a second, in one
//    of two accumulator buffers, and commits them;
//  * 8 fold warps read TMEM lane (= chunk row) and 16 right-hand sides each
//    (tcgen05.ld), fold the sum of both accumulators into float-float row sums
//    and, at the last piece of their part of a chunk, emit the rows (shared
//    chunks through the fix-up slots, last part in part order), as the other
//    row-chunk kernels.
// Piece i + 1 is decoded while the products of piece i run and piece i - 1 is
// folded.  Every wait is bounded; a wait that runs out latches the error and
// the role stops, the others run out in turn, and the CTA releases TMEM.
//
// Layouts (bytes): an operand core matrix is 8 K-rows x 16 B (8 M or N
// elements).  A limb tile: core (mi, ki) at mi * TC_ASBO + ki * TC_ALBO (SBO =
// M-direction stride 144 B, which keeps the 16-byte stores of 8 consecutive
// row groups in distinct banks; LBO = K-direction stride).  B limb tile: core
// (ni, ki) at ni * 128 + ki * TC_BLBO.  TMEM: 2 x 64 columns (double-buffered
// accumulators; columns 0..31 order 0, 32..63 orders 1 + 2).
#include <cstdint>
#include <cuda_runtime.h>

#include "decode.cuh"

namespace hm {

// warp roles: 0 copies, 1 tensor-core issue (and TMEM), 2 .. 9 decode, 10 .. 17 fold / emit
constexpr int TC_DEC0 = 2, TC_NDEC = 8, TC_EPI0 = TC_DEC0 + TC_NDEC, TC_NEPI = 8;
constexpr int TC_THREADS = 32 * (TC_EPI0 + TC_NEPI);
constexpr int TC_NS = 3;                                      // pieces in flight per CTA
constexpr int TC_TP = RP * 4 + 16;                            // multiplier row pitch in a stage
constexpr int TC_STAGE = STAGE_BYTES + PIECE_MAX_COLS * TC_TP;
constexpr int TC_ASBO = 144;                                  // A: M-direction core stride
constexpr int TC_ALBO = (CHUNK_ROWS / 8) * TC_ASBO;           // A: K-direction core stride
constexpr int TC_ATILE = (PIECE_MAX_COLS / 8) * TC_ALBO;      // one A limb tile
constexpr int TC_BSBO = 128;                                  // B: N-direction core stride
constexpr int TC_BLBO = (RP / 8) * TC_BSBO;                   // B: K-direction core stride
constexpr int TC_BTILE = (PIECE_MAX_COLS / 8) * TC_BLBO;      // one B limb tile
constexpr int TC_TILES = 3 * TC_ATILE + 3 * TC_BTILE;         // one buffer of limb tiles
constexpr size_t TC_SMEM = (size_t)TC_NS * TC_STAGE + 2 * (size_t)TC_TILES;
constexpr uint32_t TC_TMEM_COLS = 128;
static_assert(TC_STAGE % 128 == 0 && TC_ATILE % 128 == 0, "tile alignment");
static_assert(TC_SMEM + 1024 <= 227 * 1024, "one CTA per SM");
static_assert(CHUNK_ROWS == 128 && RP == 32 && PIECE_MAX_COLS % 16 == 0, "tile shape");
// instruction descriptor: D FP32, A and B BF16, both MN-major, N = RP, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                              ((uint32_t)(RP >> 3) << 17) | ((uint32_t)(CHUNK_ROWS >> 4) << 24);

// shared-memory matrix descriptor, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tc_ld16(uint32_t addr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(addr));
}

__device__ __forceinline__ void st_shared_v4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

// ceil(16384 / G): (t * c_tcdiv[G]) >> 14 == t / G for t < 16384 / G (t < 64 G, G <= 16)
__constant__ uint16_t c_tcdiv[17] = {0, 16384, 8192, 5462, 4096, 3277, 2731, 2341, 2048, 1821, 1639, 1490, 1366, 1261, 1171, 1093, 1024};

// Decode of the piece at shared address sa into the A limb tiles at sA by the
// decode warps (td = thread index among them): task (column j, row group q) writes rows 8 q .. 8 q + 7 of column j (one
// 16-byte core row per limb); columns nc .. ncp - 1 are zero.
template <int F, int B>
__device__ __forceinline__ void tc_decode(uint32_t sa, const PieceHdr& H, uint32_t sA, int ncp, int td) {
  const int R = H.nrows, nc = H.ncols, la = H.limbs;
  const bool tile = (H.flags & PH_TILE) != 0;
  const uint32_t stride = pad8u((uint32_t)R * B);
  const uint32_t cm = sa + (uint32_t)sizeof(PieceHdr);
  const uint32_t cb = cm + (tile ? 0u : pad8u(2u * nc));
  const int e_t = H.em & 0xff, m_t = H.em >> 8;
  const int G = (R + 7) >> 3;
  const int dG = (int)c_tcdiv[G];
  for (int task = td; task < ncp * G; task += 32 * TC_NDEC) {
    const int j = (task * dG) >> 14, q = task - j * G;
    uint32_t l0[4] = {0u, 0u, 0u, 0u}, l1[4] = {0u, 0u, 0u, 0u}, l2[4] = {0u, 0u, 0u, 0u};
    if (j < nc) {
      int e = e_t, m = m_t;
      if constexpr (F == 2) {
        if (!tile) {
          const uint32_t em = lds32((cm + 2u * j) & ~3u) >> (16u * (j & 1));
          e = em & 0xff;
          m = (em >> 8) & 0xff;
        }
      }
      float2 h2[4];
      decode8p<F, B>(cb + (uint32_t)j * stride + (uint32_t)(8 * q * B), e, m, h2);
#pragma unroll
      for (int u = 0; u < 4; ++u) limbs2(h2[u].x, h2[u].y, l0[u], l1[u], l2[u]);
    }
    const uint32_t a = sA + (uint32_t)(q * TC_ASBO + (j >> 3) * TC_ALBO + (j & 7) * 16);
    st_shared_v4(a, l0[0], l0[1], l0[2], l0[3]);
    if (la > 1) st_shared_v4(a + TC_ATILE, l1[0], l1[1], l1[2], l1[3]);
    if (la > 2) st_shared_v4(a + 2 * TC_ATILE, l2[0], l2[1], l2[2], l2[3]);
  }
}

// per-piece facts the later roles need: R, row0, flags, ncols | limbs << 16, PD flags, split part
struct TcInfo {
  int32_t R, row0, flags, ncl, pd, sp, pad0, pad1;
};

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_rgemv_tc(const PieceCopy* __restrict__ cps, const int32_t* __restrict__ wbeg, int nrange,
               const uint8_t* __restrict__ pay, const float* __restrict__ vec, double alpha, F2 alpha_ff,
               double beta, double* __restrict__ y, int64_t ldy, int r, const int32_t* __restrict__ perm,
               float* __restrict__ vout, const F2* __restrict__ rowscale, F2* __restrict__ fix,
               int32_t* __restrict__ fixcnt, const Split* __restrict__ splits, const int32_t* __restrict__ fan,
               int32_t fan_base, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ int4 info[TC_NS];                  // PD flags, split part of the piece in stage s
  __shared__ TcInfo tinfo[2], dinfo[2];         // the piece in tile buffer b / accumulator buffer b
  __shared__ __align__(8) uint64_t full[TC_NS], empty[TC_NS], tfull[2], tempty[2], dfull[2], dempty[2];
  __shared__ uint32_t tbase;
  __shared__ int s_last;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  // the CTA takes MP_PAIRS consecutive ranges as one stream of pieces (the
  // ranges' part flags still hold: a chunk part closed at a range end goes
  // through its fix-up slot like any other)
  const int r0 = blockIdx.x * MP_PAIRS, r1 = min(r0 + MP_PAIRS, nrange);
  if (r0 >= nrange) return;
  const int p0 = wbeg[r0], n = wbeg[r1] - p0;
  if (n <= 0) return;
  uint8_t* ring = smem;
  const uint32_t tiles0 = smem_u32(smem + (size_t)TC_NS * TC_STAGE);
  if (w == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int s = 0; s < TC_NS; ++s) {
      mbar_init(&full[s], 1 + 32);   // the payload's expect-tx arrival, one cp.async arrival per copy lane
      mbar_init(&empty[s], TC_NDEC);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], TC_NDEC);
      mbar_init(&tempty[b], 1);
      mbar_init(&dfull[b], 2);   // the commit and the issuing thread's arrive (after dinfo)
      mbar_init(&dempty[b], TC_NEPI);
    }
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  bool failed = false;
  if (w == 0) {
    // ---------------------------------------------------------------- copies
    const uint64_t pol = policy_evict_first();
    const PieceCopy zero{0, 0, 0, -1};
    PieceCopy dc = lane < n ? cps[p0 + lane] : zero;
    PieceCopy dn = 32 + lane < n ? cps[p0 + 32 + lane] : zero;
    int dbase = 0;
    // the sources of a piece's multiplier rows j = lane, lane + 32: vector
    // entries moff + j, or fan[moff - fan_base + j] for a fan-out run; loaded
    // one piece ahead so that their latency overlaps the copies of the piece before
    auto sources = [&](int i, int32_t (&src)[2]) {
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
    int32_t src[2];
    sources(0, src);
    for (int i = 0; i < n; ++i) {
      const int s = i % TC_NS;
      if (i >= TC_NS && !__all_sync(HM_FULL, mbar_wait(&empty[s], (uint32_t)(((i / TC_NS) + 1) & 1)))) {
        failed = true;
        break;
      }
      if (i - dbase >= 32) {
        dc = dn;
        dbase += 32;
        dn = dbase + 32 + lane < n ? cps[p0 + dbase + 32 + lane] : zero;
      }
      const int sl = i - dbase;
      const uint32_t off16 = __shfl_sync(HM_FULL, dc.off16, sl), bf = __shfl_sync(HM_FULL, dc.bytes_flags, sl);
      const int32_t sp = __shfl_sync(HM_FULL, dc.split_part, sl);
      uint8_t* st = ring + (size_t)s * TC_STAGE;
      const uint32_t nc = bf >> 24, pb = ((bf & 0xffffu) + 15u) & ~15u;
      fence_proxy_async();
      if (lane == 0) {
        info[s] = make_int4((int)((bf >> 16) & 0xffu), sp, 0, 0);
        mbar_expect_tx(&full[s], pb);
        bulk_g2s_hint(st, pay + (uint64_t)off16 * 16u, pb, &full[s], pol);
      }
      __syncwarp();
      // multiplier rows lane, lane + 32 by cp.async (one bulk copy per piece only)
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = lane + 32 * u;
        if (j < (int)nc) cp_row(smem_u32(st + STAGE_BYTES + j * TC_TP), vec + (int64_t)src[u] * RP);
      }
      cp_arrive(&full[s]);
      if (i + 1 < n) sources(i + 1, src);
    }
    if (failed && lane == 0) latch_error(err, 99);
    // copies still in flight land before the CTA exits (the decoders wait for them; bounded here too)
    if (lane == 0)
      for (int i = n - TC_NS < 0 ? 0 : n - TC_NS; i < n; ++i) mbar_wait(&full[i % TC_NS], (uint32_t)((i / TC_NS) & 1), failed ? 50u : 2000u);
  } else if (w == 1) {
    // ---------------------------------------------------------------- tensor-core issue
    if (lane == 0) {
      int i = 0;
      for (; i < n; ++i) {
        const int b = i & 1;
        if (!mbar_wait(&tfull[b], (uint32_t)((i >> 1) & 1)) ||
            (i >= 2 && !mbar_wait(&dempty[b], (uint32_t)(((i >> 1) + 1) & 1)))) {
          failed = true;
          break;
        }
        const TcInfo pi = tinfo[b];
        dinfo[b] = pi;
        const int nc = pi.ncl & 0xffff, ncp = (nc + 15) & ~15, la = pi.ncl >> 16;
        tc_fence_after();
        const uint32_t sA = tiles0 + (uint32_t)(b * TC_TILES), sB = sA + 3u * TC_ATILE;
        const uint32_t d = tmem + (uint32_t)(b * 64);
        for (int k = 0; k < ncp / 16; ++k) {
          uint64_t a[3], bd[3];
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            a[l] = tc_desc(sA + (uint32_t)(l * TC_ATILE + 2 * k * TC_ALBO), TC_ALBO, TC_ASBO);
            bd[l] = tc_desc(sB + (uint32_t)(l * TC_BTILE + 2 * k * TC_BLBO), TC_BLBO, TC_BSBO);
          }
          tc_mma(d, a[0], bd[0], k > 0);
          tc_mma(d + 32u, a[0], bd[1], k > 0);
          tc_mma(d + 32u, a[0], bd[2], 1u);
          if (la > 1) {
            tc_mma(d + 32u, a[1], bd[0], 1u);
            tc_mma(d + 32u, a[1], bd[1], 1u);
          }
          if (la > 2) tc_mma(d + 32u, a[2], bd[0], 1u);
        }
        // tiles b free once these products are done; accumulator b full then too
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&tempty[b]))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&dfull[b]))
                     : "memory");
        mbar_arrive(&dfull[b]);
      }
      if (failed) latch_error(err, 99);
      // products still in flight finish before TMEM is released (bounded)
      for (int j = i - 2; j < i; ++j)
        if (j >= 0) mbar_wait(&tempty[j & 1], (uint32_t)((j >> 1) & 1), failed ? 200u : 2000u);
    }
    __syncwarp();
  } else if (w < TC_EPI0) {
    // ---------------------------------------------------------------- decode
    const int td = t - 32 * TC_DEC0;   // 0 .. 32 TC_NDEC - 1
    for (int i = 0; i < n; ++i) {
      const int s = i % TC_NS, b = i & 1;
      const bool ok = mbar_wait(&full[s], (uint32_t)((i / TC_NS) & 1)) &&
                      (i < 2 || mbar_wait(&tempty[b], (uint32_t)(((i >> 1) + 1) & 1)));
      if (!__all_sync(HM_FULL, ok)) {
        failed = true;
        break;
      }
      const uint32_t sa = smem_u32(ring + (size_t)s * TC_STAGE);
      PieceHdr H;
      {
        const uint4 a = lds128(sa), bb = lds128(sa + 16);
        H.row0 = (int32_t)a.x;
        H.nrows = (uint16_t)(a.y & 0xffffu);
        H.flags = (uint16_t)(a.y >> 16);
        H.fb = (uint16_t)(a.z & 0xffffu);
        H.em = (uint16_t)(a.z >> 16);
        H.vin0 = (int32_t)a.w;
        H.ncols = (uint16_t)(bb.x & 0xffffu);
        H.limbs = (uint16_t)(bb.x >> 16);
        H.scale = F2{__uint_as_float(bb.z), __uint_as_float(bb.w)};
      }
      const int nc = H.ncols, ncp = (nc + 15) & ~15;
      const uint32_t sA = tiles0 + (uint32_t)(b * TC_TILES), sB = sA + 3u * TC_ATILE;
      switch (H.fb) {
#define HM_TD(FF_, BB_) \
  case ((FF_) << 4) | (BB_): tc_decode<FF_, BB_>(sa, H, sA, ncp, td); break;
        HM_FORMATS(HM_TD)
#undef HM_TD
        default:
          latch_error(err, 16);
      }
      {   // multipliers (times the tile scale): task (column j, rhs group ng of 8); zero past nc
        float sc = 1.0f;
        if (H.flags & PH_TILE) {
          FF f = {H.scale.hi, H.scale.lo};
          if (H.flags & PH_TALPHA) f = ff_mul(f, FF{alpha_ff.hi, alpha_ff.lo});
          sc = f.hi;
        }
        if (td < ncp * (RP / 8)) {
          const int j = td % ncp, ng = td / ncp;
          uint32_t l0[4] = {0u, 0u, 0u, 0u}, l1[4] = {0u, 0u, 0u, 0u}, l2[4] = {0u, 0u, 0u, 0u};
          if (j < nc) {
            const uint32_t ta = sa + STAGE_BYTES + (uint32_t)(j * TC_TP + 32 * ng);
            const uint4 a = lds128(ta), bb = lds128(ta + 16);
            limbs2(__uint_as_float(a.x) * sc, __uint_as_float(a.y) * sc, l0[0], l1[0], l2[0]);
            limbs2(__uint_as_float(a.z) * sc, __uint_as_float(a.w) * sc, l0[1], l1[1], l2[1]);
            limbs2(__uint_as_float(bb.x) * sc, __uint_as_float(bb.y) * sc, l0[2], l1[2], l2[2]);
            limbs2(__uint_as_float(bb.z) * sc, __uint_as_float(bb.w) * sc, l0[3], l1[3], l2[3]);
          }
          const uint32_t ba = sB + (uint32_t)(ng * TC_BSBO + (j >> 3) * TC_BLBO + (j & 7) * 16);
          st_shared_v4(ba, l0[0], l0[1], l0[2], l0[3]);
          st_shared_v4(ba + TC_BTILE, l1[0], l1[1], l1[2], l1[3]);
          st_shared_v4(ba + 2 * TC_BTILE, l2[0], l2[1], l2[2], l2[3]);
        }
      }
      if (td == 0) {
        const int4 pd = info[s];
        tinfo[b] = TcInfo{(int32_t)H.nrows, H.row0, (int32_t)H.flags, nc | ((int32_t)H.limbs << 16), pd.x, pd.y, 0, 0};
      }
      fence_proxy_async();   // the tiles are read by the tensor cores (async proxy)
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&tfull[b]);
        mbar_arrive(&empty[s]);
      }
    }
    if (failed && lane == 0) latch_error(err, 99);
  } else {
    // ---------------------------------------------------------------- fold and emit
    const int te = t - 32 * TC_EPI0;          // 0 .. 255
    const int row = 32 * (w & 3) + lane, half = te >> 7;
    const uint32_t tl = tmem + ((uint32_t)(32 * (w & 3)) << 16) + 16u * (uint32_t)half;
    float2 fhi[8], flo[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      fhi[e] = make_float2(0.f, 0.f);
      flo[e] = make_float2(0.f, 0.f);
    }
    for (int i = 0; i < n; ++i) {
      const int b = i & 1;
      // the fold warps agree (they share a named barrier when they emit)
      const bool ok = mbar_wait(&dfull[b], (uint32_t)((i >> 1) & 1));
      int anybad;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
          : "=r"(anybad)
          : "r"((int)!ok), "r"(32 * TC_NEPI)
          : "memory");
      if (anybad) {
        failed = true;
        break;
      }
      tc_fence_after();
      const TcInfo pi = dinfo[b];
      if (pi.pd & PD_FIRST) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          fhi[e] = make_float2(0.f, 0.f);
          flo[e] = make_float2(0.f, 0.f);
        }
      }
      if ((pi.ncl & 0xffff) > 0) {
        uint32_t vb[16], vs[16];
        tc_ld16(tl + (uint32_t)(b * 64), vb);
        tc_ld16(tl + (uint32_t)(b * 64 + 32), vs);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 8; ++e)
          ff_add_f2(fhi[e], flo[e],
                    __fadd2_rn(make_float2(__uint_as_float(vb[2 * e]), __uint_as_float(vb[2 * e + 1])),
                               make_float2(__uint_as_float(vs[2 * e]), __uint_as_float(vs[2 * e + 1]))));
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&dempty[b]);
      if (pi.pd & PD_LAST) {
        const int R = pi.R;
        const bool calpha = (pi.flags & PH_CALPHA) != 0;
        const bool split = (pi.pd & PD_SPLIT) != 0;
        const Split sp = split ? splits[pi.sp >> 8] : Split{0, 1};
        bool emit = !split;
        if (split) {   // this part's rows, then the last part to arrive adds them all in part order
          F2* mine = fix + (size_t)(sp.slot0 + (pi.sp & 0xff)) * CHUNK_ROWS * RP;
          if (row < R) {
#pragma unroll
            for (int e = 0; e < 8; ++e)
              *reinterpret_cast<float4*>(mine + row * RP + 16 * half + 2 * e) =
                  make_float4(fhi[e].x, flo[e].x, fhi[e].y, flo[e].y);
          }
          asm volatile("bar.sync 1, %0;" ::"r"(32 * TC_NEPI) : "memory");   // the fold warps' rows
          if (te == 0) s_last = atom_add_acq_rel(&fixcnt[pi.sp >> 8], 1) == sp.nparts - 1;
          asm volatile("bar.sync 1, %0;" ::"r"(32 * TC_NEPI) : "memory");   // the acquire before the parts are read
          emit = s_last != 0;
          if (emit) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              fhi[e] = make_float2(0.f, 0.f);
              flo[e] = make_float2(0.f, 0.f);
            }
            for (int part = 0; part < sp.nparts; ++part) {
              const F2* src = fix + (size_t)(sp.slot0 + part) * CHUNK_ROWS * RP;
              if (row < R) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                  const float4 v = __ldcg(reinterpret_cast<const float4*>(src + row * RP + 16 * half + 2 * e));
                  const FF a = ff_add(FF{fhi[e].x, flo[e].x}, FF{v.x, v.y});
                  const FF c = ff_add(FF{fhi[e].y, flo[e].y}, FF{v.z, v.w});
                  fhi[e] = make_float2(a.hi, c.hi);
                  flo[e] = make_float2(a.lo, c.lo);
                }
              }
            }
          }
        }
        if (emit && row < R) {
          if constexpr (MODE == MODE_Y) {
            const int o = __ldg(perm + pi.row0 + row);
            double yo[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int k = 16 * half + e;
              yo[e] = (beta != 0.0 && k < r) ? y[o + (int64_t)k * ldy] : 0.0;
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int k = 16 * half + e;
              if (k < r) {
                const double val = ff_to_d(FF{(e & 1) ? fhi[e >> 1].y : fhi[e >> 1].x,
                                              (e & 1) ? flo[e >> 1].y : flo[e >> 1].x});
                y[o + (int64_t)k * ldy] = (beta == 0.0) ? val : fma(beta, yo[e], val);
              }
            }
          } else {   // coefficient panels: float-float updates, one rounding to FP32
            const int gg = pi.row0 + row;
            const F2 rsc = rowscale ? rowscale[gg] : F2{1.f, 0.f};
            float* vo = vout + (int64_t)gg * RP + 16 * half;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int k = 16 * half + e;
              if (k < r) {
                FF v = {(e & 1) ? fhi[e >> 1].y : fhi[e >> 1].x, (e & 1) ? flo[e >> 1].y : flo[e >> 1].x};
                if constexpr (MODE == MODE_VEC_ADD) v = ff_add_f(v, vo[e]);
                if (rowscale) v = ff_mul(v, FF{rsc.hi, rsc.lo});
                if (calpha) v = ff_mul(v, FF{alpha_ff.hi, alpha_ff.lo});
                vo[e] = v.hi + v.lo;
              }
            }
          }
        }
        if (split && emit && te == 0) fixcnt[pi.sp >> 8] = 0;
      }
    }
    if (failed && lane == 0) latch_error(err, 99);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (w == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------- column dots
// out (nc x RP) = A^T X for each column-dot piece, on the same four roles:
// D (M = the piece's columns, N = RP, K = segment rows) = A (columns x rows,
// K-major: a column's codes are its rows) times the input rows X (rows x RP,
// MN-major), copied with every piece (cp.async).  The fold warps read TMEM lane
// (= column) and write its RP results: the partial sums, or (a column set that
// fits one segment) the scaled coefficients.
constexpr int TCC_ALBO = 144;                                 // A (K-major): K-direction core stride
constexpr int TCC_ASBO = (SEG_ROWS / 8) * TCC_ALBO;           // A: M-direction core stride
static_assert(TCC_ASBO * (CHUNK_ROWS / 8) <= TC_ATILE && SEG_ROWS <= PIECE_MAX_COLS, "column-dot tiles");
// instruction descriptor: D FP32, A and B BF16, A K-major, B MN-major, N = RP, M = 128
constexpr uint32_t TCC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(RP >> 3) << 17) |
                               ((uint32_t)(CHUNK_ROWS >> 4) << 24);

__device__ __forceinline__ void tcc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(TCC_IDESC), "r"(acc)
      : "memory");
}

// Decode of column-dot piece values: task (column j < nc, row group q < Rp / 8)
// writes rows 8 q .. 8 q + 7 of column j as one 16-byte core row per limb.
template <int F, int B>
__device__ __forceinline__ void tcc_decode(uint32_t sa, int R, int nc, int flags, int la, uint32_t sA, int td) {
  const int Rp = (R + 15) & ~15, G = Rp >> 3;
  const uint32_t stride = (uint32_t)Rp * B;
  const uint32_t cm = sa + (uint32_t)sizeof(CPieceHdr);
  const uint32_t cb = cm + ((flags & ITEM_FINAL) ? 16u : 8u) * nc;
  const int dG = (int)c_tcdiv[G];
  for (int task = td; task < nc * G; task += 32 * TC_NDEC) {
    const int j = (task * dG) >> 14, q = task - j * G;
    int e = 0, m = 0;
    if constexpr (F == 2) {
      const uint32_t em = lds32(cm + 8u * j) & 0xffffu;
      e = em & 0xff;
      m = em >> 8;
    }
    float2 h2[4];
    decode8p<F, B>(cb + (uint32_t)j * stride + (uint32_t)(8 * q * B), e, m, h2);
    uint32_t l0[4], l1[4], l2[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) limbs2(h2[u].x, h2[u].y, l0[u], l1[u], l2[u]);
    const uint32_t a = sA + (uint32_t)((j >> 3) * TCC_ASBO + q * TCC_ALBO + (j & 7) * 16);
    st_shared_v4(a, l0[0], l0[1], l0[2], l0[3]);
    if (la > 1) st_shared_v4(a + TC_ATILE, l1[0], l1[1], l1[2], l1[3]);
    if (la > 2) st_shared_v4(a + 2 * TC_ATILE, l2[0], l2[1], l2[2], l2[3]);
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_cdot_tc(const ItemCopy* __restrict__ cps, const int32_t* __restrict__ wbeg, int nrange,
              const uint8_t* __restrict__ pay, const float* __restrict__ vec, F2 alpha, float* __restrict__ partial,
              float* __restrict__ vout, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ TcInfo tinfo[2], dinfo[2];         // R, vin, flags, nc | limbs << 16
  __shared__ int32_t cout_[2][CPIECE_MAX_COLS];  // per accumulator buffer: output of column j
  __shared__ F2 cscl[2][CPIECE_MAX_COLS];        // and its scale (sets that fit one segment)
  __shared__ __align__(8) uint64_t full[TC_NS], empty[TC_NS], tfull[2], tempty[2], dfull[2], dempty[2];
  __shared__ uint32_t tbase;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int r0 = blockIdx.x * MR_CDOT_RANGES, r1 = min(r0 + MR_CDOT_RANGES, nrange);
  if (r0 >= nrange) return;
  const int p0 = wbeg[r0], n = wbeg[r1] - p0;
  if (n <= 0) return;
  uint8_t* ring = smem;
  const uint32_t tiles0 = smem_u32(smem + (size_t)TC_NS * TC_STAGE);
  if (w == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tbase)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    for (int s = 0; s < TC_NS; ++s) {
      mbar_init(&full[s], 1 + 32);
      mbar_init(&empty[s], TC_NDEC);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], TC_NDEC);
      mbar_init(&tempty[b], 1);
      mbar_init(&dfull[b], 2);
      mbar_init(&dempty[b], TC_NEPI);
    }
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tbase;
  bool failed = false;
  if (w == 0) {
    // ---------------------------------------------------------------- copies: piece (bulk) + input rows (cp.async)
    const uint64_t pol = policy_evict_first();
    const ItemCopy zero{0, 0, -1, 0};
    ItemCopy dc = lane < n ? cps[p0 + lane] : zero;
    ItemCopy dn = 32 + lane < n ? cps[p0 + 32 + lane] : zero;
    int dbase = 0;
    for (int i = 0; i < n; ++i) {
      const int s = i % TC_NS;
      if (i >= TC_NS && !__all_sync(HM_FULL, mbar_wait(&empty[s], (uint32_t)(((i / TC_NS) + 1) & 1)))) {
        failed = true;
        break;
      }
      if (i - dbase >= 32) {
        dc = dn;
        dbase += 32;
        dn = dbase + 32 + lane < n ? cps[p0 + dbase + 32 + lane] : zero;
      }
      const int sl = i - dbase;
      const uint32_t off16 = __shfl_sync(HM_FULL, dc.off16, sl), bytes = __shfl_sync(HM_FULL, dc.bytes, sl);
      const int32_t vin = __shfl_sync(HM_FULL, dc.vin, sl), nrows = __shfl_sync(HM_FULL, dc.nrows, sl);
      uint8_t* st = ring + (size_t)s * TC_STAGE;
      const uint32_t pb = (bytes + 15u) & ~15u;
      fence_proxy_async();
      if (lane == 0) {
        mbar_expect_tx(&full[s], pb);
        bulk_g2s_hint(st, pay + (uint64_t)off16 * 16u, pb, &full[s], pol);
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int k = lane + 32 * u;
        if (k < nrows) cp_row(smem_u32(st + STAGE_BYTES + k * TC_TP), vec + (int64_t)(vin + k) * RP);
      }
      cp_arrive(&full[s]);
    }
    if (failed && lane == 0) latch_error(err, 99);
    if (lane == 0)
      for (int i = n - TC_NS < 0 ? 0 : n - TC_NS; i < n; ++i)
        mbar_wait(&full[i % TC_NS], (uint32_t)((i / TC_NS) & 1), failed ? 50u : 2000u);
  } else if (w == 1) {
    // ---------------------------------------------------------------- tensor-core issue
    if (lane == 0) {
      int i = 0;
      for (; i < n; ++i) {
        const int b = i & 1;
        if (!mbar_wait(&tfull[b], (uint32_t)((i >> 1) & 1)) ||
            (i >= 2 && !mbar_wait(&dempty[b], (uint32_t)(((i >> 1) + 1) & 1)))) {
          failed = true;
          break;
        }
        const TcInfo pi = tinfo[b];
        dinfo[b] = pi;
        const int Rp = (pi.R + 15) & ~15, la = pi.ncl >> 16;
        tc_fence_after();
        const uint32_t sA = tiles0 + (uint32_t)(b * TC_TILES), sB = sA + 3u * TC_ATILE;
        const uint32_t d = tmem + (uint32_t)(b * 64);
        for (int k = 0; k < Rp / 16; ++k) {
          uint64_t a[3], bd[3];
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            a[l] = tc_desc(sA + (uint32_t)(l * TC_ATILE + 2 * k * TCC_ALBO), TCC_ALBO, TCC_ASBO);
            bd[l] = tc_desc(sB + (uint32_t)(l * TC_BTILE + 2 * k * TC_BLBO), TC_BLBO, TC_BSBO);
          }
          tcc_mma(d, a[0], bd[0], k > 0);
          tcc_mma(d + 32u, a[0], bd[1], k > 0);
          tcc_mma(d + 32u, a[0], bd[2], 1u);
          if (la > 1) {
            tcc_mma(d + 32u, a[1], bd[0], 1u);
            tcc_mma(d + 32u, a[1], bd[1], 1u);
          }
          if (la > 2) tcc_mma(d + 32u, a[2], bd[0], 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&tempty[b]))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&dfull[b]))
                     : "memory");
        mbar_arrive(&dfull[b]);
      }
      if (failed) latch_error(err, 99);
      for (int j = i - 2; j < i; ++j)
        if (j >= 0) mbar_wait(&tempty[j & 1], (uint32_t)((j >> 1) & 1), failed ? 200u : 2000u);
    }
    __syncwarp();
  } else if (w < TC_EPI0) {
    // ---------------------------------------------------------------- decode
    const int td = t - 32 * TC_DEC0;
    for (int i = 0; i < n; ++i) {
      const int s = i % TC_NS, b = i & 1;
      // the stage; tiles b (products of piece i - 2 done); column outputs b (piece i - 2 folded)
      const bool ok = mbar_wait(&full[s], (uint32_t)((i / TC_NS) & 1)) &&
                      (i < 2 || (mbar_wait(&tempty[b], (uint32_t)(((i >> 1) + 1) & 1)) &&
                                 mbar_wait(&dempty[b], (uint32_t)(((i >> 1) + 1) & 1))));
      if (!__all_sync(HM_FULL, ok)) {
        failed = true;
        break;
      }
      const uint32_t sa = smem_u32(ring + (size_t)s * TC_STAGE);
      const uint4 hw = lds128(sa);   // CPieceHdr
      const int R = (int)(hw.y & 0xffffu), nc = (int)(hw.y >> 16);
      const uint32_t fb = hw.z & 0xffffu;
      const int flags = (int)(hw.z >> 16), la = (int)hw.w;
      const int Rp = (R + 15) & ~15;
      const uint32_t sA = tiles0 + (uint32_t)(b * TC_TILES), sB = sA + 3u * TC_ATILE;
      switch (fb) {
#define HM_TCD(FF_, BB_) \
  case ((FF_) << 4) | (BB_): tcc_decode<FF_, BB_>(sa, R, nc, flags, la, sA, td); break;
        HM_FORMATS(HM_TCD)
#undef HM_TCD
        default:
          latch_error(err, 17);
      }
      if (td < Rp * (RP / 8)) {   // input rows: task (row k, rhs group ng of 8); zero for k >= R
        const int k = td % Rp, ng = td / Rp;
        uint32_t l0[4] = {0u, 0u, 0u, 0u}, l1[4] = {0u, 0u, 0u, 0u}, l2[4] = {0u, 0u, 0u, 0u};
        if (k < R) {
          const uint32_t xa = sa + STAGE_BYTES + (uint32_t)(k * TC_TP + 32 * ng);
          const uint4 a = lds128(xa), bb = lds128(xa + 16);
          limbs2(__uint_as_float(a.x), __uint_as_float(a.y), l0[0], l1[0], l2[0]);
          limbs2(__uint_as_float(a.z), __uint_as_float(a.w), l0[1], l1[1], l2[1]);
          limbs2(__uint_as_float(bb.x), __uint_as_float(bb.y), l0[2], l1[2], l2[2]);
          limbs2(__uint_as_float(bb.z), __uint_as_float(bb.w), l0[3], l1[3], l2[3]);
        }
        const uint32_t ba = sB + (uint32_t)(ng * TC_BSBO + (k >> 3) * TC_BLBO + (k & 7) * 16);
        st_shared_v4(ba, l0[0], l0[1], l0[2], l0[3]);
        st_shared_v4(ba + TC_BTILE, l1[0], l1[1], l1[2], l1[3]);
        st_shared_v4(ba + 2 * TC_BTILE, l2[0], l2[1], l2[2], l2[3]);
      }
      if (td < nc) {   // the column's output index and scale, for the fold warps
        const uint32_t cm = sa + (uint32_t)sizeof(CPieceHdr);
        cout_[b][td] = (int32_t)lds32(cm + 8u * td + 4u);
        if (flags & ITEM_FINAL) {
          const uint2 f = lds64(cm + 8u * nc + 8u * td);
          cscl[b][td] = F2{__uint_as_float(f.x), __uint_as_float(f.y)};
        }
      }
      if (td == 0) tinfo[b] = TcInfo{R, (int32_t)hw.x, flags, nc | (la << 16), 0, 0, 0, 0};
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&tfull[b]);
        mbar_arrive(&empty[s]);
      }
    }
    if (failed && lane == 0) latch_error(err, 99);
  } else {
    // ---------------------------------------------------------------- write the column results
    const int te = t - 32 * TC_EPI0;
    const int j = 32 * (w & 3) + lane, half = te >> 7;   // TMEM lane = column
    const uint32_t tl = tmem + ((uint32_t)(32 * (w & 3)) << 16) + 16u * (uint32_t)half;
    const FF fa = {alpha.hi, alpha.lo};
    for (int i = 0; i < n; ++i) {
      const int b = i & 1;
      if (!__all_sync(HM_FULL, mbar_wait(&dfull[b], (uint32_t)((i >> 1) & 1)))) {
        failed = true;
        break;
      }
      tc_fence_after();
      const TcInfo pi = dinfo[b];
      const int nc = pi.ncl & 0xffff;
      uint32_t vb[16], vs[16];
      tc_ld16(tl + (uint32_t)(b * 64), vb);
      tc_ld16(tl + (uint32_t)(b * 64 + 32), vs);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      int32_t out = 0;
      FF sc = {1.f, 0.f};
      if (j < nc) {
        out = cout_[b][j];
        if (pi.flags & ITEM_FINAL) {
          sc = FF{cscl[b][j].hi, cscl[b][j].lo};
          if (pi.flags & ITEM_ALPHA) sc = ff_mul(sc, fa);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&dempty[b]);
      if (j < nc) {
        float r2[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) r2[e] = __uint_as_float(vb[e]) + __uint_as_float(vs[e]);
        if (pi.flags & ITEM_FINAL) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const FF v = ff_mul(FF{r2[e], 0.f}, sc);
            r2[e] = v.hi + v.lo;
          }
          float4* o = reinterpret_cast<float4*>(vout + (int64_t)out * RP + 16 * half);
#pragma unroll
          for (int e = 0; e < 4; ++e) o[e] = make_float4(r2[4 * e], r2[4 * e + 1], r2[4 * e + 2], r2[4 * e + 3]);
        } else {
          float4* o = reinterpret_cast<float4*>(partial + (int64_t)out * RP + 16 * half);
#pragma unroll
          for (int e = 0; e < 4; ++e) o[e] = make_float4(r2[4 * e], r2[4 * e + 1], r2[4 * e + 2], r2[4 * e + 3]);
        }
      }
    }
    if (failed && lane == 0) latch_error(err, 99);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (w == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

cudaError_t tc_init() {
  cudaError_t e = cudaFuncSetAttribute(k_rgemv_tc<MODE_Y>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_tc<MODE_VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_tc<MODE_VEC_ADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  return e;
}

// nrange ranges, MR_CDOT_RANGES consecutive ones per CTA
cudaError_t launch_cdot_tc(const ItemCopy* items, const int32_t* wbeg, int nrange, const uint8_t* pay, const float* vec,
                           F2 alpha, float* partial, float* vout, int* err, cudaStream_t st) {
  if (nrange <= 0) return cudaSuccess;
  k_cdot_tc<<<(unsigned)((nrange + MR_CDOT_RANGES - 1) / MR_CDOT_RANGES), TC_THREADS, TC_SMEM, st>>>(
      items, wbeg, nrange, pay, vec, alpha, partial, vout, err);
  return cudaGetLastError();
}

// nrange ranges, MP_PAIRS consecutive ones per CTA
cudaError_t launch_rgemv_tc(int mode, const PieceCopy* pieces, const int32_t* wbeg, int nrange, const uint8_t* pay,
                            const float* vec, double alpha, F2 alpha_ff, double beta, double* y, int64_t ldy, int r,
                            const int32_t* perm, float* vout, const F2* rowscale, F2* fix, int32_t* fixcnt,
                            const Split* splits, const int32_t* fan, int32_t fan_base, int* err, cudaStream_t st) {
  if (nrange <= 0) return cudaSuccess;
#define HM_TCG(M)                                                                                              \
  k_rgemv_tc<M><<<(unsigned)((nrange + MP_PAIRS - 1) / MP_PAIRS), TC_THREADS, TC_SMEM, st>>>(pieces, wbeg, nrange, pay, vec, alpha, alpha_ff, \
                                                               beta, y, ldy, r, perm, vout, rowscale, fix, fixcnt, \
                                                               splits, fan, fan_base, err)
  if (mode == MODE_Y)
    HM_TCG(MODE_Y);
  else if (mode == MODE_VEC)
    HM_TCG(MODE_VEC);
  else
    HM_TCG(MODE_VEC_ADD);
#undef HM_TCG
  return cudaGetLastError();
}

}  // namespace hm
