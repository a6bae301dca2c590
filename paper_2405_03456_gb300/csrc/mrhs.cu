// Multi-RHS products (the precision / multi-RHS form): y := alpha*M*X + beta*y
// for panels of up to RP right-hand sides, FP32 tier.
//
// The matrix is streamed once per panel.  Each block owns a contiguous range of
// the launch's packed units (the same pieces the single-RHS kernels read) and
// pulls them through a ring of shared-memory stages with bulk copies: the
// piece and the RP-wide rows of the vectors it multiplies (input segment /
// multiplier runs), laid out row-major as v[entry * RP + k].  The block decodes
// a piece once into a shared FP32 tile, then every thread owns a small block of
// (row or column) x (right-hand side) outputs, multiplied in FP32 pairs
// (FFMA2) and summed per piece into float-float accumulators.  Chunks shared by
// several blocks are finished by the last block to arrive (fixed order).
#include <cstdint>
#include <cuda_runtime.h>

#include "decode.cuh"

namespace hm {

constexpr int MR_THREADS = 256;
constexpr int MR_STAGES = 3;
constexpr int MR_VEC = SEG_ROWS * RP * 4;           // input rows / multipliers of a stage (64 entries x RP)
constexpr int MR_STAGE = STAGE_BYTES + MR_VEC;      // 10240 bytes

__device__ __forceinline__ uint32_t pad16m(uint32_t x) { return (x + 15u) & ~15u; }

// decode a lane task (8 rows of one column) of a piece into FP32 (FP32 tier)
template <int F, int B>
__device__ __forceinline__ void mr_decode8(uint32_t a, int e, int m, float (&v)[8]) {
  float2 h2[4];
  decode8p<F, B>(a, e, m, h2);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = h2[k].x;
    v[2 * k + 1] = h2[k].y;
  }
}

// ceil(16384 / G): (t * c_div16384[G]) >> 14 == t / G for t < 16384 / G, which
// holds for the decode tasks of a piece (t < 64 G, G <= 16).
__constant__ uint16_t c_div16384[17] = {0, 16384, 8192, 5462, 4096, 3277, 2731, 2341, 2048, 1821, 1639, 1490, 1366, 1261, 1171, 1093, 1024};

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

// ---------------------------------------------------------------- block pipeline
// Stage ring of one block: thread 0 issues the bulk copies of unit i into
// stage i % MR_STAGES; all threads wait on the stage's mbarrier.
struct MrRing {
  uint8_t* base;
  uint64_t* bars;
  __device__ uint8_t* stage(int s) const { return base + (size_t)s * MR_STAGE; }
};

// All threads wait for stage s (unit i); if any thread's bounded wait gave up,
// the whole block agrees (barrier vote), thread 0 waits (bounded) for the
// copies still in flight, the error is latched and true is returned.
__device__ __forceinline__ bool mr_wait_all(const MrRing& ring, int s, int i, int n, int* err) {
  const bool ok = mbar_wait(&ring.bars[s], (uint32_t)((i / MR_STAGES) & 1));
  if (!__syncthreads_or(!ok)) return false;
  if (threadIdx.x == 0) {
    latch_error(err, 99);
    for (int j = i; j < n && j < i + MR_STAGES; ++j)
      mbar_wait(&ring.bars[j % MR_STAGES], (uint32_t)((j / MR_STAGES) & 1), 50u);
  }
  return true;
}

// ---------------------------------------------------------------- tensor-core tiles
// BF16 limb tiles in shared memory (2-byte elements):
//  * column dots: A_l[j][row] (piece column j, segment row), pitch CA halves;
//    X_l[row][k] (input rows x right-hand sides), pitch CB halves;
//  * row chunks:  At_l[j][row] (piece column j, chunk row), pitch CT halves;
//    T_l[j][k] (multipliers x right-hand sides), pitch CB halves.
// Pitches are 16-byte multiples that are 16 mod 128 bytes, so the eight row
// addresses of an ldmatrix hit distinct banks.
constexpr int CA = SEG_ROWS + 8;          // 72 halves = 144 bytes
constexpr int CT = CHUNK_ROWS + 8;        // 136 halves = 272 bytes
constexpr int CB = RP + 8;                // 24 halves = 48 bytes
constexpr int MR_LIMB_A = PIECE_MAX_COLS * CT * 2;   // bytes of one A limb tile (row chunks; column dots use less)
constexpr int MR_LIMB_B = SEG_ROWS * CB * 2;         // bytes of one B limb tile (64 x RP)
constexpr int NT = RP / 8;                           // 8-wide right-hand-side tiles of a panel
constexpr int MR_PAIRS = NT;                         // (row tile, rhs tile) pairs per warp in a row chunk
static_assert(CHUNK_ROWS / 16 == MR_THREADS / 32, "one 16-row tile of a row chunk per warp");
constexpr int MR_TILES = 3 * MR_LIMB_A + 3 * MR_LIMB_B;

// 8 FP32 values -> their first `limbs` BF16 limbs, 16 bytes per limb at dst + l * lstride
__device__ __forceinline__ void store_limbs8(const float (&v)[8], int limbs, uint32_t dst, uint32_t lstride) {
  uint16_t q[3][8];
#pragma unroll
  for (int u = 0; u < 8; ++u) split_bf16x3(v[u], q[0][u], q[1][u], q[2][u]);
#pragma unroll
  for (int l = 0; l < 3; ++l)
    if (l < limbs) {
      const uint32_t w0 = q[l][0] | ((uint32_t)q[l][1] << 16), w1 = q[l][2] | ((uint32_t)q[l][3] << 16);
      const uint32_t w2 = q[l][4] | ((uint32_t)q[l][5] << 16), w3 = q[l][6] | ((uint32_t)q[l][7] << 16);
      asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(dst + l * lstride), "r"(w0), "r"(w1), "r"(w2),
                   "r"(w3)
                   : "memory");
    }
}

// 4 FP32 values -> 3 limbs, 8 bytes per limb at dst + l * lstride
__device__ __forceinline__ void store_limbs4(const float (&v)[4], uint32_t dst, uint32_t lstride) {
  uint16_t q[3][4];
#pragma unroll
  for (int u = 0; u < 4; ++u) split_bf16x3(v[u], q[0][u], q[1][u], q[2][u]);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const uint32_t w0 = q[l][0] | ((uint32_t)q[l][1] << 16), w1 = q[l][2] | ((uint32_t)q[l][3] << 16);
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(dst + l * lstride), "r"(w0), "r"(w1) : "memory");
  }
}

// Limb products A_i B_jb with i + jb <= 2, i < la, accumulated by order
// (d[i + jb]: three independent accumulator chains, added smallest first at
// the end).  A fragments af[i], B fragment pairs (b0[jb], b1[jb]).
__device__ __forceinline__ void mma_limbs(float (&d)[3][4], const uint32_t (&af)[3][4], const uint32_t (&b0)[3],
                                          const uint32_t (&b1)[3], int la) {
  mma_bf16(d[0], af[0], b0[0], b1[0]);
  mma_bf16(d[1], af[0], b0[1], b1[1]);
  mma_bf16(d[2], af[0], b0[2], b1[2]);
  if (la > 1) {
    mma_bf16(d[1], af[1], b0[0], b1[0]);
    mma_bf16(d[2], af[1], b0[1], b1[1]);
  }
  if (la > 2) mma_bf16(d[2], af[2], b0[0], b1[0]);
}

__device__ __forceinline__ void mma_sum(const float (&d)[3][4], float (&o)[4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) o[u] = (d[2][u] + d[1][u]) + d[0][u];
}

// ---------------------------------------------------------------- column dots
// out (nc x RP) = A^T (nc x R) X (R x RP) for one piece on the tensor cores:
// the piece is decoded once into BF16 limb tiles A_l[j][row] (exact: `limbs`
// limbs per value; zero columns up to the next multiple of 16), the input rows
// into 3 limb tiles; warp w computes the 16 x 8 output tile (columns 16 (w / 2)
// .., right-hand sides 8 (w % 2) ..).
template <int F, int B>
__device__ __forceinline__ void mr_cdot_decode(uint32_t sa, uint32_t ta, int R, int nc, int flags, int limbs) {
  const uint32_t stride = (((uint32_t)R + 15u) & ~15u) * B;
  const bool fin = (flags & ITEM_FINAL) != 0;
  const uint32_t cm = sa + (uint32_t)sizeof(CPieceHdr);
  const uint32_t cb = cm + (fin ? 16u : 8u) * nc;
  const int Rp = (R + 15) & ~15, ncp = (nc + 15) & ~15;
  const int G = Rp / RPL;   // rows >= R are zero codes
  const int dG = (int)c_div16384[G];
  for (int task = threadIdx.x; task < ncp * G; task += MR_THREADS) {
    const int j = (task * dG) >> 14, q = task - j * G;   // task / G, task % G (task < 64 G)
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (j < nc) {
      int e = 0, m = 0;
      if constexpr (F == 2) {
        const uint32_t em = lds32(cm + 8u * j) & 0xffffu;
        e = em & 0xff;
        m = em >> 8;
      }
      mr_decode8<F, B>(cb + (uint32_t)j * stride + (uint32_t)(q * RPL * B), e, m, v);
    }
    store_limbs8(v, limbs, ta + (uint32_t)(j * CA + q * RPL) * 2u, MR_LIMB_A);
  }
}

__device__ __forceinline__ void mr_cdot_mma(uint32_t sa, uint32_t xa, uint32_t ta, int R, int nc, int flags,
                                            int limbs, F2 alpha, float* __restrict__ partial,
                                            float* __restrict__ vout) {
  const int t = threadIdx.x;
  const bool fin = (flags & ITEM_FINAL) != 0;
  const uint32_t cm = sa + (uint32_t)sizeof(CPieceHdr);
  const uint32_t sc = cm + 8u * nc;
  const int Rp = (R + 15) & ~15, ncp = (nc + 15) & ~15;
  const uint32_t xl = ta + 3u * MR_LIMB_A;   // X limb tiles
  // input rows: task = (row < Rp, 4 right-hand sides)
  for (int task = t; task < Rp * (RP / 4); task += MR_THREADS) {
    const int row = task / (RP / 4), k4 = task % (RP / 4);
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (row < R) {
      const uint4 x = lds128(xa + (uint32_t)(row * RP + 4 * k4) * 4u);
      v[0] = __uint_as_float(x.x);
      v[1] = __uint_as_float(x.y);
      v[2] = __uint_as_float(x.z);
      v[3] = __uint_as_float(x.w);
    }
    store_limbs4(v, xl + (uint32_t)(row * CB + 4 * k4) * 2u, MR_LIMB_B);
  }
  __syncthreads();
  const int w = t >> 5, L = t & 31;
  // (column tile, pair of rhs tiles) q = w + 8 s: columns 16 (q / (NT / 2)) ..,
  // rhs 16 (q % (NT / 2)) ..; one ldmatrix.x4.trans per limb feeds both rhs tiles
  const int g = L >> 2, tq = L & 3;
  for (int q = w; q < (ncp / 16) * (NT / 2); q += 8) {
    const int mt = q / (NT / 2), h = q % (NT / 2);
    float dd[2][3][4] = {};
    for (int k0 = 0; k0 < Rp; k0 += 16) {
      uint32_t af[3][4], bf[3][4];
      const uint32_t aad = ta + (uint32_t)((16 * mt + (L & 15)) * CA + k0 + (L >> 4) * 8) * 2u;
      const uint32_t bad = xl + (uint32_t)((k0 + (L & 7) + ((L >> 3) & 1) * 8) * CB + 16 * h + (L >> 4) * 8) * 2u;
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        if (l < limbs) ldsm_x4(aad + l * MR_LIMB_A, af[l]);
        ldsm_x4_t(bad + l * MR_LIMB_B, bf[l]);
      }
      const uint32_t e0[3] = {bf[0][0], bf[1][0], bf[2][0]}, e1[3] = {bf[0][1], bf[1][1], bf[2][1]};
      const uint32_t o0[3] = {bf[0][2], bf[1][2], bf[2][2]}, o1[3] = {bf[0][3], bf[1][3], bf[2][3]};
      mma_limbs(dd[0], af, e0, e1, limbs);
      mma_limbs(dd[1], af, o0, o1, limbs);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      float d[4];
      mma_sum(dd[u], d);
      // C fragment: d0 (col g, rhs 2tq), d1 (g, 2tq + 1), d2 (g + 8, 2tq), d3 (g + 8, 2tq + 1)
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {
        const int j = 16 * mt + g + 8 * hr;
        if (j < nc) {
          const int32_t out = (int32_t)lds32(cm + 8u * j + 4u);
          const int k = 8 * (2 * h + u) + 2 * tq;
          const float r0 = d[2 * hr], r1 = d[2 * hr + 1];
          if (fin) {
            const uint2 f = lds64(sc + 8u * j);
            FF scl = {__uint_as_float(f.x), __uint_as_float(f.y)};
            if (flags & ITEM_ALPHA) scl = ff_mul(scl, FF{alpha.hi, alpha.lo});
            const FF v0 = ff_mul(FF{r0, 0.f}, scl), v1 = ff_mul(FF{r1, 0.f}, scl);
            *reinterpret_cast<float2*>(vout + (int64_t)out * RP + k) = make_float2(v0.hi + v0.lo, v1.hi + v1.lo);
          } else {
            *reinterpret_cast<float2*>(partial + (int64_t)out * RP + k) = make_float2(r0, r1);
          }
        }
      }
    }
  }
}

__global__ void __launch_bounds__(MR_THREADS, MR_BLOCKS_PER_SM)
    k_cdot_mr(const ItemCopy* __restrict__ cps, const int32_t* __restrict__ wbeg, int nblk,
              const uint8_t* __restrict__ pay, const float* __restrict__ vec, F2 alpha, float* __restrict__ partial,
              float* __restrict__ vout, int* err) {
  extern __shared__ __align__(128) uint8_t smem[];
  if ((int)blockIdx.x >= nblk) return;
  const int p0 = wbeg[blockIdx.x], n = wbeg[blockIdx.x + 1] - p0;
  if (n <= 0) return;
  MrRing ring{smem, reinterpret_cast<uint64_t*>(smem + MR_STAGES * MR_STAGE)};
  const uint32_t tiles = smem_u32(smem + MR_STAGES * MR_STAGE + 64);
  const uint64_t pol = policy_evict_first();
  // warp 0 issues the copies; its lanes hold the copy descriptors 32 at a time
  const int lane = threadIdx.x & 31;
  const ItemCopy zero{0, 0, 0, 0};
  ItemCopy dc = zero, dn = zero;
  int dbase = 0;
  if (threadIdx.x < 32) {
    dc = lane < n ? cps[p0 + lane] : zero;
    dn = 32 + lane < n ? cps[p0 + 32 + lane] : zero;
  }
  auto issue = [&](int i) {   // warp 0
    if (i - dbase >= 32) {
      dc = dn;
      dbase += 32;
      dn = dbase + 32 + lane < n ? cps[p0 + dbase + 32 + lane] : zero;
    }
    const int sl = i - dbase;
    const uint32_t off16 = __shfl_sync(HM_FULL, dc.off16, sl), bytes = __shfl_sync(HM_FULL, dc.bytes, sl);
    const int32_t vin = __shfl_sync(HM_FULL, dc.vin, sl), nrows = __shfl_sync(HM_FULL, dc.nrows, sl);
    if (lane == 0) {
      const int s = i % MR_STAGES;
      const uint32_t pb = pad16m(bytes), xb = (uint32_t)nrows * RP * 4u;
      fence_proxy_async();
      mbar_expect_tx(&ring.bars[s], pb + xb);
      bulk_g2s_hint(ring.stage(s), pay + (uint64_t)off16 * 16u, pb, &ring.bars[s], pol);
      bulk_g2s(ring.stage(s) + STAGE_BYTES, vec + (int64_t)vin * RP, xb, &ring.bars[s]);
    }
  };
  if (threadIdx.x < 32) {
    if (lane == 0) {
      for (int s = 0; s < MR_STAGES; ++s) mbar_init(&ring.bars[s], 1);
      mbar_init_fence();
    }
    __syncwarp();
    for (int i = 0; i < MR_STAGES && i < n; ++i) issue(i);
  }
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    const int s = i % MR_STAGES;
    if (mr_wait_all(ring, s, i, n, err)) return;
    const uint32_t sa = smem_u32(ring.stage(s));
    const uint4 hw = lds128(sa);
    const int R = (int)(hw.y & 0xffffu), nc = (int)(hw.y >> 16);
    const uint32_t fb = hw.z & 0xffffu, flags = hw.z >> 16;
    const int limbs = (int)hw.w;
    switch (fb) {
#define HM_MC(FF_, BB_) \
  case ((FF_) << 4) | (BB_): mr_cdot_decode<FF_, BB_>(sa, tiles, R, nc, (int)flags, limbs); break;
      HM_FORMATS(HM_MC)
#undef HM_MC
      default:
        latch_error(err, 11);
    }
    mr_cdot_mma(sa, sa + STAGE_BYTES, tiles, R, nc, (int)flags, limbs, alpha, partial, vout);
    __syncthreads();
    if (threadIdx.x < 32 && i + MR_STAGES < n) issue(i + MR_STAGES);
  }
}

// ---------------------------------------------------------------- row chunks
// Decode of a row-chunk piece into the A limb tiles At_l[j][row] (zero columns
// up to the next multiple of 16) and of its multipliers T[j][k] (times the
// tile's scale) into 3 limb tiles T_l[j][k].
template <int F, int B>
__device__ __forceinline__ void mr_rgemv_decode(uint32_t sa, uint32_t ta, const PieceHdr& H, F2 alpha_ff) {
  const int R = H.nrows, nc = H.ncols, ncp = (nc + 15) & ~15;
  const bool tile_piece = (H.flags & PH_TILE) != 0;
  const uint32_t stride = pad8u((uint32_t)R * B);
  const uint32_t cm = sa + (uint32_t)sizeof(PieceHdr);
  const uint32_t cb = cm + (tile_piece ? 0u : pad8u(2u * nc));
  const int e_t = H.em & 0xff, m_t = H.em >> 8;
  const int G = (R + RPL - 1) / RPL;
  const int dG = (int)c_div16384[G];
  for (int task = threadIdx.x; task < ncp * G; task += MR_THREADS) {
    const int j = (task * dG) >> 14, q = task - j * G;   // task / G, task % G (task < 64 G)
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (j < nc) {
      int e = e_t, m = m_t;
      if constexpr (F == 2) {
        if (!tile_piece) {
          const uint32_t em = lds32((cm + 2u * j) & ~3u) >> (16u * (j & 1));
          e = em & 0xff;
          m = (em >> 8) & 0xff;
        }
      }
      mr_decode8<F, B>(cb + (uint32_t)j * stride + (uint32_t)(q * RPL * B), e, m, v);
    }
    store_limbs8(v, H.limbs, ta + (uint32_t)(j * CT + q * RPL) * 2u, MR_LIMB_A);
  }
  float sc = 1.0f;
  if (tile_piece) {
    FF f = {H.scale.hi, H.scale.lo};
    if (H.flags & PH_TALPHA) f = ff_mul(f, FF{alpha_ff.hi, alpha_ff.lo});
    sc = f.hi;
  }
  const uint32_t tl = ta + 3u * MR_LIMB_A, mv = sa + STAGE_BYTES;
  for (int task = threadIdx.x; task < ncp * (RP / 4); task += MR_THREADS) {
    const int j = task / (RP / 4), k4 = task % (RP / 4);
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (j < nc) {
      const uint4 x = lds128(mv + (uint32_t)(j * RP + 4 * k4) * 4u);
      v[0] = __uint_as_float(x.x) * sc;
      v[1] = __uint_as_float(x.y) * sc;
      v[2] = __uint_as_float(x.z) * sc;
      v[3] = __uint_as_float(x.w) * sc;
    }
    store_limbs4(v, tl + (uint32_t)(j * CB + 4 * k4) * 2u, MR_LIMB_B);
  }
}

template <int MODE>
__global__ void __launch_bounds__(MR_THREADS, MR_BLOCKS_PER_SM)
    k_rgemv_mr(const PieceCopy* __restrict__ cps, const int32_t* __restrict__ wbeg, int nblk,
               const uint8_t* __restrict__ pay, const float* __restrict__ vec, double alpha, F2 alpha_ff,
               double beta, double* __restrict__ y, int64_t ldy, int r, const int32_t* __restrict__ perm,
               float* __restrict__ vout, const F2* __restrict__ rowscale, F2* __restrict__ fix,
               int32_t* __restrict__ fixcnt, const Split* __restrict__ splits, const int32_t* __restrict__ fan,
               int32_t fan_base, int* err) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ int4 info[MR_STAGES];
  __shared__ int s_last;
  if ((int)blockIdx.x >= nblk) return;
  const int p0 = wbeg[blockIdx.x], n = wbeg[blockIdx.x + 1] - p0;
  if (n <= 0) return;
  MrRing ring{smem, reinterpret_cast<uint64_t*>(smem + MR_STAGES * MR_STAGE)};
  const uint32_t tiles = smem_u32(smem + MR_STAGES * MR_STAGE + 64);
  const uint64_t pol = policy_evict_first();
  // warp 0 issues the copies; its lanes hold the copy descriptors 32 at a time
  const int lane = threadIdx.x & 31;
  const PieceCopy zero{0, 0, 0, -1};
  PieceCopy dc = zero, dn = zero;
  int dbase = 0;
  if (threadIdx.x < 32) {
    dc = lane < n ? cps[p0 + lane] : zero;
    dn = 32 + lane < n ? cps[p0 + 32 + lane] : zero;
  }
  auto issue = [&](int i) {   // warp 0
    if (i - dbase >= 32) {
      dc = dn;
      dbase += 32;
      dn = dbase + 32 + lane < n ? cps[p0 + dbase + 32 + lane] : zero;
    }
    const int sl = i - dbase;
    const uint32_t off16 = __shfl_sync(HM_FULL, dc.off16, sl), bf = __shfl_sync(HM_FULL, dc.bytes_flags, sl);
    const int32_t moff = __shfl_sync(HM_FULL, dc.moff, sl), sp = __shfl_sync(HM_FULL, dc.split_part, sl);
    const int s = i % MR_STAGES;
    const uint32_t nc = bf >> 24;
    const bool fan_run = moff >= fan_base;   // multipliers scattered over the coefficient rows
    if (lane == 0) {
      const uint32_t pb = pad16m(bf & 0xffffu), mb = nc * RP * 4u;
      info[s] = make_int4((int)((bf >> 16) & 0xffu), sp, 0, 0);
      fence_proxy_async();
      mbar_expect_tx(&ring.bars[s], pb + mb);
      bulk_g2s_hint(ring.stage(s), pay + (uint64_t)off16 * 16u, pb, &ring.bars[s], pol);
      if (mb && !fan_run) bulk_g2s(ring.stage(s) + STAGE_BYTES, vec + (int64_t)moff * RP, mb, &ring.bars[s]);
    }
    if (fan_run) {   // row j of the run: the RP values of coefficient fan[moff - fan_base + j]
      __syncwarp();
      for (int j = lane; j < (int)nc; j += 32) {
        const int32_t src = __ldg(fan + (moff - fan_base) + j);
        bulk_g2s(ring.stage(s) + STAGE_BYTES + j * RP * 4, vec + (int64_t)src * RP, RP * 4u, &ring.bars[s]);
      }
    }
  };
  if (threadIdx.x < 32) {
    if (lane == 0) {
      for (int s = 0; s < MR_STAGES; ++s) mbar_init(&ring.bars[s], 1);
      mbar_init_fence();
    }
    __syncwarp();
    for (int i = 0; i < MR_STAGES && i < n; ++i) issue(i);
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
  const int g = L >> 2, tq = L & 3;
  // warp w owns rows 16 w .. 16 w + 15 of the chunk and every right-hand side:
  // pair sp2 = rhs tile 8 sp2 ..; accumulators per pair and C-fragment row half
  // (row 16 w + g / + 8), float-float pairs over (rhs 8 sp2 + 2 tq, + 1)
  float2 ahi[MR_PAIRS][2], alo[MR_PAIRS][2];
#pragma unroll
  for (int a = 0; a < MR_PAIRS; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      ahi[a][b] = make_float2(0.f, 0.f);
      alo[a][b] = make_float2(0.f, 0.f);
    }
  for (int i = 0; i < n; ++i) {
    const int s = i % MR_STAGES;
    if (mr_wait_all(ring, s, i, n, err)) return;
    const uint32_t sa = smem_u32(ring.stage(s));
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
    const int4 rinfo = info[s];
    if (rinfo.x & PD_FIRST) {
#pragma unroll
      for (int a = 0; a < MR_PAIRS; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          ahi[a][b] = make_float2(0.f, 0.f);
          alo[a][b] = make_float2(0.f, 0.f);
        }
    }
    switch (H.fb) {
#define HM_MD(FF_, BB_) \
  case ((FF_) << 4) | (BB_): mr_rgemv_decode<FF_, BB_>(sa, tiles, H, alpha_ff); break;
      HM_FORMATS(HM_MD)
#undef HM_MD
      default:
        latch_error(err, 12);
    }
    __syncthreads();
    const int R = H.nrows, ncp = (H.ncols + 15) & ~15, la = H.limbs;
    // rows 16 w ..: A fragments once per k step (limbs l < la), B fragments of
    // two rhs tiles per ldmatrix.x4.trans (registers 0, 1: tile 2 h; 2, 3: 2 h + 1)
    if (16 * w < R) {
      float dd[NT][3][4];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
          for (int u = 0; u < 4; ++u) dd[nt][l][u] = 0.f;
      const uint32_t tl = tiles + 3u * MR_LIMB_A;
      for (int k0 = 0; k0 < ncp; k0 += 16) {
        uint32_t af[3][4];
        const uint32_t aad =
            tiles + (uint32_t)((k0 + (L & 7) + ((L >> 4) << 3)) * CT + 16 * w + ((L >> 3) & 1) * 8) * 2u;
#pragma unroll
        for (int l = 0; l < 3; ++l)
          if (l < la) ldsm_x4_t(aad + l * MR_LIMB_A, af[l]);
#pragma unroll
        for (int h = 0; h < NT / 2; ++h) {
          uint32_t bf[3][4];
          const uint32_t bad = tl + (uint32_t)((k0 + (L & 7) + ((L >> 3) & 1) * 8) * CB + 16 * h + (L >> 4) * 8) * 2u;
#pragma unroll
          for (int l = 0; l < 3; ++l) ldsm_x4_t(bad + l * MR_LIMB_B, bf[l]);
          const uint32_t e0[3] = {bf[0][0], bf[1][0], bf[2][0]}, e1[3] = {bf[0][1], bf[1][1], bf[2][1]};
          const uint32_t o0[3] = {bf[0][2], bf[1][2], bf[2][2]}, o1[3] = {bf[0][3], bf[1][3], bf[2][3]};
          mma_limbs(dd[2 * h], af, e0, e1, la);
          mma_limbs(dd[2 * h + 1], af, o0, o1, la);
        }
      }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        float d[4];
        mma_sum(dd[nt], d);
        ff_add_f2(ahi[nt][0], alo[nt][0], make_float2(d[0], d[1]));
        ff_add_f2(ahi[nt][1], alo[nt][1], make_float2(d[2], d[3]));
      }
    }
    if (rinfo.x & PD_LAST) {
      const bool calpha = (H.flags & PH_CALPHA) != 0;
      const bool split = (rinfo.x & PD_SPLIT) != 0;
      const Split sp = split ? splits[rinfo.y >> 8] : Split{0, 1};
      F2* mine = split ? fix + (size_t)(sp.slot0 + (rinfo.y & 0xff)) * CHUNK_ROWS * RP : nullptr;
      if (split) {
#pragma unroll
        for (int sp2 = 0; sp2 < MR_PAIRS; ++sp2)
#pragma unroll
          for (int hr = 0; hr < 2; ++hr) {
            const int row = 16 * w + g + 8 * hr, k = 8 * sp2 + 2 * tq;
            if (row < R) {
              mine[row * RP + k] = F2{ahi[sp2][hr].x, alo[sp2][hr].x};
              mine[row * RP + k + 1] = F2{ahi[sp2][hr].y, alo[sp2][hr].y};
            }
          }
      }
      bool emit = !split;
      if (split) {
        __syncthreads();   // every thread's part rows before thread 0's release
        if (threadIdx.x == 0) s_last = atom_add_acq_rel(&fixcnt[rinfo.y >> 8], 1) == sp.nparts - 1;
        __syncthreads();   // thread 0's acquire before the threads read the other parts
        emit = s_last != 0;
      }
      if (emit) {
        // the thread's elements of pair sp2: rows 16 w + g + 8 hr, right-hand
        // sides 8 sp2 + 2 tq + c, held as (ahi, alo)[sp2][hr].{x, y}; per pair
        // all global loads of a phase are issued before their values are used
#pragma unroll
        for (int sp2 = 0; sp2 < MR_PAIRS; ++sp2) {
          const int k0 = 8 * sp2 + 2 * tq;
          int row[2];
#pragma unroll
          for (int hr = 0; hr < 2; ++hr) row[hr] = 16 * w + g + 8 * hr;
          if (16 * w >= R) continue;
          if (split) {   // the parts in part order
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
              ahi[sp2][hr] = make_float2(0.f, 0.f);
              alo[sp2][hr] = make_float2(0.f, 0.f);
            }
            for (int part = 0; part < sp.nparts; ++part) {
              const F2* src = fix + (size_t)(sp.slot0 + part) * CHUNK_ROWS * RP;
              float4 v[2];
#pragma unroll
              for (int hr = 0; hr < 2; ++hr)
                v[hr] = row[hr] < R ? __ldcg(reinterpret_cast<const float4*>(src + row[hr] * RP + k0))
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int hr = 0; hr < 2; ++hr) {
                const FF a = ff_add(FF{ahi[sp2][hr].x, alo[sp2][hr].x}, FF{v[hr].x, v[hr].y});
                const FF b = ff_add(FF{ahi[sp2][hr].y, alo[sp2][hr].y}, FF{v[hr].z, v[hr].w});
                ahi[sp2][hr] = make_float2(a.hi, b.hi);
                alo[sp2][hr] = make_float2(a.lo, b.lo);
              }
            }
          }
          if constexpr (MODE == MODE_Y) {
            int o[2];
            double yo[2][2];
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) o[hr] = row[hr] < R ? __ldg(perm + H.row0 + row[hr]) : 0;
#pragma unroll
            for (int hr = 0; hr < 2; ++hr)
#pragma unroll
              for (int c = 0; c < 2; ++c)
                yo[hr][c] = (beta != 0.0 && row[hr] < R && k0 + c < r) ? y[o[hr] + (int64_t)(k0 + c) * ldy] : 0.0;
#pragma unroll
            for (int hr = 0; hr < 2; ++hr)
#pragma unroll
              for (int c = 0; c < 2; ++c)
                if (row[hr] < R && k0 + c < r) {
                  const double val = ff_to_d(FF{c ? ahi[sp2][hr].y : ahi[sp2][hr].x, c ? alo[sp2][hr].y : alo[sp2][hr].x});
                  y[o[hr] + (int64_t)(k0 + c) * ldy] = (beta == 0.0) ? val : fma(beta, yo[hr][c], val);
                }
          } else {   // coefficient panels: float-float updates, one rounding to FP32
            float2 old[2];
            F2 sc[2];
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
              const bool on = row[hr] < R;
              const int gg = H.row0 + row[hr];
              old[hr] = (MODE == MODE_VEC_ADD && on) ? *reinterpret_cast<const float2*>(vout + (int64_t)gg * RP + k0)
                                                     : make_float2(0.f, 0.f);
              sc[hr] = (rowscale && on) ? rowscale[gg] : F2{1.f, 0.f};
            }
#pragma unroll
            for (int hr = 0; hr < 2; ++hr)
#pragma unroll
              for (int c = 0; c < 2; ++c)
                if (row[hr] < R && k0 + c < r) {
                  FF v = {c ? ahi[sp2][hr].y : ahi[sp2][hr].x, c ? alo[sp2][hr].y : alo[sp2][hr].x};
                  if constexpr (MODE == MODE_VEC_ADD) v = ff_add_f(v, c ? old[hr].y : old[hr].x);
                  if (rowscale) v = ff_mul(v, FF{sc[hr].hi, sc[hr].lo});
                  if (calpha) v = ff_mul(v, FF{alpha_ff.hi, alpha_ff.lo});
                  vout[(int64_t)(H.row0 + row[hr]) * RP + k0 + c] = v.hi + v.lo;
                }
          }
        }
      }
      if (split && emit && threadIdx.x == 0) fixcnt[rinfo.y >> 8] = 0;
    }
    __syncthreads();
    if (threadIdx.x < 32 && i + MR_STAGES < n) issue(i + MR_STAGES);
  }
}

// ---------------------------------------------------------------- row chunks, register fragments
// The row-chunk panel product for chunks of at most MP_ROWS rows with the piece
// values decoded straight into mma.sync fragments: no shared-memory limb
// tiles and no block barriers.  Two warps (a pair) own a range of pieces and a
// ring of MP_NS stages (piece + its multiplier rows, filled by the pair's warp
// 0); warp wi of the pair takes rows 32 wi .. 32 wi + 31 of every piece and all
// RP right-hand sides.
//
// m16n8k16 fragments (lane = 4 g + tq): A (16 x 16) = piece values, B (16 x 8)
// = multipliers T[column][rhs], C (16 x 8) = row sums.  A rows are permuted so
// that fragment rows g (h = 0) and g + 8 (h = 1) of the warp's row tiles mt =
// 0, 1 are the consecutive chunk rows 32 wi + 4 g + 2 mt + h: a lane decodes 4
// consecutive codes of each of its columns k0 + 2 tq + {0, 1} (A registers 0,
// 1) and k0 + 2 tq + 8 + {0, 1} (registers 2, 3).  B's n is the right-hand side
// 8 nt + g.  C registers (c0, c1 | c2, c3) of tile (mt, nt) hold rows
// 32 wi + 4 g + 2 mt (+ 1), right-hand sides 8 nt + 2 tq + {0, 1}.
//
// Values and multipliers are cut into three BF16 limbs by truncation (exact);
// the products of limb order 0 and of orders 1 + 2 go into two FP32 chains,
// added per piece and folded into float-float row sums.
constexpr int MP_NS = 3;                                   // stages per pair
constexpr int MP_TP = RP * 4 + 16;                         // multiplier row pitch in a stage (bytes)
constexpr int MP_STAGE = STAGE_BYTES + PIECE_MAX_COLS * MP_TP;
constexpr int MP_THREADS = MP_PAIRS * 64;
static_assert(MP_STAGE % 128 == 0, "stage alignment");

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

// One piece for warp wi of the pair: the products of its rows, folded into the
// float-float sums fhi / flo [mt][nt][h] (rows 32 wi + 4 g + 2 mt + h, rhs
// 8 nt + 2 tq + {0, 1}).
template <int F, int B>
__device__ __forceinline__ void mp_piece(uint32_t sa, const PieceHdr& H, F2 alpha_ff, int wi, int lane,
                                         float2 (&fhi)[2][NT][2], float2 (&flo)[2][NT][2]) {
  const int R = H.nrows, nc = H.ncols, la = H.limbs;
  const bool tile = (H.flags & PH_TILE) != 0;
  const uint32_t stride = pad8u((uint32_t)R * B);
  const uint32_t cm = sa + (uint32_t)sizeof(PieceHdr);
  const int g = lane >> 2, tq = lane & 3;
  const uint32_t cb = cm + (tile ? 0u : pad8u(2u * nc)) + (uint32_t)((32 * wi + 4 * g) * B);
  const uint32_t tv = sa + STAGE_BYTES + 4u * g;
  const int e_t = H.em & 0xff, m_t = H.em >> 8;
  float sc = 1.0f;
  if (tile) {
    FF f = {H.scale.hi, H.scale.lo};
    if (H.flags & PH_TALPHA) f = ff_mul(f, FF{alpha_ff.hi, alpha_ff.lo});
    sc = f.hi;
  }
  float big[2][NT][4], sml[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        big[mt][nt][u] = 0.f;
        sml[mt][nt][u] = 0.f;
      }
  for (int k0 = 0; k0 < nc; k0 += 16) {
    uint32_t af[3][2][4];
    {
      float v[4][4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = k0 + 2 * tq + (c & 1) + 8 * (c >> 1);
        const bool on = j < nc;
        const int jj = on ? j : 0;
        int e = e_t, m = m_t;
        if constexpr (F == 2) {
          if (!tile) {
            const uint32_t em = lds32((cm + 2u * jj) & ~3u) >> (16u * (jj & 1));
            e = em & 0xff;
            m = (em >> 8) & 0xff;
          }
        }
        uint32_t w[B];
#pragma unroll
        for (int b = 0; b < B; ++b) w[b] = lds32(cb + (uint32_t)jj * stride + 4u * b);
        float l[4];
        decode4<TIER_F32, F, B>(w, e, m, v[c], l);
#pragma unroll
        for (int u = 0; u < 4; ++u) v[c][u] = on ? v[c][u] : 0.f;
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          limbs2(v[0][2 * mt + h], v[1][2 * mt + h], af[0][mt][h], af[1][mt][h], af[2][mt][h]);
          limbs2(v[2][2 * mt + h], v[3][2 * mt + h], af[0][mt][2 + h], af[1][mt][2 + h], af[2][mt][2 + h]);
        }
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      float t[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = k0 + 2 * tq + (c & 1) + 8 * (c >> 1);
        t[c] = j < nc ? __uint_as_float(lds32(tv + (uint32_t)j * MP_TP + 32u * nt)) * sc : 0.f;
      }
      uint32_t bf[3][2];
      limbs2(t[0], t[1], bf[0][0], bf[1][0], bf[2][0]);
      limbs2(t[2], t[3], bf[0][1], bf[1][1], bf[2][1]);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        mma_bf16(big[mt][nt], af[0][mt], bf[0][0], bf[0][1]);
        mma_bf16(sml[mt][nt], af[0][mt], bf[1][0], bf[1][1]);
        mma_bf16(sml[mt][nt], af[0][mt], bf[2][0], bf[2][1]);
        if (la > 1) {
          mma_bf16(sml[mt][nt], af[1][mt], bf[0][0], bf[0][1]);
          mma_bf16(sml[mt][nt], af[1][mt], bf[1][0], bf[1][1]);
        }
        if (la > 2) mma_bf16(sml[mt][nt], af[2][mt], bf[0][0], bf[0][1]);
      }
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      ff_add_f2(fhi[mt][nt][0], flo[mt][nt][0],
                __fadd2_rn(make_float2(big[mt][nt][0], big[mt][nt][1]), make_float2(sml[mt][nt][0], sml[mt][nt][1])));
      ff_add_f2(fhi[mt][nt][1], flo[mt][nt][1],
                __fadd2_rn(make_float2(big[mt][nt][2], big[mt][nt][3]), make_float2(sml[mt][nt][2], sml[mt][nt][3])));
    }
}

// The same piece on the FP32 pipes: every product is one FP32 FMA (FFMA2 over
// right-hand-side pairs), as in the single-RHS kernels.  The lane keeps the
// fragment kernel's output mapping (rows 32 wi + 4 g + u, u = 2 mt + h;
// right-hand sides 8 nt + 2 tq + {0, 1}): per column it decodes its 4 codes
// and reads its 8 multipliers.
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

// ENG 0: tensor-core fragments (mp_piece); 1: FP32 pipes (ms_piece).
template <int MODE, int ENG>
__global__ void __launch_bounds__(MP_THREADS, 1)
    k_rgemv_mp(const PieceCopy* __restrict__ cps, const int32_t* __restrict__ wbeg, int nrange,
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
#define HM_MP(FF_, BB_)                                          \
  case ((FF_) << 4) | (BB_):                                     \
    if constexpr (ENG == 0)                                      \
      mp_piece<FF_, BB_>(sa, H, alpha_ff, wi, lane, fhi, flo);   \
    else                                                         \
      ms_piece<FF_, BB_>(sa, H, alpha_ff, wi, lane, fhi, flo);   \
    break;
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

// ---------------------------------------------------------------- column dots, register fragments
// out (nc x RP) = A^T (nc x R) X (R x RP) for each piece, with the piece values
// decoded straight into mma.sync A fragments.  A pair of warps owns a range of
// pieces and a ring of MP_NS stages (piece, and the input segment's RP-wide
// rows when the segment changes); warp wi takes the piece's columns
// 32 wi .. 32 wi + 31.  The B fragments of the input segment (its rows x RP,
// three BF16 limbs) are built once per segment into a per-pair cache.
//
// m16n8k16 fragments (lane = 4 g + tq): A (16 x 16) rows = columns
// 32 wi + 16 mt + g (+ 8), A columns = segment rows, permuted so that fragment
// k = 2 tq + {0, 1} / 2 tq + 8 + {0, 1} of k step ks are the rows
// 16 ks + 4 tq + {0, 1} / + {2, 3}: a lane decodes 4 consecutive codes of each
// of its two columns.  B (16 x 8) = X rows x right-hand sides 8 nt + g.  C
// registers (c0, c1 | c2, c3) of tile (mt, nt) hold column 32 wi + 16 mt + g
// (| + 8), right-hand sides 8 nt + 2 tq + {0, 1}.
constexpr int CP_STAGE = STAGE_BYTES + SEG_ROWS * RP * 4;            // piece + input segment rows
constexpr int CP_XF = (SEG_ROWS / 16) * 3 * 2 * 32 * 16;             // B-fragment cache of one pair
constexpr size_t CP_SMEM = (size_t)MP_PAIRS * (MP_NS * CP_STAGE + CP_XF) + (size_t)MP_PAIRS * MP_NS * 8;
static_assert(CP_STAGE % 128 == 0 && CP_XF % 128 == 0, "stage alignment");
static_assert(CP_SMEM <= 227 * 1024, "register-fragment column-dot kernel: one block per SM");

// B fragments of k step ks of the segment whose rows (R of them, RP values each)
// start at shared address xa, for this lane: limb l, rhs tiles 4 h + {0..3}...
// stored as uint4 q = (ks * 3 + l) * 2 + h at xf + (q * 32 + lane) * 16 holding
// (nt = 2 h, r0), (2 h, r1), (2 h + 1, r0), (2 h + 1, r1).
__device__ __forceinline__ void cp_build_xf(uint32_t xa, uint32_t xf, int ks, int R, int lane) {
  const int g = lane >> 2, tq = lane & 3;
  uint32_t b[3][NT][2];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    float x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int row = 16 * ks + 4 * tq + u;
      x[u] = row < R ? __uint_as_float(lds32(xa + (uint32_t)(row * RP + 8 * nt + g) * 4u)) : 0.f;
    }
    limbs2(x[0], x[1], b[0][nt][0], b[1][nt][0], b[2][nt][0]);
    limbs2(x[2], x[3], b[0][nt][1], b[1][nt][1], b[2][nt][1]);
  }
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t q = (uint32_t)((ks * 3 + l) * 2 + h);
      asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(xf + (q * 32u + (uint32_t)lane) * 16u),
                   "r"(b[l][2 * h][0]), "r"(b[l][2 * h][1]), "r"(b[l][2 * h + 1][0]), "r"(b[l][2 * h + 1][1])
                   : "memory");
    }
}

template <int F, int B>
__device__ __forceinline__ void cp_piece(uint32_t sa, uint32_t xf, int R, int nc, int flags, int la, F2 alpha,
                                         int wi, int lane, float* __restrict__ partial, float* __restrict__ vout) {
  const int g = lane >> 2, tq = lane & 3;
  const bool fin = (flags & ITEM_FINAL) != 0;
  const int Rp = (R + 15) & ~15;   // rows R .. Rp - 1 hold zero codes
  const uint32_t stride = (uint32_t)Rp * B;
  const uint32_t cm = sa + (uint32_t)sizeof(CPieceHdr);
  const uint32_t scl = cm + 8u * nc;
  const uint32_t cb = cm + (fin ? 16u : 8u) * nc + (uint32_t)(4 * tq * B);
  float big[2][NT][4], sml[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        big[mt][nt][u] = 0.f;
        sml[mt][nt][u] = 0.f;
      }
  // decode parameters and code addresses of the lane's 4 columns (mt, +8)
  int ee[2][2], mm[2][2];
  uint32_t ca[2][2];
  bool on[2][2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int j = 32 * wi + 16 * mt + g + 8 * c;
      on[mt][c] = j < nc;
      const int jj = on[mt][c] ? j : 0;
      ee[mt][c] = 0;
      mm[mt][c] = 0;
      if constexpr (F == 2) {
        const uint32_t em = lds32(cm + 8u * jj) & 0xffffu;
        ee[mt][c] = em & 0xff;
        mm[mt][c] = em >> 8;
      }
      ca[mt][c] = cb + (uint32_t)jj * stride;
    }
  const bool mt1 = 32 * wi + 16 < nc;   // the second column tile holds a column
  for (int ks = 0; ks < Rp / 16; ++ks) {
    uint32_t bx[3][NT][2];
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint4 v = lds128(xf + ((uint32_t)((ks * 3 + l) * 2 + h) * 32u + (uint32_t)lane) * 16u);
        bx[l][2 * h][0] = v.x;
        bx[l][2 * h][1] = v.y;
        bx[l][2 * h + 1][0] = v.z;
        bx[l][2 * h + 1][1] = v.w;
      }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      if (mt == 1 && !mt1) break;
      float v[2][4];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        uint32_t w[B];
#pragma unroll
        for (int b = 0; b < B; ++b) w[b] = lds32(ca[mt][c] + (uint32_t)(16 * ks * B) + 4u * b);
        float l[4];
        decode4<TIER_F32, F, B>(w, ee[mt][c], mm[mt][c], v[c], l);
#pragma unroll
        for (int u = 0; u < 4; ++u) v[c][u] = on[mt][c] ? v[c][u] : 0.f;
      }
      uint32_t af[3][4];
      limbs2(v[0][0], v[0][1], af[0][0], af[1][0], af[2][0]);
      limbs2(v[1][0], v[1][1], af[0][1], af[1][1], af[2][1]);
      limbs2(v[0][2], v[0][3], af[0][2], af[1][2], af[2][2]);
      limbs2(v[1][2], v[1][3], af[0][3], af[1][3], af[2][3]);
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        mma_bf16(big[mt][nt], af[0], bx[0][nt][0], bx[0][nt][1]);
        mma_bf16(sml[mt][nt], af[0], bx[1][nt][0], bx[1][nt][1]);
        mma_bf16(sml[mt][nt], af[0], bx[2][nt][0], bx[2][nt][1]);
        if (la > 1) {
          mma_bf16(sml[mt][nt], af[1], bx[0][nt][0], bx[0][nt][1]);
          mma_bf16(sml[mt][nt], af[1], bx[1][nt][0], bx[1][nt][1]);
        }
        if (la > 2) mma_bf16(sml[mt][nt], af[2], bx[0][nt][0], bx[0][nt][1]);
      }
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (!on[mt][c]) continue;
      const int j = 32 * wi + 16 * mt + g + 8 * c;
      const int32_t out = (int32_t)lds32(cm + 8u * j + 4u);
      FF sc = {1.f, 0.f};
      if (fin) {
        const uint2 f = lds64(scl + 8u * j);
        sc = FF{__uint_as_float(f.x), __uint_as_float(f.y)};
        if (flags & ITEM_ALPHA) sc = ff_mul(sc, FF{alpha.hi, alpha.lo});
      }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const float2 r2 = __fadd2_rn(make_float2(big[mt][nt][2 * c], big[mt][nt][2 * c + 1]),
                                     make_float2(sml[mt][nt][2 * c], sml[mt][nt][2 * c + 1]));
        const int k = 8 * nt + 2 * tq;
        if (fin) {
          const FF v0 = ff_mul(FF{r2.x, 0.f}, sc), v1 = ff_mul(FF{r2.y, 0.f}, sc);
          *reinterpret_cast<float2*>(vout + (int64_t)out * RP + k) = make_float2(v0.hi + v0.lo, v1.hi + v1.lo);
        } else {
          *reinterpret_cast<float2*>(partial + (int64_t)out * RP + k) = r2;
        }
      }
    }
}

__global__ void __launch_bounds__(MP_THREADS, 1)
    k_cdot_mp(const ItemCopy* __restrict__ cps, const int32_t* __restrict__ wbeg, int nrange,
              const uint8_t* __restrict__ pay, const float* __restrict__ vec, F2 alpha, float* __restrict__ partial,
              float* __restrict__ vout, int* err) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int pair = threadIdx.x >> 6, wi = (threadIdx.x >> 5) & 1, lane = threadIdx.x & 31;
  const int gp = blockIdx.x * MP_PAIRS + pair;
  if (gp >= nrange) return;   // the whole pair
  const int p0 = wbeg[gp], n = wbeg[gp + 1] - p0;
  if (n <= 0) return;
  uint8_t* ring = smem + (size_t)pair * (MP_NS * CP_STAGE + CP_XF);
  const uint32_t xf = smem_u32(ring + (size_t)MP_NS * CP_STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)MP_PAIRS * (MP_NS * CP_STAGE + CP_XF)) + pair * MP_NS;
  const int bid = 1 + pair;
  const uint64_t pol = policy_evict_first();
  const ItemCopy zero{0, 0, -1, 0};
  ItemCopy dc = zero, dn = zero;
  int dbase = 0;
  int32_t last_vin = -1, last_rows = -1;   // input segment of the last issued piece
  if (wi == 0) {
    dc = lane < n ? cps[p0 + lane] : zero;
    dn = 32 + lane < n ? cps[p0 + 32 + lane] : zero;
  }
  auto issue = [&](int i) {   // warp 0 of the pair
    if (i - dbase >= 32) {
      dc = dn;
      dbase += 32;
      dn = dbase + 32 + lane < n ? cps[p0 + dbase + 32 + lane] : zero;
    }
    const int sl = i - dbase;
    const uint32_t off16 = __shfl_sync(HM_FULL, dc.off16, sl), bytes = __shfl_sync(HM_FULL, dc.bytes, sl);
    const int32_t vin = __shfl_sync(HM_FULL, dc.vin, sl), nrows = __shfl_sync(HM_FULL, dc.nrows, sl);
    const bool newx = vin != last_vin || nrows != last_rows;
    last_vin = vin;
    last_rows = nrows;
    if (lane == 0) {
      const int s = i % MP_NS;
      uint8_t* st = ring + (size_t)s * CP_STAGE;
      const uint32_t pb = pad16m(bytes), xb = newx ? (uint32_t)nrows * RP * 4u : 0u;
      fence_proxy_async();
      mbar_expect_tx(&bars[s], pb + xb);
      bulk_g2s_hint(st, pay + (uint64_t)off16 * 16u, pb, &bars[s], pol);
      if (newx) bulk_g2s(st + STAGE_BYTES, vec + (int64_t)vin * RP, xb, &bars[s]);
    }
  };
  if (wi == 0) {
    if (lane == 0) {
      for (int s = 0; s < MP_NS; ++s) mbar_init(&bars[s], 1);
      mbar_init_fence();
    }
    __syncwarp();
    for (int i = 0; i < MP_NS && i < n; ++i) issue(i);
  }
  pair_sync(bid);   // the barriers are initialised before warp 1 waits on them
  int32_t xv = -1, xr = -1;   // segment of the fragment cache
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
    const uint32_t sa = smem_u32(ring + (size_t)s * CP_STAGE);
    const uint4 hw = lds128(sa);   // CPieceHdr
    const int32_t hvin = (int32_t)hw.x;
    const int R = (int)(hw.y & 0xffffu), nc = (int)(hw.y >> 16);
    const uint32_t fb = hw.z & 0xffffu, flags = hw.z >> 16;
    const int la = (int)hw.w;
    if (hvin != xv || R != xr) {   // this piece brought a new input segment: rebuild the cache
      for (int ks = wi; ks < (R + 15) / 16; ks += 2) cp_build_xf(sa + STAGE_BYTES, xf, ks, R, lane);
      xv = hvin;
      xr = R;
      pair_sync(bid);
    }
    if (32 * wi < nc) {
      switch (fb) {
#define HM_CP(FF_, BB_) \
  case ((FF_) << 4) | (BB_): cp_piece<FF_, BB_>(sa, xf, R, nc, (int)flags, la, alpha, wi, lane, partial, vout); break;
        HM_FORMATS(HM_CP)
#undef HM_CP
        default:
          latch_error(err, 14);
      }
    }
    pair_sync(bid);   // both warps are done with stage s and the cache
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
constexpr size_t MR_SMEM_C = (size_t)MR_STAGES * MR_STAGE + 64 + MR_TILES;
constexpr size_t MR_SMEM_R = (size_t)MR_STAGES * MR_STAGE + 64 + MR_TILES;
static_assert(MR_SMEM_R <= 227 * 1024 / MR_BLOCKS_PER_SM, "multi-RHS blocks per SM");
constexpr size_t MP_SMEM = (size_t)MP_PAIRS * MP_NS * MP_STAGE + (size_t)MP_PAIRS * MP_NS * 8;
static_assert(MP_SMEM <= 227 * 1024, "register-fragment row-chunk kernel: one block per SM");

cudaError_t mr_init() {
  cudaError_t e = cudaFuncSetAttribute(k_cdot_mp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CP_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cdot_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CW_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_mr<MODE_Y>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MR_SMEM_R);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_mr<MODE_VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MR_SMEM_R);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_mr<MODE_VEC_ADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MR_SMEM_R);
#define HM_MPA(M, E) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rgemv_mp<M, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MP_SMEM);
  HM_MPA(MODE_Y, 0) HM_MPA(MODE_VEC, 0) HM_MPA(MODE_VEC_ADD, 0) HM_MPA(MODE_Y, 1) HM_MPA(MODE_VEC, 1) HM_MPA(MODE_VEC_ADD, 1)
#undef HM_MPA
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

// nblk ranges; engine 0: tensor-core fragments (one range per warp pair),
// 1: FP32 pipes (one range per warp)
cudaError_t launch_cdot_mr(int engine, const ItemCopy* items, const int32_t* wbeg, int nblk, const uint8_t* pay,
                           const float* vec, F2 alpha, float* partial, float* vout, int* err, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  if (engine == 0)
    k_cdot_mp<<<(unsigned)((nblk + MP_PAIRS - 1) / MP_PAIRS), MP_THREADS, CP_SMEM, st>>>(items, wbeg, nblk, pay, vec,
                                                                                          alpha, partial, vout, err);
  else
    k_cdot_ws<<<(unsigned)((nblk + CW_WARPS - 1) / CW_WARPS), CW_WARPS * 32, CW_SMEM, st>>>(items, wbeg, nblk, pay,
                                                                                             vec, alpha, partial, vout,
                                                                                             err);
  return cudaGetLastError();
}

// nblk ranges (one per warp pair); maxrows = rows of the launch's widest chunk;
// engine 0: tensor-core fragments, 1: FP32 pipes (chunks of at most MP_ROWS rows)
cudaError_t launch_rgemv_mr(int mode, int engine, const PieceCopy* pieces, const int32_t* wbeg, int nblk, int maxrows,
                            const uint8_t* pay, const float* vec, double alpha, F2 alpha_ff, double beta, double* y,
                            int64_t ldy, int r, const int32_t* perm, float* vout, const F2* rowscale, F2* fix,
                            int32_t* fixcnt, const Split* splits, const int32_t* fan, int32_t fan_base, int* err,
                            cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  if (maxrows <= MP_ROWS) {
    const unsigned grid = (unsigned)((nblk + MP_PAIRS - 1) / MP_PAIRS);
#define HM_MPG(M, E)                                                                                         \
  k_rgemv_mp<M, E><<<grid, MP_THREADS, MP_SMEM, st>>>(pieces, wbeg, nblk, pay, vec, alpha, alpha_ff, beta, y, ldy, \
                                                      r, perm, vout, rowscale, fix, fixcnt, splits, fan, fan_base, err)
    if (engine == 0) {
      if (mode == MODE_Y)
        HM_MPG(MODE_Y, 0);
      else if (mode == MODE_VEC)
        HM_MPG(MODE_VEC, 0);
      else
        HM_MPG(MODE_VEC_ADD, 0);
    } else {
      if (mode == MODE_Y)
        HM_MPG(MODE_Y, 1);
      else if (mode == MODE_VEC)
        HM_MPG(MODE_VEC, 1);
      else
        HM_MPG(MODE_VEC_ADD, 1);
    }
#undef HM_MPG
    return cudaGetLastError();
  }
#define HM_MRG(M)                                                                                           \
  k_rgemv_mr<M><<<nblk, MR_THREADS, MR_SMEM_R, st>>>(pieces, wbeg, nblk, pay, vec, alpha, alpha_ff, beta, y, ldy, r, \
                                                     perm, vout, rowscale, fix, fixcnt, splits, fan, fan_base, err)
  if (mode == MODE_Y)
    HM_MRG(MODE_Y);
  else if (mode == MODE_VEC)
    HM_MRG(MODE_VEC);
  else
    HM_MRG(MODE_VEC_ADD);
#undef HM_MRG
  return cudaGetLastError();
}

}  // namespace hm
