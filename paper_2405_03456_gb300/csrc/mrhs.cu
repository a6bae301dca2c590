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
  FF s = {0.f, 0.f};
  for (int p = O.p0; p < O.p1; ++p) {
    const float x = partial[(int64_t)p * RP + k];
    if (O.flags & 2) {
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

// ---------------------------------------------------------------- launchers
constexpr size_t MR_SMEM_C = (size_t)MR_STAGES * MR_STAGE + 64 + MR_TILES;
constexpr size_t MR_SMEM_R = (size_t)MR_STAGES * MR_STAGE + 64 + MR_TILES;
static_assert(MR_SMEM_R <= 227 * 1024 / MR_BLOCKS_PER_SM, "multi-RHS blocks per SM");

cudaError_t mr_init() {
  cudaError_t e = cudaFuncSetAttribute(k_cdot_mr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MR_SMEM_C);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_mr<MODE_Y>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MR_SMEM_R);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_mr<MODE_VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MR_SMEM_R);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rgemv_mr<MODE_VEC_ADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MR_SMEM_R);
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

cudaError_t launch_cdot_mr(const ItemCopy* items, const int32_t* wbeg, int nblk, const uint8_t* pay, const float* vec,
                           F2 alpha, float* partial, float* vout, int* err, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
  k_cdot_mr<<<nblk, MR_THREADS, MR_SMEM_C, st>>>(items, wbeg, nblk, pay, vec, alpha, partial, vout, err);
  return cudaGetLastError();
}

cudaError_t launch_rgemv_mr(int mode, const PieceCopy* pieces, const int32_t* wbeg, int nblk, const uint8_t* pay,
                            const float* vec, double alpha, F2 alpha_ff, double beta, double* y, int64_t ldy, int r,
                            const int32_t* perm, float* vout, const F2* rowscale, F2* fix, int32_t* fixcnt,
                            const Split* splits, const int32_t* fan, int32_t fan_base, int* err, cudaStream_t st) {
  if (nblk <= 0) return cudaSuccess;
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
