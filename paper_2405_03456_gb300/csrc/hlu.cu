// Triangular solves with compressed H-LU factors (Sec. 5, Conclusion: the
// triangular solves of an H-LU factorisation read the same compressed blocks
// as the product, with sequential dependencies between them).
//
// x = U^-1 L^-1 b runs as ONE persistent cooperative launch over the work list
// of build_lu_program: warps take the items in list order from a counter, and
// an item first waits (lane 0, bounded acquire spin) for the flags of the items
// it depends on, all of which come earlier in the list -- so the earliest
// unfinished item never waits for anything unfinished and the launch cannot
// stall.  Row items solve one leaf cluster (forward with the unit lower
// triangle of L, backward with the upper triangle of U) after subtracting the
// contributions of every factor block in the leaf's block rows; column items
// form the coefficients t_b = S_b X_b^T z_sigma of low-rank factor blocks.
// Every packed value is decoded with the float-float-tier decoders of the
// product kernels (exact: head + tail is the stored value) and the arithmetic
// is FP64: the solve's cost is its dependency chain, not its arithmetic.
#include <cstdint>
#include <cuda_runtime.h>

#include "decode.cuh"

namespace hm {

constexpr int LU_NW = 8;   // warps per block of the persistent solve

struct LuArgs {
  const LuCol* cols;
  const LuItem* items;
  int nitems;
  const LuDep* deps;
  const uint8_t* pay;
  const double* b;    // right-hand side, cluster order
  double* w;          // forward result, cluster order
  double* x;          // solution, cluster order
  double* coef;       // coefficients of the low-rank factor blocks
  int* flags;         // done flags and coefficient counters (zeroed before the launch)
  unsigned* claim;    // items handed out
  int* abort;         // set on the first timeout: every other wait gives up
  int* err;
};

// Wait (bounded, lane 0) until *f >= target; acquire.
__device__ __forceinline__ bool lu_wait(const LuArgs& A, const int* f, int target) {
  for (uint32_t i = 0; i < (1u << 22); ++i) {   // each try is an L2 round trip: about 2 s in all
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    if (v >= target) return true;
    if ((i & 255u) == 255u && *(volatile int*)A.abort) return false;
  }
  atomicExch(A.abort, 1);
  return false;
}

// The 8 values of rows 8 g .. 8 g + 7 of packed column c, exactly (FP64),
// times c.scale when `scaled`.  The lane copies the group's 8 B bytes into its
// shared-memory slot and decodes them there, as the product kernels do.
__device__ __forceinline__ bool lu_group(const LuArgs& A, const LuCol& c, int g, uint64_t* slot, double (&v)[8]) {
  const int B = c.fb & 15;
  const uint64_t* src = reinterpret_cast<const uint64_t*>(A.pay + c.off + (uint64_t)g * RPL * B);
  for (int i = 0; i < B; ++i) slot[i] = src[i];
  const uint32_t a = smem_u32(slot);
  const int e = c.em & 0xff, m = c.em >> 8;
  float h[8], l[8];
  switch (c.fb) {
#define HM_LU(FF_, BB_) \
  case ((FF_) << 4) | (BB_): decode8s<TIER_FF, FF_, BB_>(a, e, m, h, l); break;
    HM_FORMATS(HM_LU)
#undef HM_LU
    default:
      return false;
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) v[u] = (double)h[u] + (double)l[u];
  return true;
}

// Row item: the leaf's rows r0 .. r0 + R - 1 (R <= 128): lanes (p, g) = (lane / 16,
// lane % 16) take rows 8 g .. 8 g + 7 of the contribution columns p, p + 2, ...;
// the two halves are added, the residual goes to shared memory, and the
// triangle is solved column by column (each lane updates only its own rows).
__device__ bool lu_row(const LuArgs& A, const LuItem& it, int lane, uint64_t* slot, double* rb) {
  const bool fwd = it.kind == LU_ROW_L;
  const double* vin = fwd ? A.w : A.x;
  const int R = it.nr, p = lane >> 4, g = lane & 15;
  const bool mine = 8 * g < R;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool ok = true;
  for (int j = it.c0 + p; j < it.c1; j += 2) {
    const LuCol c = A.cols[j];
    const double mlt = ((c.flags & LC_COEF) ? A.coef[c.mult] : vin[c.mult]) * c.scale;
    if (mine) {
      double v[8];
      ok = lu_group(A, c, g, slot, v) && ok;
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = fma(v[u], mlt, acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] += __shfl_xor_sync(HM_FULL, acc[u], 16);
  const double* rhs = fwd ? A.b : A.w;
  if (p == 0 && mine)
    for (int u = 0; u < 8 && 8 * g + u < R; ++u) rb[8 * g + u] = rhs[it.r0 + 8 * g + u] - acc[u];
  __syncwarp();
  if (fwd) {   // unit lower triangle: z_j final, then rows i > j lose L_ij z_j
    for (int j = 0; j < R; ++j) {
      const double zj = rb[j];
      if (p == 0 && mine && 8 * g + 7 > j) {
        double v[8];
        ok = lu_group(A, A.cols[it.tri + j], g, slot, v) && ok;
        const double sc = A.cols[it.tri + j].scale;
        for (int u = 0; u < 8; ++u) {
          const int i = 8 * g + u;
          if (i > j && i < R) rb[i] = fma(-v[u] * sc, zj, rb[i]);
        }
      }
      __syncwarp();
    }
  } else {     // upper triangle: x_j = r_j / U_jj, then rows i < j lose U_ij x_j
    for (int j = R - 1; j >= 0; --j) {
      double v[8];
      const bool act = p == 0 && mine && 8 * g <= j;
      const double sc = A.cols[it.tri + j].scale;
      if (act) {
        ok = lu_group(A, A.cols[it.tri + j], g, slot, v) && ok;
        if (g == (j >> 3)) rb[j] = rb[j] / (v[j & 7] * sc);
      }
      __syncwarp();
      const double xj = rb[j];
      if (act)
        for (int u = 0; u < 8; ++u) {
          const int i = 8 * g + u;
          if (i < j) rb[i] = fma(-v[u] * sc, xj, rb[i]);
        }
      __syncwarp();
    }
  }
  double* out = fwd ? A.w : A.x;
  if (p == 0 && mine)
    for (int u = 0; u < 8 && 8 * g + u < R; ++u) out[it.r0 + 8 * g + u] = rb[8 * g + u];
  return ok;
}

// Column item: t[c.mult] = c.scale * sum_r X[r, j] z_sigma[r] for each of its
// columns; lanes take the 8-row groups g = lane, lane + 32, ...; fixed xor tree.
__device__ bool lu_col(const LuArgs& A, const LuItem& it, int lane, uint64_t* slot) {
  const double* vin = it.kind == LU_COL_L ? A.w : A.x;
  bool ok = true;
  for (int j = it.c0; j < it.c1; ++j) {
    const LuCol c = A.cols[j];
    double s = 0.0;
    for (int g = lane; 8 * g < it.nr; g += 32) {
      double v[8];
      ok = lu_group(A, c, g, slot, v) && ok;
      for (int u = 0; u < 8; ++u) {
        const int r = 8 * g + u;
        if (r < it.nr) s = fma(v[u], vin[it.r0 + r], s);
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(HM_FULL, s, o);
    if (lane == 0) A.coef[c.mult] = s * c.scale;
  }
  return ok;
}

__global__ void __launch_bounds__(LU_NW * 32, 1) k_lusolve(LuArgs A) {
  __shared__ __align__(16) uint64_t stage[LU_NW * 32 * 8];
  __shared__ double rows[LU_NW * CHUNK_ROWS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* slot = stage + (warp * 32 + lane) * 8;
  double* rb = rows + warp * CHUNK_ROWS;
  for (;;) {
    int i = 0;
    if (lane == 0) i = (int)atomicAdd(A.claim, 1u);
    i = __shfl_sync(HM_FULL, i, 0);
    if (i >= A.nitems) return;
    const LuItem it = A.items[i];
    int ok = 1;
    if (lane == 0)
      for (int d = it.d0; d < it.d1 && ok; ++d) ok = lu_wait(A, A.flags + A.deps[d].flag, A.deps[d].target);
    ok = __shfl_sync(HM_FULL, ok, 0);
    if (!ok) {
      if (lane == 0) latch_error(A.err, 99);
      return;
    }
    __syncwarp();   // lane 0's acquires before the lanes' reads
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    bool good;
    if (it.kind == LU_ROW_L || it.kind == LU_ROW_U)
      good = lu_row(A, it, lane, slot, rb);
    else
      good = lu_col(A, it, lane, slot);
    if (!good) latch_error(A.err, 2);
    asm volatile("fence.acq_rel.gpu;" ::: "memory");   // this lane's stores before the flag
    __syncwarp();
    if (lane == 0) {
      const int add = (it.kind == LU_ROW_L || it.kind == LU_ROW_U) ? 1 : it.c1 - it.c0;
      asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(A.flags + it.flag), "r"(add) : "memory");
    }
  }
}

__global__ void k_lu_gather(const double* __restrict__ b, const int32_t* __restrict__ perm, int n,
                            double* __restrict__ bz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) bz[i] = b[perm[i]];
}

__global__ void k_lu_scatter(const double* __restrict__ xz, const int32_t* __restrict__ perm, int n,
                             double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[perm[i]] = xz[i];
}

// One solve x = U^-1 L^-1 b (original order, device) on stream st; flags,
// counter and abort word (nflags + 2 ints at `flags`) are zeroed first.
cudaError_t launch_lusolve(int nsm, const LuCol* cols, const LuItem* items, int nitems, const LuDep* deps,
                           const uint8_t* pay, const int32_t* perm, int n, const double* b, double* bz, double* w,
                           double* xz, double* x, double* coef, int* flags, int nflags, int* err, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)(nflags + 2) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_lu_gather<<<(n + 255) / 256, 256, 0, st>>>(b, perm, n, bz);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  LuArgs A{cols, items, nitems, deps, pay, bz, w, xz, coef, flags, reinterpret_cast<unsigned*>(flags + nflags),
           flags + nflags + 1, err};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nsm);
  cfg.blockDim = dim3(LU_NW * 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if ((e = cudaLaunchKernelEx(&cfg, k_lusolve, A)) != cudaSuccess) return e;
  k_lu_scatter<<<(n + 255) / 256, 256, 0, st>>>(xz, perm, n, x);
  return cudaGetLastError();
}

// Blocks of the persistent solve that fit on the device at once.
int lusolve_max_blocks() {
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lusolve, LU_NW * 32, 0) != cudaSuccess) return 0;
  return per_sm * nsm;
}

}  // namespace hm
