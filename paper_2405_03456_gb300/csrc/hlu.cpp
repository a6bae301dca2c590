// H-LU triangular solves (Sec. 5, Conclusion): the hm_lu_* entry points of
// include/hm.h.  The host factorisation is lu_factor.cpp (dense elimination
// without pivoting, cut along the block tree of A); the packed factors and the
// work list come from build_lu_program (program.cpp); the solve runs as one
// persistent launch in hlu.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include <cuda_runtime.h>

#include "program.h"

namespace hm {
cudaError_t launch_lusolve(int nsm, const LuCol* cols, const LuItem* items, int nitems, const LuDep* deps,
                           const uint8_t* pay, const int32_t* perm, int n, const double* b, double* bz, double* w,
                           double* xz, double* x, double* coef, int* flags, int nflags, int* err, cudaStream_t st);
int lusolve_max_blocks();
}  // namespace hm

using namespace hm;

struct hm_lu {
  HostMatrix L, U;
  int64_t n = 0;
  bool compressed = false;
  double eps = 0;
  int codec = 0, valr = 0;
  LuProgram prog;
  int nsm = 0;
  uint8_t* d_pay = nullptr;
  LuCol* d_cols = nullptr;
  LuItem* d_items = nullptr;
  LuDep* d_deps = nullptr;
  int32_t* d_perm = nullptr;
  int* d_flags = nullptr;
  int* d_err = nullptr;
  double* d_coef = nullptr;
  double* d_vec = nullptr;   // b, w, x in cluster order (3 n)
  void release() {
    for (void* p : {(void*)d_pay, (void*)d_cols, (void*)d_items, (void*)d_deps, (void*)d_perm, (void*)d_flags,
                    (void*)d_err, (void*)d_coef, (void*)d_vec})
      if (p) cudaFree(p);
    d_pay = nullptr;
    d_cols = nullptr;
    d_items = nullptr;
    d_deps = nullptr;
    d_perm = nullptr;
    d_flags = nullptr;
    d_err = nullptr;
    d_coef = nullptr;
    d_vec = nullptr;
    compressed = false;
  }
};

namespace {

template <typename T>
cudaError_t up(T** d, const std::vector<T>& v) {
  const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T) + 64;
  cudaError_t e = cudaMalloc(d, bytes);
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  return cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

extern "C" {

hm_status hm_lu_build(const hm_build_params* prm, const double* pts, int64_t n, hm_lu** out) {
  if (!prm || !pts || !out || n < 1) return HM_ERR_ARG;
  if (prm->leaf_size < 1 || prm->leaf_size > 128) return HM_ERR_ARG;
  if (!(prm->eta > 0) || !(prm->eps_build > 0 && prm->eps_build < 1)) return HM_ERR_ARG;
  if (prm->kernel != HM_KERNEL_LAPLACE && prm->kernel != HM_KERNEL_MATERN15 && prm->kernel != HM_KERNEL_LAPLACE_W)
    return HM_ERR_ARG;
  if (prm->adm < HM_ADM_STANDARD || prm->adm > HM_ADM_BLR) return HM_ERR_ARG;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(pts[i])) return HM_ERR_ARG;
  if (n > LU_MAX_DENSE) return HM_ERR_CAPACITY;
  std::unique_ptr<hm_lu> F;
  try {
    F.reset(new hm_lu());
    F->n = n;
    if (!lu_factor_host(*prm, pts, n, F->L, F->U)) return HM_ERR_UNSUPPORTED;
  } catch (const std::bad_alloc&) {
    return HM_ERR_OOM;
  }
  *out = F.release();
  return HM_OK;
}

hm_status hm_lu_compress(hm_lu* F, double eps, int32_t codec, int32_t valr) {
  if (!F || !(eps > 0 && eps < 1) || codec < HM_CODEC_NONE || codec > HM_CODEC_FPX) return HM_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HM_ERR_CUDA;
  cudaDeviceSynchronize();
  F->release();
  bool ok;
  try {
    ok = build_lu_program(F->L, F->U, codec, eps, valr, F->prog);
  } catch (const std::bad_alloc&) {
    return HM_ERR_OOM;
  }
  if (!ok) return HM_ERR_UNSUPPORTED;
  const int nb = lusolve_max_blocks();
  if (nb <= 0) return HM_ERR_CUDA;
  F->nsm = std::min(nb, nsm);
  const LuProgram& P = F->prog;
  std::vector<int32_t> perm((size_t)F->n);
  for (int64_t i = 0; i < F->n; ++i) perm[i] = (int32_t)F->L.ct.perm[i];
  cudaError_t e;
  if ((e = up(&F->d_pay, P.pk.pay)) != cudaSuccess || (e = up(&F->d_cols, P.cols)) != cudaSuccess ||
      (e = up(&F->d_items, P.items)) != cudaSuccess || (e = up(&F->d_deps, P.deps)) != cudaSuccess ||
      (e = up(&F->d_perm, perm)) != cudaSuccess ||
      (e = cudaMalloc(&F->d_flags, (size_t)(P.nflags + 2) * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&F->d_err, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(F->d_err, 0, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&F->d_coef, (size_t)std::max<int64_t>(P.ncoef, 1) * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&F->d_vec, (size_t)(3 * F->n) * sizeof(double))) != cudaSuccess) {
    F->release();
    return e == cudaErrorMemoryAllocation ? HM_ERR_OOM : HM_ERR_CUDA;
  }
  F->eps = eps;
  F->codec = codec;
  F->valr = valr ? 1 : 0;
  F->compressed = true;
  return HM_OK;
}

hm_status hm_lu_solve(hm_lu* F, const double* b, int64_t ldb, double* x, int64_t ldx, int64_t nrhs, void* stream) {
  if (!F || !b || !x || nrhs < 1 || ldb < F->n || ldx < F->n) return HM_ERR_ARG;
  if (!F->compressed) return HM_ERR_STATE;
  const int64_t n = F->n;
  const double* be = b + ldb * (nrhs - 1) + n;
  const double* xe = x + ldx * (nrhs - 1) + n;
  if (!(be <= x || xe <= b)) return HM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const LuProgram& P = F->prog;
  for (int64_t r = 0; r < nrhs; ++r)
    if (launch_lusolve(F->nsm, F->d_cols, F->d_items, (int)P.items.size(), F->d_deps, F->d_pay, F->d_perm, (int)n,
                       b + r * ldb, F->d_vec, F->d_vec + n, F->d_vec + 2 * n, x + r * ldx, F->d_coef, F->d_flags,
                       (int)P.nflags, F->d_err, st) != cudaSuccess)
      return HM_ERR_CUDA;
  return HM_OK;
}

hm_status hm_lu_sync_status(hm_lu* F, void* stream) {
  if (!F) return HM_ERR_ARG;
  if (!F->d_err) return HM_OK;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return HM_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, F->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HM_ERR_CUDA;
  if (v != 0) {
    cudaMemset(F->d_err, 0, sizeof(int));
    return v == 99 ? HM_ERR_TIMEOUT : HM_ERR_DEVICE;
  }
  return HM_OK;
}

hm_status hm_lu_info(const hm_lu* F, int64_t* stats, int32_t nstats) {
  if (!F || !stats || nstats < 0) return HM_ERR_ARG;
  const int64_t v[7] = {F->n,
                        (int64_t)F->prog.pk.pay.size(),
                        F->prog.pk.value_bytes,
                        F->prog.bytes_fp64,
                        (int64_t)F->prog.items.size(),
                        F->prog.nleaves,
                        (int64_t)(F->L.lr.size() + F->U.lr.size())};
  for (int32_t i = 0; i < nstats && i < 7; ++i) stats[i] = v[i];
  return HM_OK;
}

hm_status hm_lu_free(hm_lu* F) {
  if (!F) return HM_OK;
  F->release();
  delete F;
  return HM_OK;
}

}  // extern "C"
