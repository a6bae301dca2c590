// Allocation-free host-buffer product: hm_matvec_host_noalloc.
//
// hm_matvec_host stages x and y through device buffers that it allocates
// (and re-allocates when a call needs more room).  Some callers cannot let a
// library call cudaMalloc or cudaFree: a serving process that has reserved its
// whole HBM budget up front and admits work against it, or code that must not
// stall other streams (cudaFree synchronises the whole device).  This file
// gives them the same product with its staging area in a fixed device array
// that is part of the loaded library instead, so the call allocates nothing.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds HM_NOALLOC_MAX_ENTRIES * 2 doubles (16 MiB) of it until the
// process exits.  Host code cannot use the variable's name as a device
// address, so the address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/hm.h"

namespace {

constexpr int64_t kMaxEntries = HM_NOALLOC_MAX_ENTRIES;
constexpr int kMaxDevices = 256;

// [0, kMaxEntries): x staging, [kMaxEntries, 2*kMaxEntries): y staging.
static __device__ __align__(256) double hm_noalloc_scratch[2 * kMaxEntries];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (first call per
// device does the lookup).
hm_status scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HM_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, hm_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return HM_ERR_CUDA;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return HM_OK;
}

}  // namespace

extern "C" hm_status hm_matvec_host_noalloc(hm_matrix* m, double alpha, const double* x, double beta,
                                            double* y, int64_t nrhs, void* stream) {
  if (!m || !x || !y || nrhs < 1 || nrhs > 64) return HM_ERR_ARG;
  hm_info_t info;
  hm_status s = hm_info(m, &info);
  if (s != HM_OK) return s;
  const int64_t n = info.n;
  if (n > kMaxEntries / nrhs) return HM_ERR_CAPACITY;
  double* base = nullptr;
  if ((s = scratch_address(&base)) != HM_OK) return s;
  double* dx = base;
  double* dy = base + kMaxEntries;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)(n * nrhs) * sizeof(double);
  // x and y are copied in whole (y only when beta != 0; with beta == 0 the
  // product writes every entry of y without reading it), so nothing left over
  // from an earlier call is ever read and no part of the array needs clearing.
  if (cudaMemcpyAsync(dx, x, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return HM_ERR_CUDA;
  if (beta != 0.0 && cudaMemcpyAsync(dy, y, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HM_ERR_CUDA;
  s = hm_matvec(m, alpha, dx, n, beta, dy, n, nrhs, stream);
  if (s != HM_OK) return s;
  if (cudaMemcpyAsync(y, dy, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HM_ERR_CUDA;
  return HM_OK;
}
