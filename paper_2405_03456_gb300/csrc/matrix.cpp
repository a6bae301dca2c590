// libhm: C ABI (include/hm.h), device upload and the launch sequence of one
// product.  The packed layout and the launch program are built by
// program.cpp; the kernels live in kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <map>
#include <mutex>
#include <thread>

#include <cuda_runtime.h>

#include "program.h"

namespace hm {
cudaError_t kernels_init();
cudaError_t launch_gather(const double* x, const int32_t* perm, int n, float2* xo, cudaStream_t st);
cudaError_t launch_cdot(int tier, int cfg, const ItemCopy* items, const int32_t* wbeg, int nw, const uint8_t* pay,
                        const float2* vec, F2 alpha, F2* partial, float2* vout, int* err, cudaStream_t st);
cudaError_t launch_fanout(const int32_t* src, int n, float2* dst, const float2* vec, cudaStream_t st);
cudaError_t launch_gsum(const GsumOut* outs, int nouts, const F2* pscale, const F2* partial, F2 alpha, float2* vout,
                        const int32_t* fan_dst, const int32_t* csrc, const int32_t* cdst, int ncopy, cudaStream_t st);
cudaError_t launch_rgemv(int tier, int mode, int cfg, const PieceCopy* pieces, const int32_t* wbeg, int nw,
                         const uint8_t* pay, const float2* vec, double alpha, F2 alpha_ff, double beta, double* y,
                         const int32_t* perm, float2* vout, const F2* rowscale, F2* fix, int32_t* fixcnt,
                         const Split* splits, int* err, cudaStream_t st);
cudaError_t launch_rseq(int tier, int nblk, const SeqPhase* phases, int nph, const PieceCopy* pieces,
                        const int32_t* wbeg, const uint8_t* pay, float2* vec, double alpha, F2 alpha_ff, double beta,
                        double* y, const int32_t* perm, const F2* rowscale, F2* fix, int32_t* fixcnt,
                        const Split* splits, const SeqDep* deps, unsigned* ver, int nchunks, int* err,
                        cudaStream_t st);
int rseq_max_blocks();
cudaError_t launch_prog(int tier, int nblk, const ProgPhase* phases, int nphases, const double* x,
                        const ItemCopy* items, const GsumOut* gouts, const F2* pscale, F2* partial,
                        const int32_t* fan, const PieceCopy* pieces, const int32_t* wbeg, const SeqPhase* seqph,
                        const SeqDep* deps, unsigned* state, int nstate, const uint8_t* pay, float2* vec,
                        double alpha, double beta, double* y, const int32_t* perm, const F2* rowscale, F2* fix,
                        int32_t* fixcnt, const Split* splits, const int32_t* fan_dst, const int32_t* fan_copy_src,
                        const int32_t* fan_copy_dst, int* err, cudaStream_t st);
int prog_max_blocks();
cudaError_t mr_init();
cudaError_t tc_init();
cudaError_t launch_cdot_tc(const ItemCopy* items, const int32_t* wbeg, int nrange, const uint8_t* pay, const float* vec,
                           F2 alpha, float* partial, float* vout, int* err, cudaStream_t st);
cudaError_t launch_rgemv_tc(int mode, const PieceCopy* pieces, const int32_t* wbeg, int nrange, const uint8_t* pay,
                            const float* vec, double alpha, F2 alpha_ff, double beta, double* y, int64_t ldy, int r,
                            const int32_t* perm, float* vout, const F2* rowscale, F2* fix, int32_t* fixcnt,
                            const Split* splits, const int32_t* fan, int32_t fan_base, int* err, cudaStream_t st);
cudaError_t launch_gather_mr(const double* x, int64_t ldx, int r, const int32_t* perm, int n, float* v,
                             cudaStream_t st);
cudaError_t launch_gsum_mr(const GsumOut* outs, int nouts, const F2* pscale, const float* partial, F2 alpha, float* v,
                           cudaStream_t st);
cudaError_t launch_cdot_ws(const ItemCopy* items, const int32_t* wbeg, int nblk, const uint8_t* pay, const float* vec,
                           F2 alpha, float* partial, float* vout, int* err, cudaStream_t st);
cudaError_t launch_rgemv_ms(int mode, const PieceCopy* pieces, const int32_t* wbeg, int nblk, const uint8_t* pay,
                            const float* vec, double alpha, F2 alpha_ff, double beta, double* y, int64_t ldy, int r,
                            const int32_t* perm, float* vout, const F2* rowscale, F2* fix, int32_t* fixcnt,
                            const Split* splits, const int32_t* fan, int32_t fan_base, int* err, cudaStream_t st);
cudaError_t launch_decode(const uint8_t* p, int64_t n, int B, int fmt, int e, int m, double vmin,
                          double* out, cudaStream_t st);
cudaError_t launch_decode_debug(int tier, const DbgTask* tasks, int64_t ntask, const uint8_t* pay, float2* out,
                                int* err, cudaStream_t st);
}  // namespace hm

using namespace hm;

namespace {

template <typename T>
struct DevArr {
  T* p = nullptr;
  size_t n = 0;
  cudaError_t upload(const std::vector<T>& v) {
    n = v.size();
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T) + 64);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(p, v.data(), n * sizeof(T), cudaMemcpyHostToDevice);
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

hm_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HM_OK;
  if (e == cudaErrorMemoryAllocation) return HM_ERR_OOM;
  return HM_ERR_CUDA;
}

}  // namespace

struct hm_matrix {
  HostMatrix H;
  bool compressed = false;
  int codec = 0, valr = 0;
  double eps = 0;
  Program prog;
  // device copies of the program
  DevArr<uint8_t> d_pay;
  DevArr<ItemCopy> d_items;
  DevArr<GsumOut> d_gout;
  DevArr<F2> d_pscale;
  DevArr<PieceCopy> d_pieces;
  DevArr<int32_t> d_wbeg;
  DevArr<int32_t> d_fan;
  DevArr<int32_t> d_fan_dst, d_fcopy_src, d_fcopy_dst;   // folded fan-outs
  DevArr<Split> d_splits;
  DevArr<F2> d_rowscale_ff;     // row scales of coefficient vectors (float-float pairs)
  DevArr<int32_t> d_perm;
  F2* d_fix = nullptr;         // row sums of the parts of chunks shared by warps
  float* d_vmr = nullptr;      // multi-RHS vectors: nvec x RP (FP32 tier)
  float* d_pmr = nullptr;      // multi-RHS column-dot partials: npartial x RP
  F2* d_fixmr = nullptr;       // multi-RHS fix-up rows: nfix_mr x CHUNK_ROWS x RP
  int32_t* d_fixcnt = nullptr; // arrival counters of those chunks (reset by the last part)
  float2* d_vec = nullptr;     // vector workspace (x, coefficient vectors)
  F2* d_part = nullptr;        // column-dot partial sums (float-float)
  int* d_err = nullptr;        // latched device error word
  double* d_hx = nullptr;      // host-path staging (hm_matvec_host)
  double* d_hy = nullptr;
  cudaStream_t h_side = nullptr;          // host path: second copy stream (x and y copies overlap)
  cudaEvent_t h_ev0 = nullptr, h_ev1 = nullptr;
  int64_t d_h_cap = 0;
  int nsm = 0;
  // persistent launches: runs [first, last) of consecutive row-chunk launches
  // executed as the phases of one cooperative launch (dataflow between phases)
  int64_t width_bytes[8] = {};  // packed code bytes by code width B (set at compress time)
  int fuse = 1;                // 0 per launch, 1 runs of row-chunk launches fused, 2 the whole product
  int mr_engine = 1;           // multi-RHS panels: 0 tensor cores (tcgen05), 1 FP32 pipes
  DevArr<ProgPhase> d_prog;    // phases of the whole-product launch
  unsigned* d_pstate = nullptr;  // its barrier counter, abort word and the runs' state
  int pstate_n = 0;
  struct Run {
    size_t first, last;
    int64_t ph0;   // first phase in d_phases
    int nchunks;   // coefficient chunks written in the run (versions ver[0 .. nchunks))
  };
  std::vector<Run> runs;
  DevArr<SeqPhase> d_phases;
  DevArr<SeqDep> d_deps;       // per piece (pieces of runs only)
  unsigned* d_ver = nullptr;   // chunk versions, abort word and per-phase range counters of the largest run
  // the transposed matrix (adjoint products), built on first use, owned
  hm_matrix* adj = nullptr;
  std::mutex mu;
  // CUDA graph of the whole launch sequence, cached per call signature
  bool use_graph = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  struct GKey {
    const double* x = nullptr;
    double* y = nullptr;
    int64_t ldx = 0, ldy = 0, nrhs = 0;
    double alpha = 0, beta = 0;
    bool operator==(const GKey& o) const {
      return x == o.x && y == o.y && ldx == o.ldx && ldy == o.ldy && nrhs == o.nrhs && alpha == o.alpha &&
             beta == o.beta;
    }
  } gkey;
  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }
  // profiling: event pairs per launch
  bool prof = false;
  struct Rec {
    int kind;
    cudaEvent_t e0, e1;
    int64_t bytes;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> evpool;
  cudaEvent_t take_event() {
    if (!evpool.empty()) {
      cudaEvent_t e = evpool.back();
      evpool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }

  void release_device() {
    drop_graph();
    d_pay.release();
    d_items.release();
    d_gout.release();
    d_pscale.release();
    d_pieces.release();
    d_wbeg.release();
    d_fan.release();
    d_fan_dst.release();
    d_fcopy_src.release();
    d_fcopy_dst.release();
    d_splits.release();
    d_rowscale_ff.release();
    d_phases.release();
    d_deps.release();
    d_prog.release();
    if (d_pstate) cudaFree(d_pstate);
    d_pstate = nullptr;
    pstate_n = 0;
    runs.clear();
    if (d_ver) cudaFree(d_ver);
    d_ver = nullptr;
    d_perm.release();
    if (d_fix) cudaFree(d_fix);
    if (d_fixcnt) cudaFree(d_fixcnt);
    if (d_vmr) cudaFree(d_vmr);
    if (d_pmr) cudaFree(d_pmr);
    if (d_fixmr) cudaFree(d_fixmr);
    d_vmr = d_pmr = nullptr;
    d_fixmr = nullptr;
    d_fix = nullptr;
    d_fixcnt = nullptr;
    if (d_vec) cudaFree(d_vec);
    if (d_part) cudaFree(d_part);
    if (d_err) cudaFree(d_err);
    if (d_hx) cudaFree(d_hx);
    if (d_hy) cudaFree(d_hy);
    d_vec = nullptr;
    d_part = nullptr;
    d_err = nullptr;
    d_hx = d_hy = nullptr;
    d_h_cap = 0;
    compressed = false;
  }
};

namespace hm {
// Access for persist.cpp (hm_save / hm_load).
HostMatrix& host_of(hm_matrix* m) { return m->H; }
bool compressed_state(const hm_matrix* m, double& eps, int& codec, int& valr) {
  eps = m->eps;
  codec = m->codec;
  valr = m->valr;
  return m->compressed;
}
hm_matrix* new_matrix() { return new hm_matrix(); }
}  // namespace hm

namespace {

std::once_flag g_kinit;
cudaError_t g_kinit_err = cudaSuccess;

hm_status upload(hm_matrix* M) {
  Program& P = M->prog;
  cudaError_t e;
  std::call_once(g_kinit, [] {
    g_kinit_err = kernels_init();
    if (g_kinit_err == cudaSuccess) g_kinit_err = mr_init();
    if (g_kinit_err == cudaSuccess) g_kinit_err = tc_init();
  });
  if (g_kinit_err != cudaSuccess) return HM_ERR_CUDA;
#define UP(arr, vec) \
  if ((e = M->arr.upload(vec)) != cudaSuccess) return cuda_status(e);
  UP(d_pay, P.pk.pay)
  UP(d_items, P.items)
  UP(d_gout, P.gouts)
  UP(d_pscale, P.pscale)
  {
    std::vector<PieceCopy> all;
    for (int cf = 0; cf < NSHAPES; ++cf) all.insert(all.end(), P.pdesc[cf].begin(), P.pdesc[cf].end());
    UP(d_pieces, all)
  }
  UP(d_wbeg, P.wbeg)
  UP(d_fan, P.fan_src)
  UP(d_fan_dst, P.fan_dst)
  UP(d_fcopy_src, P.fan_copy_src)
  UP(d_fcopy_dst, P.fan_copy_dst)
  UP(d_splits, P.splits)
  {
    std::vector<F2> rs(P.rowscale.size());
    for (size_t i = 0; i < rs.size(); ++i) rs[i] = split_ff(P.rowscale[i]);
    UP(d_rowscale_ff, rs)
  }
#undef UP
  std::vector<int32_t> perm(M->H.n);
  for (int64_t i = 0; i < M->H.n; ++i) perm[i] = (int32_t)M->H.ct.perm[i];
  if ((e = M->d_perm.upload(perm)) != cudaSuccess) return cuda_status(e);
  // +16 entries: 16-byte aligned bulk copies of a segment may read past the end
  if ((e = cudaMalloc(&M->d_vec, (std::max<int64_t>(P.nvec, 1) + 16) * sizeof(float2))) != cudaSuccess)
    return cuda_status(e);
  if ((e = cudaMemset(M->d_vec, 0, (std::max<int64_t>(P.nvec, 1) + 16) * sizeof(float2))) != cudaSuccess)
    return cuda_status(e);
  if ((e = cudaMalloc(&M->d_part, std::max<int64_t>(P.npartial, 1) * sizeof(F2))) != cudaSuccess)
    return cuda_status(e);
  if ((e = cudaMalloc(&M->d_fix, std::max<int64_t>(P.nfix, 1) * CHUNK_ROWS * sizeof(F2))) != cudaSuccess)
    return cuda_status(e);
  const size_t ncnt = std::max<size_t>(P.splits.size(), 1) * sizeof(int32_t);
  if ((e = cudaMalloc(&M->d_fixcnt, ncnt)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemset(M->d_fixcnt, 0, ncnt)) != cudaSuccess) return cuda_status(e);
  if (P.tier == TIER_F32) {   // multi-RHS workspace (panels of RP right-hand sides; no fan-out slots)
    const size_t nv = (size_t)(std::max<int64_t>(P.fan_base, 1) + SEG_ROWS) * RP * sizeof(float);
    if ((e = cudaMalloc(&M->d_vmr, nv)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemset(M->d_vmr, 0, nv)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMalloc(&M->d_pmr, (size_t)std::max<int64_t>(P.npartial, 1) * RP * sizeof(float))) != cudaSuccess)
      return cuda_status(e);
    if ((e = cudaMalloc(&M->d_fixmr, (size_t)std::max<int64_t>(P.nfix_mr, 1) * CHUNK_ROWS * RP * sizeof(F2))) !=
        cudaSuccess)
      return cuda_status(e);
  }
  if ((e = cudaMalloc(&M->d_err, sizeof(int))) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemset(M->d_err, 0, sizeof(int))) != cudaSuccess) return cuda_status(e);
  // persistent runs: maximal sequences of >= 2 row-chunk launches, when a
  // cooperative launch of one block per SM fits (phases use the SEQ_SHAPE ranges)
  {
    std::vector<SeqPhase> ph;
    std::vector<SeqDep> deps;
    int maxchunks = 0;
    const auto& Ls = P.launches;
    const bool fits = rseq_max_blocks() >= M->nsm && M->nsm > 0;
    for (size_t i = 0; fits && i < Ls.size();) {
      size_t j = i;
      while (j < Ls.size() && Ls[j].kind == Launch::RGEMV) ++j;
      hm_matrix::Run R{i, j, (int64_t)ph.size(), 0};
      if (j - i >= 2 && seq_dependencies(P, i, j, deps, R.nchunks)) {
        M->runs.push_back(R);
        maxchunks = std::max(maxchunks, R.nchunks);
        for (size_t k = i; k < j; ++k) {
          const Launch& L = Ls[k];
          ph.push_back(SeqPhase{L.mode, (int32_t)L.woff[SEQ_SHAPE], L.nw[SEQ_SHAPE], L.use_rowscale ? 1 : 0});
        }
      }
      i = std::max(j, i + 1);
    }
    if (!ph.empty()) {
      if ((e = M->d_phases.upload(ph)) != cudaSuccess) return cuda_status(e);
      if ((e = M->d_deps.upload(deps)) != cudaSuccess) return cuda_status(e);
      int maxph = 0;
      for (const hm_matrix::Run& R : M->runs) maxph = std::max(maxph, (int)(R.last - R.first));
      if ((e = cudaMalloc(&M->d_ver, (size_t)(maxchunks + 1 + maxph) * sizeof(unsigned))) != cudaSuccess)
        return cuda_status(e);
    }
  }
  // the whole product as one launch (hm_persistent mode 2): one phase per
  // launch, one per run of row-chunk launches; state = barrier counter, abort
  // word, then per run its versions, abort word and range counters
  if (prog_max_blocks() >= M->nsm && M->nsm > 0) {
    std::vector<ProgPhase> pp;
    int64_t nstate = 2;
    const auto& Ls = P.launches;
    size_t ri = 0;
    for (size_t li = 0; li < Ls.size();) {
      const Launch& L = Ls[li];
      ProgPhase ph{};
      if (ri < M->runs.size() && M->runs[ri].first == li) {
        const hm_matrix::Run& R = M->runs[ri];
        ph.kind = PP_RUN;
        ph.off = (int32_t)R.ph0;
        ph.n = (int32_t)(R.last - R.first);
        ph.mode = (int32_t)ri;
        ph.aux = (int32_t)nstate;
        ph.nchunks = R.nchunks;
        nstate += R.nchunks + 1 + ph.n;
        pp.push_back(ph);
        li = R.last;
        ++ri;
        continue;
      }
      switch (L.kind) {
        case Launch::GATHER: ph = ProgPhase{PP_GATHER, 0, (int32_t)L.n, 0, 0, 0, 0, 0}; break;
        case Launch::CDOT: ph = ProgPhase{PP_CDOT, (int32_t)L.woff[0], L.nw[0], 0, 0, 0, 0, 0}; break;
        case Launch::GSUM:
          ph = ProgPhase{PP_GSUM, (int32_t)L.off, (int32_t)L.n, (int32_t)L.copy_off, 0, L.scatter ? 1 : 0,
                         (int32_t)L.copy_n, 0};
          break;
        case Launch::FANOUT:
          ph = ProgPhase{PP_FANOUT, (int32_t)L.off, (int32_t)L.n, 0, 0, (int32_t)P.fan_base, 0, 0};
          break;
        case Launch::RGEMV:
          ph = ProgPhase{PP_RGEMV, (int32_t)L.woff[SEQ_SHAPE], L.nw[SEQ_SHAPE], L.mode, L.use_rowscale ? 1 : 0, 0, 0, 0};
          break;
      }
      pp.push_back(ph);
      ++li;
    }
    if (!pp.empty() && nstate < INT32_MAX) {
      if ((e = M->d_prog.upload(pp)) != cudaSuccess) return cuda_status(e);
      if ((e = cudaMalloc(&M->d_pstate, (size_t)nstate * sizeof(unsigned))) != cudaSuccess) return cuda_status(e);
      M->pstate_n = (int)nstate;
    }
  }
  return HM_OK;
}

}  // namespace

namespace {

// One packed column of a unit of the payload: byte offset of its first code,
// rows, decode class fb = fmt << 4 | B and em = e | m << 8.
struct PackedCol {
  uint64_t off;
  int32_t rows;
  uint16_t fb, em;
};

// The packed columns of units [u0, u1) in payload order: column-dot pieces
// (P.items) first, then row-chunk pieces (in program order), each read from its
// inline header exactly as the kernels read it.
void packed_columns(const Program& P, int64_t u0, int64_t u1, std::vector<PackedCol>& cols) {
  const uint8_t* pay = P.pk.pay.data();
  const int64_t ni = (int64_t)P.items.size();
  for (int64_t u = u0; u < u1; ++u) {
    if (u < ni) {
      const uint64_t off = (uint64_t)P.items[u].off16 * 16u;
      CPieceHdr h;
      std::memcpy(&h, pay + off, sizeof h);
      const int B = h.fb & 15, nc = h.ncols, R = h.nrows;
      const bool fin = (h.flags & ITEM_FINAL) != 0;
      const uint64_t cm = off + sizeof(CPieceHdr);
      const uint64_t cb = cm + (uint64_t)(fin ? 16 : 8) * nc;
      const uint64_t stride = (uint64_t)((R + 15) & ~15) * B;
      for (int j = 0; j < nc; ++j) {
        CColMeta c;
        std::memcpy(&c, pay + cm + 8u * j, sizeof c);
        cols.push_back(PackedCol{cb + j * stride, R, h.fb, c.em});
      }
    } else {
      const uint64_t off = (uint64_t)P.pdesc[0][u - ni].off16 * 16u;
      PieceHdr h;
      std::memcpy(&h, pay + off, sizeof h);
      const int B = h.fb & 15, nc = h.ncols, R = h.nrows;
      const bool tile = (h.flags & PH_TILE) != 0;
      const uint64_t cm = off + sizeof(PieceHdr);
      const uint64_t cb = cm + (tile ? 0 : (uint64_t)((2 * nc + 7) & ~7));
      const uint64_t stride = (uint64_t)((R * B + 7) & ~7);
      for (int j = 0; j < nc; ++j) {
        uint16_t em = h.em;
        if (!tile) std::memcpy(&em, pay + cm + 2u * j, 2);
        cols.push_back(PackedCol{cb + j * stride, R, h.fb, em});
      }
    }
  }
}

}  // namespace

// ==================================================================== C ABI
extern "C" {

const char* hm_status_str(hm_status s) {
  switch (s) {
    case HM_OK: return "ok";
    case HM_ERR_ARG: return "invalid argument";
    case HM_ERR_OOM: return "out of memory";
    case HM_ERR_CUDA: return "CUDA runtime error";
    case HM_ERR_STATE: return "invalid call order";
    case HM_ERR_TIMEOUT: return "device wait timed out";
    case HM_ERR_IO: return "I/O error";
    case HM_ERR_DEVICE: return "device-side error latched";
    case HM_ERR_UNSUPPORTED: return "data outside the decodable range";
    case HM_ERR_CAPACITY: return "request exceeds a fixed limit (noalloc scratch, or the packed form's addressing)";
  }
  return "unknown status";
}

hm_status hm_build(const hm_build_params* prm, const double* pts, int64_t n, hm_matrix** out) {
  if (!prm || !pts || !out || n < 1 || n > (int64_t)INT32_MAX / 2) return HM_ERR_ARG;
  if (prm->leaf_size < 1 || prm->leaf_size > 128) return HM_ERR_ARG;
  if (!(prm->eta > 0) || !(prm->eps_build > 0 && prm->eps_build < 1)) return HM_ERR_ARG;
  if (prm->format < HM_FMT_H || prm->format > HM_FMT_UH_SEP) return HM_ERR_ARG;
  if (prm->kernel != HM_KERNEL_LAPLACE && prm->kernel != HM_KERNEL_MATERN15 && prm->kernel != HM_KERNEL_LAPLACE_W)
    return HM_ERR_ARG;
  if (prm->adm < HM_ADM_STANDARD || prm->adm > HM_ADM_BLR) return HM_ERR_ARG;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(pts[i])) return HM_ERR_ARG;
  std::unique_ptr<hm_matrix> M;
  try {
    M.reset(new hm_matrix());
    HostMatrix& H = M->H;
    H.prm = *prm;
    H.n = n;
    H.kparam = prm->kparam > 0 ? prm->kparam
                               : (prm->kernel != HM_KERNEL_MATERN15 ? std::sqrt(4.0 * M_PI / (double)n) : 0.1);
    H.pts.assign(pts, pts + 3 * n);
    int nth = prm->nthreads > 0 ? prm->nthreads : (int)std::max(1u, std::thread::hardware_concurrency());
    build_cluster_tree(H.pts.data(), n, prm->leaf_size, H.ct);
    build_block_tree(H.ct, prm->eta, H.blocks, prm->adm);
    build_lowrank_blocks(H, nth);
    if (prm->format == HM_FMT_UH || prm->format == HM_FMT_UH_SEP) build_uniform_bases(H, nth);
    if (prm->format == HM_FMT_H2) build_nested_bases(H, nth);
  } catch (const std::bad_alloc&) {
    return HM_ERR_OOM;
  }
  *out = M.release();
  return HM_OK;
}

hm_status hm_compress(hm_matrix* M, double eps, int32_t codec, int32_t valr) {
  if (!M || !(eps > 0 && eps < 1)) return HM_ERR_ARG;
  if (codec < HM_CODEC_NONE || codec > HM_CODEC_FPX) return HM_ERR_ARG;
  std::lock_guard<std::mutex> g(M->mu);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HM_ERR_CUDA;
  cudaDeviceSynchronize();
  M->release_device();
  if (M->adj) {
    hm_free(M->adj);
    M->adj = nullptr;
  }
  bool ok;
  try {
    ok = build_program(M->H, codec, eps, valr, nsm, M->prog);
  } catch (const std::bad_alloc&) {
    return HM_ERR_OOM;
  }
  if (!ok) return M->prog.too_large ? HM_ERR_CAPACITY : HM_ERR_UNSUPPORTED;
  M->nsm = nsm;
  hm_status s = upload(M);
  if (s != HM_OK) {
    M->release_device();
    return s;
  }
  M->codec = codec;
  M->valr = valr ? 1 : 0;
  M->eps = eps;
  M->compressed = true;
  {   // code bytes by width, from the units' inline headers (in slices: bounded memory)
    std::fill(M->width_bytes, M->width_bytes + 8, 0);
    const int64_t nu = (int64_t)M->prog.items.size() + M->prog.npieces;
    std::vector<PackedCol> cols;
    for (int64_t u0 = 0; u0 < nu; u0 += 4096) {
      cols.clear();
      packed_columns(M->prog, u0, std::min(nu, u0 + 4096), cols);
      for (const PackedCol& c : cols) {
        const int B = c.fb & 15;
        if (B >= 1 && B <= 8) M->width_bytes[B - 1] += (int64_t)c.rows * B;
      }
    }
  }
  return HM_OK;
}

static cudaError_t run_launch(hm_matrix* M, const Launch& L, double alpha, const double* x, double beta, double* y,
                              cudaStream_t st) {
  Program& P = M->prog;
  const F2 aff = split_ff(alpha);
  const int cf = L.cfg;
  switch (L.kind) {
    case Launch::GATHER:
      return launch_gather(x, M->d_perm.p, (int)L.n, M->d_vec, st);
    case Launch::CDOT:
      return launch_cdot(P.tier, cf, M->d_items.p, M->d_wbeg.p + L.woff[cf], L.nw[cf], M->d_pay.p, M->d_vec, aff,
                         M->d_part, M->d_vec, M->d_err, st);
    case Launch::GSUM:
      if (L.scatter)   // with the fan-out folded into it
        return launch_gsum(M->d_gout.p + L.off, (int)L.n, M->d_pscale.p, M->d_part, aff, M->d_vec, M->d_fan_dst.p,
                           M->d_fcopy_src.p + L.copy_off, M->d_fcopy_dst.p + L.copy_off, (int)L.copy_n, st);
      return launch_gsum(M->d_gout.p + L.off, (int)L.n, M->d_pscale.p, M->d_part, aff, M->d_vec, nullptr, nullptr,
                         nullptr, 0, st);
    case Launch::FANOUT:
      return launch_fanout(M->d_fan.p + L.off, (int)L.n, M->d_vec + P.fan_base + L.off, M->d_vec, st);
    case Launch::RGEMV:
      return launch_rgemv(P.tier, L.mode, cf, M->d_pieces.p + (size_t)cf * P.npieces, M->d_wbeg.p + L.woff[cf],
                          L.nw[cf], M->d_pay.p, M->d_vec, alpha, aff, beta, y, M->d_perm.p, M->d_vec,
                          L.use_rowscale ? M->d_rowscale_ff.p : nullptr, M->d_fix, M->d_fixcnt, M->d_splits.p,
                          M->d_err, st);
  }
  return cudaErrorInvalidValue;
}

// One panel of r <= RP right-hand sides (FP32 tier): the same launch sequence
// with the multi-RHS kernels on the block-range split of every launch.
static cudaError_t run_launch_mr(hm_matrix* M, const Launch& L, double alpha, const double* x, int64_t ldx,
                                 double beta, double* y, int64_t ldy, int r, cudaStream_t st) {
  Program& P = M->prog;
  const F2 aff = split_ff(alpha);
  switch (L.kind) {
    case Launch::GATHER:
      return launch_gather_mr(x, ldx, r, M->d_perm.p, (int)L.n, M->d_vmr, st);
    case Launch::CDOT:
      if (M->mr_engine == 0)
        return launch_cdot_tc(M->d_items.p, M->d_wbeg.p + L.woff[MR_SHAPE], L.nw[MR_SHAPE], M->d_pay.p, M->d_vmr, aff,
                              M->d_pmr, M->d_vmr, M->d_err, st);
      return launch_cdot_ws(M->d_items.p, M->d_wbeg.p + L.woff[MR_SHAPE], L.nw[MR_SHAPE], M->d_pay.p, M->d_vmr, aff,
                            M->d_pmr, M->d_vmr, M->d_err, st);
    case Launch::GSUM:
      return launch_gsum_mr(M->d_gout.p + L.off, (int)L.n, M->d_pscale.p, M->d_pmr, aff, M->d_vmr, st);
    case Launch::FANOUT:   // the multi-RHS row-chunk kernel copies each multiplier row from its coefficient
      return cudaSuccess;
    case Launch::RGEMV:
      if (M->mr_engine == 0 || L.maxrows > MP_ROWS)
        return launch_rgemv_tc(L.mode, M->d_pieces.p + (size_t)MR_SHAPE * P.npieces, M->d_wbeg.p + L.woff[MR_SHAPE],
                               L.nw[MR_SHAPE], M->d_pay.p, M->d_vmr, alpha, aff, beta, y, ldy, r, M->d_perm.p,
                               M->d_vmr, L.use_rowscale ? M->d_rowscale_ff.p : nullptr, M->d_fixmr, M->d_fixcnt,
                               M->d_splits.p, M->d_fan.p, (int32_t)P.fan_base, M->d_err, st);
      return launch_rgemv_ms(L.mode, M->d_pieces.p + (size_t)MR_SHAPE * P.npieces, M->d_wbeg.p + L.woff[MR_SHAPE],
                             L.nw[MR_SHAPE], M->d_pay.p, M->d_vmr, alpha, aff, beta, y, ldy, r, M->d_perm.p, M->d_vmr,
                             L.use_rowscale ? M->d_rowscale_ff.p : nullptr, M->d_fixmr, M->d_fixcnt, M->d_splits.p,
                             M->d_fan.p, (int32_t)P.fan_base, M->d_err, st);
  }
  return cudaErrorInvalidValue;
}

static hm_status run_program_mr(hm_matrix* M, double alpha, const double* x, int64_t ldx, double beta, double* y,
                                int64_t ldy, int r, cudaStream_t st) {
  for (const Launch& L : M->prog.launches) {
    hm_matrix::Rec rec{(int)L.kind, nullptr, nullptr, L.bytes};
    if (M->prof) {
      rec.e0 = M->take_event();
      rec.e1 = M->take_event();
      cudaEventRecord(rec.e0, st);
    }
    if (run_launch_mr(M, L, alpha, x, ldx, beta, y, ldy, r, st) != cudaSuccess) return HM_ERR_CUDA;
    if (M->prof) {
      cudaEventRecord(rec.e1, st);
      M->recs.push_back(rec);
    }
  }
  return HM_OK;
}

static hm_status run_program(hm_matrix* M, double alpha, const double* x, double beta, double* y,
                             cudaStream_t st);

// All right-hand sides: panels of RP through the multi-RHS kernels (FP32
// tier), the rest (or everything in the float-float tier) as one single-RHS
// product per right-hand side.  A panel reads the matrix once; it costs about
// as much as MR_MIN_RHS single products on GB300, so smaller remainders run
// as single products.
constexpr int64_t MR_MIN_RHS = 9;
static hm_status run_all(hm_matrix* M, double alpha, const double* x, int64_t ldx, double beta, double* y,
                         int64_t ldy, int64_t nrhs, cudaStream_t st) {
  hm_status s = HM_OK;
  int64_t r0 = 0;
  if (M->d_vmr)   // panels of RP; a panel of fewer than MR_MIN_RHS is cheaper as single products
    for (; r0 < nrhs && nrhs - r0 >= MR_MIN_RHS && s == HM_OK; r0 += RP)
      s = run_program_mr(M, alpha, x + r0 * ldx, ldx, beta, y + r0 * ldy, ldy, (int)std::min<int64_t>(RP, nrhs - r0),
                         st);
  for (int64_t r = r0; r < nrhs && s == HM_OK; ++r) s = run_program(M, alpha, x + r * ldx, beta, y + r * ldy, st);
  return s;
}

static hm_status run_program(hm_matrix* M, double alpha, const double* x, double beta, double* y,
                             cudaStream_t st) {
  const auto& Ls = M->prog.launches;
  if (M->fuse == 2 && !M->prof && M->d_pstate) {   // the whole product as one launch
    Program& P = M->prog;
    return launch_prog(P.tier, M->nsm, M->d_prog.p, (int)M->d_prog.n, x, M->d_items.p, M->d_gout.p, M->d_pscale.p,
                       M->d_part, M->d_fan.p, M->d_pieces.p + (size_t)SEQ_SHAPE * P.npieces, M->d_wbeg.p,
                       M->d_phases.p, M->d_deps.p, M->d_pstate, M->pstate_n, M->d_pay.p, M->d_vec, alpha, beta, y,
                       M->d_perm.p, M->d_rowscale_ff.p, M->d_fix, M->d_fixcnt, M->d_splits.p, M->d_fan_dst.p,
                       M->d_fcopy_src.p, M->d_fcopy_dst.p, M->d_err,
                       st) == cudaSuccess
               ? HM_OK
               : HM_ERR_CUDA;
  }
  size_t ri = 0;
  for (size_t li = 0; li < Ls.size(); ++li) {
    const Launch& L = Ls[li];
    if (M->fuse && !M->prof && ri < M->runs.size() && M->runs[ri].first == li) {   // persistent run
      const hm_matrix::Run& R = M->runs[ri++];
      Program& P = M->prog;
      if (launch_rseq(P.tier, M->nsm, M->d_phases.p + R.ph0, (int)(R.last - R.first),
                      M->d_pieces.p + (size_t)SEQ_SHAPE * P.npieces, M->d_wbeg.p, M->d_pay.p, M->d_vec, alpha,
                      split_ff(alpha), beta, y, M->d_perm.p, M->d_rowscale_ff.p, M->d_fix, M->d_fixcnt,
                      M->d_splits.p, M->d_deps.p, M->d_ver, R.nchunks, M->d_err, st) != cudaSuccess)
        return HM_ERR_CUDA;
      li = R.last - 1;
      continue;
    }
    if (ri < M->runs.size() && M->runs[ri].first == li) ++ri;
    hm_matrix::Rec rec{(int)L.kind, nullptr, nullptr, L.bytes};
    if (M->prof) {
      rec.e0 = M->take_event();
      rec.e1 = M->take_event();
      cudaEventRecord(rec.e0, st);
    }
    if (run_launch(M, L, alpha, x, beta, y, st) != cudaSuccess) return HM_ERR_CUDA;
    if (M->prof) {
      cudaEventRecord(rec.e1, st);
      M->recs.push_back(rec);
    }
  }
  return HM_OK;
}

hm_status hm_matvec(hm_matrix* M, double alpha, const double* x, int64_t ldx, double beta, double* y,
                    int64_t ldy, int64_t nrhs, void* stream) {
  if (!M || !x || !y || nrhs < 1 || nrhs > 64) return HM_ERR_ARG;
  if (!M->compressed) return HM_ERR_STATE;
  const int64_t n = M->H.n;
  if (ldx < n || ldy < n) return HM_ERR_ARG;
  const double* xe = x + ldx * (nrhs - 1) + n;
  const double* ye = y + ldy * (nrhs - 1) + n;
  if (!(xe <= y || ye <= x)) return HM_ERR_ARG;     // x and y must not overlap
  cudaStream_t st = (cudaStream_t)stream;
  if (M->use_graph && !M->prof) {
    hm_matrix::GKey key{x, y, ldx, ldy, nrhs, alpha, beta};
    if (!M->gexec || !(key == M->gkey)) {
      M->drop_graph();
      if (!M->cap_stream && cudaStreamCreateWithFlags(&M->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return HM_ERR_CUDA;
      if (cudaStreamBeginCapture(M->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return HM_ERR_CUDA;
      hm_status s = run_all(M, alpha, x, ldx, beta, y, ldy, nrhs, M->cap_stream);
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(M->cap_stream, &g);
      if (s != HM_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return s != HM_OK ? s : HM_ERR_CUDA;
      }
      const cudaError_t ie = cudaGraphInstantiate(&M->gexec, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        M->gexec = nullptr;
        return HM_ERR_CUDA;
      }
      M->gkey = key;
    }
    return cudaGraphLaunch(M->gexec, st) == cudaSuccess ? HM_OK : HM_ERR_CUDA;
  }
  return run_all(M, alpha, x, ldx, beta, y, ldy, nrhs, st);
}

hm_status hm_graph(hm_matrix* M, int32_t enable) {
  if (!M) return HM_ERR_ARG;
  std::lock_guard<std::mutex> g(M->mu);
  M->use_graph = enable != 0;
  if (!M->use_graph) M->drop_graph();
  return HM_OK;
}

hm_status hm_persistent(hm_matrix* M, int32_t enable) {
  if (!M) return HM_ERR_ARG;
  std::lock_guard<std::mutex> g(M->mu);
  if (enable < 0 || enable > 2) return HM_ERR_ARG;
  M->fuse = enable;
  M->drop_graph();
  return HM_OK;
}

hm_status hm_matvec_host(hm_matrix* M, double alpha, const double* x, double beta, double* y, int64_t nrhs,
                         void* stream) {
  if (!M || !x || !y || nrhs < 1 || nrhs > 64) return HM_ERR_ARG;
  if (!M->compressed) return HM_ERR_STATE;
  const int64_t n = M->H.n;
  cudaStream_t st = (cudaStream_t)stream;
  if (M->d_h_cap < n * nrhs) {
    if (M->d_hx) cudaFree(M->d_hx);
    if (M->d_hy) cudaFree(M->d_hy);
    M->d_hx = M->d_hy = nullptr;
    M->d_h_cap = 0;
    if (cudaMalloc(&M->d_hx, n * nrhs * sizeof(double)) != cudaSuccess) return HM_ERR_OOM;
    if (cudaMalloc(&M->d_hy, n * nrhs * sizeof(double)) != cudaSuccess) return HM_ERR_OOM;
    M->d_h_cap = n * nrhs;
  }
  const size_t bytes = n * nrhs * sizeof(double);
  if (beta != 0.0) {   // y's copy on a second stream, after the stream's earlier work, overlapping x's
    if (!M->h_side && (cudaStreamCreateWithFlags(&M->h_side, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaEventCreateWithFlags(&M->h_ev0, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&M->h_ev1, cudaEventDisableTiming) != cudaSuccess))
      return HM_ERR_CUDA;
    if (cudaEventRecord(M->h_ev0, st) != cudaSuccess || cudaStreamWaitEvent(M->h_side, M->h_ev0, 0) != cudaSuccess ||
        cudaMemcpyAsync(M->d_hy, y, bytes, cudaMemcpyHostToDevice, M->h_side) != cudaSuccess ||
        cudaEventRecord(M->h_ev1, M->h_side) != cudaSuccess)
      return HM_ERR_CUDA;
  }
  if (cudaMemcpyAsync(M->d_hx, x, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return HM_ERR_CUDA;
  if (beta != 0.0 && cudaStreamWaitEvent(st, M->h_ev1, 0) != cudaSuccess) return HM_ERR_CUDA;
  hm_status s = hm_matvec(M, alpha, M->d_hx, n, beta, M->d_hy, n, nrhs, stream);
  if (s != HM_OK) return s;
  if (cudaMemcpyAsync(y, M->d_hy, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HM_ERR_CUDA;
  return HM_OK;
}

hm_status hm_matvec_adjoint(hm_matrix* M, double alpha, const double* x, int64_t ldx, double beta, double* y,
                            int64_t ldy, int64_t nrhs, void* stream) {
  if (!M || !x || !y || nrhs < 1 || nrhs > 64) return HM_ERR_ARG;
  hm_matrix* A = nullptr;
  {
    std::lock_guard<std::mutex> g(M->mu);
    if (!M->compressed) return HM_ERR_STATE;
    if (!M->adj) {   // first adjoint product: transpose, compress with the same settings, upload
      std::unique_ptr<hm_matrix> T;
      try {
        T.reset(new hm_matrix());
        transpose_host(M->H, T->H);
      } catch (const std::bad_alloc&) {
        return HM_ERR_OOM;
      }
      if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return HM_ERR_CUDA;
      const hm_status s = hm_compress(T.get(), M->eps, M->codec, M->valr);
      if (s != HM_OK) return s;
      M->adj = T.release();
    }
    M->adj->use_graph = M->use_graph;
    M->adj->fuse = M->fuse;
    A = M->adj;
  }
  return hm_matvec(A, alpha, x, ldx, beta, y, ldy, nrhs, stream);
}

hm_status hm_autotune(hm_matrix* M, int32_t reps, void* stream) {
  if (!M || reps < 1 || reps > 1000) return HM_ERR_ARG;
  std::lock_guard<std::mutex> g(M->mu);
  if (!M->compressed) return HM_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = M->H.n;
  double *x = nullptr, *y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hm_status out = HM_OK;
  if (cudaMalloc(&x, n * sizeof(double)) != cudaSuccess || cudaMalloc(&y, n * sizeof(double)) != cudaSuccess ||
      cudaMemsetAsync(x, 0, n * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(y, 0, n * sizeof(double), st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    out = HM_ERR_CUDA;
  }
  if (out == HM_OK && run_program(M, 1.0, x, 0.0, y, st) != HM_OK) out = HM_ERR_CUDA;   // warm-up
  for (Launch& L : M->prog.launches) {
    if (out != HM_OK) break;
    if (L.kind != Launch::CDOT && L.kind != Launch::RGEMV) continue;
    float best = 0.f;
    int bestc = 0;
    for (int cf = 0; cf < NCFG && out == HM_OK; ++cf) {
      L.cfg = cf;
      if (run_launch(M, L, 1.0, x, 0.0, y, st) != cudaSuccess) out = HM_ERR_CUDA;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && out == HM_OK; ++r)
        if (run_launch(M, L, 1.0, x, 0.0, y, st) != cudaSuccess) out = HM_ERR_CUDA;
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        out = HM_ERR_CUDA;
      if (cf == 0 || ms < best) {
        best = ms;
        bestc = cf;
      }
    }
    L.cfg = bestc;
  }
  // then how the launches run: one launch per step (with the tuned shapes),
  // fused runs of row-chunk steps, or the whole product as one launch --
  // whole products timed, the fastest kept
  {
    float best = 0.f;
    int bestm = M->fuse;
    for (int mode = 0; mode <= 2 && out == HM_OK; ++mode) {
      if (mode == 2 && !M->d_pstate) continue;
      if (mode == 1 && M->runs.empty()) continue;   // same launches as mode 0
      M->fuse = mode;
      if (run_program(M, 1.0, x, 0.0, y, st) != HM_OK) out = HM_ERR_CUDA;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && out == HM_OK; ++r)
        if (run_program(M, 1.0, x, 0.0, y, st) != HM_OK) out = HM_ERR_CUDA;
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        out = HM_ERR_CUDA;
      if (mode == 0 || ms < best) {
        best = ms;
        bestm = mode;
      }
    }
    M->fuse = bestm;
  }
  // multi-RHS panels (FP32 tier): the row-chunk engine, whole RP-wide panels timed
  double *xp = nullptr, *yp = nullptr;
  if (out == HM_OK && M->d_vmr) {
    const size_t pb = (size_t)n * RP * sizeof(double);
    if (cudaMalloc(&xp, pb) != cudaSuccess || cudaMalloc(&yp, pb) != cudaSuccess ||
        cudaMemsetAsync(xp, 0, pb, st) != cudaSuccess)
      out = HM_ERR_CUDA;
    float best = 0.f;
    int beste = M->mr_engine;
    for (int eng = 0; eng <= 1 && out == HM_OK; ++eng) {
      M->mr_engine = eng;
      if (run_program_mr(M, 1.0, xp, n, 0.0, yp, n, RP, st) != HM_OK) out = HM_ERR_CUDA;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && out == HM_OK; ++r)
        if (run_program_mr(M, 1.0, xp, n, 0.0, yp, n, RP, st) != HM_OK) out = HM_ERR_CUDA;
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        out = HM_ERR_CUDA;
      if (eng == 0 || ms < best) {
        best = ms;
        beste = eng;
      }
    }
    M->mr_engine = beste;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && out == HM_OK) out = HM_ERR_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (x) cudaFree(x);
  if (y) cudaFree(y);
  if (xp) cudaFree(xp);
  if (yp) cudaFree(yp);
  M->drop_graph();
  return out;
}

hm_status hm_launch_shapes(const hm_matrix* M, int32_t* shapes, int32_t cap, int32_t* count) {
  if (!M || !count || cap < 0 || (cap > 0 && !shapes)) return HM_ERR_ARG;
  const auto& Ls = M->prog.launches;
  *count = (int32_t)Ls.size();
  for (int32_t i = 0; i < cap && i < (int32_t)Ls.size(); ++i)
    shapes[i] = (Ls[i].kind == Launch::CDOT || Ls[i].kind == Launch::RGEMV) ? Ls[i].cfg : -1;
  return HM_OK;
}

hm_status hm_persistent_mode(const hm_matrix* M, int32_t* mode) {
  if (!M || !mode) return HM_ERR_ARG;
  *mode = M->fuse;
  return HM_OK;
}

hm_status hm_set_multi_rhs_engine(hm_matrix* M, int32_t engine) {
  if (!M || engine < 0 || engine > 1) return HM_ERR_ARG;
  std::lock_guard<std::mutex> g(M->mu);
  M->mr_engine = engine;
  return HM_OK;
}

hm_status hm_multi_rhs_engine(const hm_matrix* M, int32_t* engine) {
  if (!M || !engine) return HM_ERR_ARG;
  *engine = M->mr_engine;
  return HM_OK;
}

// Tuning record: TUNE_MAGIC, version, the fingerprint (2 words), the launch
// count, every launch's shape, the launch mode, the multi-RHS engine.  The
// fingerprint hashes (FNV-1a) the device's SM count and name and the program's
// structure (tier, every launch's kind, mode, unit range and warp-range counts),
// so a record applies only to a matrix whose launches it was timed on.
constexpr int32_t TUNE_MAGIC = 0x484d5455;   // "HMTU"
constexpr int32_t TUNE_VERSION = 1;

static uint64_t tuning_fingerprint(const hm_matrix* M) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xffu;
      h *= 1099511628211ull;
    }
  };
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
    for (const char* c = prop.name; *c; ++c) mix((uint64_t)(unsigned char)*c);
  mix((uint64_t)M->nsm);
  const Program& P = M->prog;
  mix((uint64_t)P.tier);
  for (const Launch& L : P.launches) {
    mix((uint64_t)L.kind | ((uint64_t)L.mode << 8));
    mix((uint64_t)L.off);
    mix((uint64_t)L.n);
    for (int cf = 0; cf < NSHAPES; ++cf) mix((uint64_t)L.nw[cf]);
  }
  return h;
}

hm_status hm_tuning(const hm_matrix* M, int32_t* rec, int32_t cap, int32_t* len) {
  if (!M || !len || cap < 0 || (cap > 0 && !rec)) return HM_ERR_ARG;
  if (!M->compressed) return HM_ERR_STATE;
  const auto& Ls = M->prog.launches;
  const uint64_t fp = tuning_fingerprint(M);
  std::vector<int32_t> v = {TUNE_MAGIC, TUNE_VERSION, (int32_t)(uint32_t)fp, (int32_t)(uint32_t)(fp >> 32),
                            (int32_t)Ls.size()};
  for (const Launch& L : Ls) v.push_back(L.cfg);
  v.push_back(M->fuse);
  v.push_back(M->mr_engine);
  *len = (int32_t)v.size();
  for (int32_t i = 0; i < cap && i < (int32_t)v.size(); ++i) rec[i] = v[i];
  return HM_OK;
}

hm_status hm_set_tuning(hm_matrix* M, const int32_t* rec, int32_t len) {
  if (!M || !rec || len < 7) return HM_ERR_ARG;
  std::lock_guard<std::mutex> g(M->mu);
  if (!M->compressed) return HM_ERR_STATE;
  auto& Ls = M->prog.launches;
  const uint64_t fp = tuning_fingerprint(M);
  if (rec[0] != TUNE_MAGIC || rec[1] != TUNE_VERSION || rec[2] != (int32_t)(uint32_t)fp ||
      rec[3] != (int32_t)(uint32_t)(fp >> 32) || rec[4] != (int32_t)Ls.size() || len != 7 + (int32_t)Ls.size())
    return HM_ERR_ARG;
  for (size_t i = 0; i < Ls.size(); ++i)
    if (rec[5 + i] < 0 || rec[5 + i] >= NCFG) return HM_ERR_ARG;
  const int32_t mode = rec[5 + Ls.size()], eng = rec[6 + Ls.size()];
  if (mode < 0 || mode > 2 || eng < 0 || eng > 1) return HM_ERR_ARG;
  for (size_t i = 0; i < Ls.size(); ++i) Ls[i].cfg = rec[5 + i];
  M->fuse = mode;
  M->mr_engine = eng;
  M->drop_graph();
  return HM_OK;
}

hm_status hm_set_launch_shapes(hm_matrix* M, int32_t shape) {
  if (!M || shape < 0 || shape >= NCFG) return HM_ERR_ARG;
  std::lock_guard<std::mutex> g(M->mu);
  for (Launch& L : M->prog.launches) L.cfg = shape;
  M->drop_graph();
  return HM_OK;
}

hm_status hm_profile(hm_matrix* M, int32_t enable) {
  if (!M) return HM_ERR_ARG;
  M->prof = enable != 0;
  return HM_OK;
}

hm_status hm_profile_read(hm_matrix* M, hm_kernel_stat* out, int32_t nout) {
  if (!M || !out || nout < 0 || nout > 5) return HM_ERR_ARG;
  hm_kernel_stat acc[5];
  std::memset(acc, 0, sizeof(acc));
  hm_status st = HM_OK;
  for (auto& r : M->recs) {
    float ms = 0;
    if (cudaEventSynchronize(r.e1) != cudaSuccess || cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess)
      st = HM_ERR_CUDA;
    acc[r.kind].ms += ms;
    acc[r.kind].launches += 1;
    acc[r.kind].bytes += r.bytes;
    M->evpool.push_back(r.e0);
    M->evpool.push_back(r.e1);
  }
  M->recs.clear();
  for (int i = 0; i < nout; ++i) out[i] = acc[i];
  return st;
}

hm_status hm_alg_bytes(const hm_matrix* M, int64_t* bytes) {
  if (!M || !bytes) return HM_ERR_ARG;
  int64_t b = 0;
  for (const Launch& L : M->prog.launches) b += L.bytes;
  *bytes = b;
  return HM_OK;
}

hm_status hm_free(hm_matrix* M) {
  if (!M) return HM_OK;
  if (M->h_side) cudaStreamDestroy(M->h_side);
  if (M->h_ev0) cudaEventDestroy(M->h_ev0);
  if (M->h_ev1) cudaEventDestroy(M->h_ev1);
  if (M->adj) hm_free(M->adj);
  M->adj = nullptr;
  M->drop_graph();
  if (M->cap_stream) cudaStreamDestroy(M->cap_stream);
  for (auto& r : M->recs) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  for (auto e : M->evpool) cudaEventDestroy(e);
  M->release_device();
  delete M;
  return HM_OK;
}

hm_status hm_sync_status(hm_matrix* M, void* stream) {
  if (!M) return HM_ERR_ARG;
  if (!M->d_err) return HM_OK;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return HM_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, M->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HM_ERR_CUDA;
  if (v != 0) {
    cudaMemset(M->d_err, 0, sizeof(int));
    return v == 99 ? HM_ERR_TIMEOUT : HM_ERR_DEVICE;
  }
  return HM_OK;
}

hm_status hm_info(const hm_matrix* M, hm_info_t* o) {
  if (!M || !o) return HM_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  const HostMatrix& H = M->H;
  o->n = H.n;
  o->format = H.prm.format;
  o->codec = M->codec;
  o->valr = M->valr;
  o->eps = M->compressed ? M->eps : 0.0;
  o->nclusters = (int64_t)H.ct.cl.size();
  for (const auto& c : H.ct.cl)
    if (c.leaf()) o->nleaves++;
  o->nblocks = (int64_t)H.blocks.size();
  o->nlowrank = (int64_t)H.lr.size();
  o->ndense = (int64_t)H.dn.size();
  o->depth = H.ct.depth;
  for (const auto& L : H.lr) o->max_rank = std::max(o->max_rank, L.k);
  const Program& P = M->prog;
  o->bytes_fp64 = P.fp64_lowrank + P.fp64_dense;
  o->bytes_lowrank_fp64 = P.fp64_lowrank;
  o->bytes_dense_fp64 = P.fp64_dense;
  o->bytes_payload = (int64_t)P.pk.pay.size();
  o->bytes_values = P.pk.value_bytes;
  o->bytes_meta = P.pk.meta_bytes +
                  (int64_t)(P.items.size() * sizeof(ItemCopy) + NSHAPES * P.npieces * sizeof(PieceCopy) +
                            P.wbeg.size() * 4 + P.splits.size() * sizeof(Split) + P.gouts.size() * sizeof(GsumOut) +
                            P.pscale.size() * 8 + P.rowscale.size() * 8 +
                            (P.fan_src.size() + P.fan_dst.size() + 2 * P.fan_copy_src.size()) * 4) +
                  H.n * 4;
  o->bytes_workspace = P.nvec * 8 + P.npartial * 8 + P.nfix * CHUNK_ROWS * 8;
  if (M->d_vmr)
    o->bytes_workspace += ((P.fan_base + SEG_ROWS) + P.npartial) * RP * 4 + P.nfix_mr * CHUNK_ROWS * RP * 8;
  o->nlaunches = (int64_t)P.launches.size();
  o->tier = P.tier;
  o->nunits = (int64_t)P.items.size() + P.npieces;
  o->bytes_inline_meta = P.pk.meta_bytes;
  o->bytes_alg = M->compressed ? P.pk.value_bytes + P.pk.meta_bytes + 24 * H.n + 16 * (P.fan_base - H.n) : 0;
  for (int b = 0; b < 8; ++b) o->bytes_by_width[b] = M->width_bytes[b];
  return HM_OK;
}

hm_status hm_structure(const hm_matrix* M, int64_t* perm, int64_t* clusters, int64_t* blocks, int32_t* ranks) {
  if (!M) return HM_ERR_ARG;
  const HostMatrix& H = M->H;
  if (perm)
    for (int64_t i = 0; i < H.n; ++i) perm[i] = H.ct.perm[i];
  if (clusters)
    for (size_t c = 0; c < H.ct.cl.size(); ++c) {
      clusters[4 * c + 0] = H.ct.cl[c].start;
      clusters[4 * c + 1] = H.ct.cl[c].end;
      clusters[4 * c + 2] = H.ct.cl[c].level;
      clusters[4 * c + 3] = H.ct.cl[c].parent;
    }
  if (blocks)
    for (size_t b = 0; b < H.blocks.size(); ++b) {
      blocks[3 * b + 0] = H.blocks[b].row;
      blocks[3 * b + 1] = H.blocks[b].col;
      blocks[3 * b + 2] = H.blocks[b].adm ? 1 : 0;
    }
  if (ranks)
    for (size_t b = 0; b < H.blocks.size(); ++b)
      ranks[b] = H.blocks[b].adm ? H.lr[H.slot[b]].k : -1;
  return HM_OK;
}

hm_status hm_codec_encode(const double* v, int64_t n, int32_t codec, int32_t key, uint8_t* out, int64_t cap,
                          hm_codec_header* hdr) {
  if ((!v && n > 0) || !out || !hdr || n < 0 || key < 0 || key > 60) return HM_ERR_ARG;
  if (codec != HM_CODEC_AFLP && codec != HM_CODEC_FPX && codec != HM_CODEC_NONE) return HM_ERR_ARG;
  std::vector<uint64_t> codes(std::max<int64_t>(n, 1));
  CodeHdr h;
  if (!encode_values(v, n, 1, codec, key, h, codes.data())) return HM_ERR_ARG;
  if (cap < n * h.B) return HM_ERR_ARG;
  for (int64_t i = 0; i < n; ++i)
    for (int b = 0; b < h.B; ++b) out[i * h.B + b] = (uint8_t)(codes[i] >> (8 * b));
  hdr->B = h.B;
  hdr->fmt = h.fmt;
  hdr->e = h.e;
  hdr->m = h.m;
  hdr->vmin = h.vmin;
  return HM_OK;
}

hm_status hm_codec_decode(const uint8_t* packed, int64_t n, const hm_codec_header* h, double* out,
                          void* stream) {
  if (!h || n < 0 || (n > 0 && (!packed || !out))) return HM_ERR_ARG;
  if (h->B < 1 || h->B > 8 || h->fmt < 0 || h->fmt > 3) return HM_ERR_ARG;
  if (h->fmt == FMT_AFLP && (h->e < 1 || h->m < 1 || 1 + h->e + h->m != 8 * h->B)) return HM_ERR_ARG;
  cudaError_t e = launch_decode(packed, n, h->B, h->fmt, h->e, h->m, h->vmin, out, (cudaStream_t)stream);
  return e == cudaSuccess ? HM_OK : HM_ERR_CUDA;
}

hm_status hm_decompress_debug(hm_matrix* M, int32_t tier, int64_t u0, int64_t u1, int64_t cap, float* head,
                              float* tail, uint64_t* code, uint16_t* fmt, int64_t* count, void* stream) {
  if (!M || !count || (tier != TIER_F32 && tier != TIER_FF) || u0 < 0 || u1 < u0) return HM_ERR_ARG;
  if (!M->compressed) return HM_ERR_STATE;
  const Program& P = M->prog;
  const int64_t nunits = (int64_t)P.items.size() + P.npieces;
  u1 = std::min(u1, nunits);
  u0 = std::min(u0, u1);
  std::vector<PackedCol> cols;
  try {
    packed_columns(P, u0, u1, cols);
  } catch (const std::bad_alloc&) {
    return HM_ERR_OOM;
  }
  int64_t nv = 0;
  for (const PackedCol& c : cols) nv += c.rows;
  *count = nv;
  if (!head) return HM_OK;
  if (!tail || !code || !fmt || cap < nv) return HM_ERR_ARG;
  if (nv == 0) return HM_OK;
  std::vector<DbgTask> tasks;
  const uint8_t* pay = P.pk.pay.data();
  int64_t v = 0;
  for (const PackedCol& c : cols) {
    const int B = c.fb & 15;
    const uint16_t f16 = (uint16_t)(B | (((c.fb >> 4) & 3) << 4) | ((c.em & 0xf) << 6) | (((c.em >> 8) & 0x3f) << 10));
    for (int r = 0; r < c.rows; ++r) {
      uint64_t cv = 0;
      for (int b = 0; b < B; ++b) cv |= (uint64_t)pay[c.off + (uint64_t)r * B + b] << (8 * b);
      code[v + r] = cv;
      fmt[v + r] = f16;
    }
    for (int q = 0; q * RPL < c.rows; ++q)
      tasks.push_back(DbgTask{c.off + (uint64_t)q * RPL * B, (uint32_t)c.fb | ((uint32_t)c.em << 16),
                              (int32_t)(v + q * RPL), std::min(RPL, c.rows - q * RPL), 0});
    v += c.rows;
  }
  if (nv > (int64_t)INT32_MAX) return HM_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  DbgTask* dt = nullptr;
  float2* dout = nullptr;
  hm_status out = HM_OK;
  if (cudaMalloc(&dt, tasks.size() * sizeof(DbgTask)) != cudaSuccess ||
      cudaMalloc(&dout, (size_t)nv * sizeof(float2)) != cudaSuccess) {
    out = HM_ERR_OOM;
  } else if (cudaMemcpyAsync(dt, tasks.data(), tasks.size() * sizeof(DbgTask), cudaMemcpyHostToDevice, st) !=
                 cudaSuccess ||
             launch_decode_debug(tier, dt, (int64_t)tasks.size(), M->d_pay.p, dout, M->d_err, st) != cudaSuccess) {
    out = HM_ERR_CUDA;
  } else {
    std::vector<float2> hv((size_t)nv);
    if (cudaMemcpyAsync(hv.data(), dout, (size_t)nv * sizeof(float2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      out = HM_ERR_CUDA;
    } else {
      for (int64_t i = 0; i < nv; ++i) {
        head[i] = hv[i].x;
        tail[i] = hv[i].y;
      }
    }
  }
  if (dt) cudaFree(dt);
  if (dout) cudaFree(dout);
  return out;
}

}  // extern "C"
