// Internal host-side data structures of libhm (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hm.h"

namespace hm {

// ---------------------------------------------------------------- trees
struct Cluster {
  int64_t start = 0, end = 0;   // range in the cluster (permuted) order
  int level = 0;
  int parent = -1;
  int son[2] = {-1, -1};
  int nsons = 0;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  int64_t size() const { return end - start; }
  bool leaf() const { return nsons == 0; }
};

struct ClusterTree {
  std::vector<Cluster> cl;      // pre-order, cl[0] = root
  std::vector<int64_t> perm;    // perm[position] = original index
  int depth = 0;
};

struct BlockLeaf {
  int row = 0, col = 0;
  bool adm = false;
};

void build_cluster_tree(const double* pts, int64_t n, int leaf, ClusterTree& ct);
void build_block_tree(const ClusterTree& ct, double eta, std::vector<BlockLeaf>& out, int mode = HM_ADM_STANDARD);

// ---------------------------------------------------------------- dense algebra (column-major)
// Thin Householder QR of an m x n matrix (m >= n or not): A = Q R, Q m x r, R r x n, r = min(m, n).
void qr_thin(int64_t m, int64_t n, const double* A, int64_t lda, std::vector<double>& Q,
             std::vector<double>& R);
// SVD of a small m x n matrix by one-sided Jacobi: A = U diag(s) V^T, s descending, r = min(m,n).
void svd_jacobi(int64_t m, int64_t n, const double* A, int64_t lda, std::vector<double>& U,
                std::vector<double>& s, std::vector<double>& V);

// ---------------------------------------------------------------- kernel entries
struct KernelFn {
  int kind = HM_KERNEL_LAPLACE;
  double param = 1.0;   // Laplace diagonal spacing h / Matern length scale
  const double* pts = nullptr;
  double operator()(int64_t i, int64_t j) const;   // original indices
};

// ---------------------------------------------------------------- H-matrix data
struct LowRankBlock {
  int k = 0;
  std::vector<double> W;   // n_t x k, orthonormal columns
  std::vector<double> s;   // k singular values, descending
  std::vector<double> X;   // n_s x k, orthonormal columns
};

struct DenseBlock {
  std::vector<double> D;   // n_t x n_s, column-major
};

// Shared or nested cluster bases of one side (rows: W, columns: X).
struct Bases {
  std::vector<std::vector<double>> B;       // explicit basis per cluster (UH: all; H2: leaves)
  std::vector<std::vector<double>> sig;     // singular values per cluster (VALR weights)
  std::vector<std::vector<double>> E;       // H2 transfer per non-root cluster (k_child x k_parent)
  std::vector<int> k;                       // rank per cluster
  double tau = 0;                           // truncation threshold the bases were built with
};

struct HostMatrix {
  hm_build_params prm{};
  int64_t n = 0;
  double kparam = 0;
  std::vector<double> pts;
  ClusterTree ct;
  std::vector<BlockLeaf> blocks;
  std::vector<int> slot;                    // per block: index into lr (adm) or dn (dense)
  std::vector<LowRankBlock> lr;
  std::vector<DenseBlock> dn;
  // UH / H2
  Bases rowb, colb;
  std::vector<std::vector<double>> coupling;   // per low-rank block (k_t x k_s), col-major
  // UH_SEP: the two factors of each coupling, S = Sr Sc^T, per low-rank block:
  // Sr (k_t x k_b) and Sc^T (k_b x k_s), col-major
  std::vector<std::vector<double>> coupling_r, coupling_ct;
};

void build_lowrank_blocks(HostMatrix& hm, int nthreads);
// Low-rank approximation of a dense m x n block (column-major, leading dimension
// lda) by ACA, QR and SVD recompression, truncated at sigma_k <= eps sigma_0.
void lowrank_dense(const double* A, int64_t lda, int64_t m, int64_t n, double eps, LowRankBlock& out);
void build_uniform_bases(HostMatrix& hm, int nthreads);
void build_nested_bases(HostMatrix& hm, int nthreads);
// The transpose: blocks (t, s) -> (s, t) with W and X, row and column bases and
// their transfer matrices swapped, dense blocks and couplings transposed.
void transpose_host(const HostMatrix& H, HostMatrix& T);

// ---------------------------------------------------------------- codecs (Sec. 4.1)
enum { FMT_FPX8 = 0, FMT_FPX11 = 1, FMT_AFLP = 2, FMT_RAW = 3 };

struct CodeHdr {
  int B = 8, fmt = FMT_RAW, e = 0, m = 52;
  double vmin = 1.0;
};

int ceil_log2(double r);
int m_eps(double eps);
int valr_key(double sigma, double delta);
void fpx_format(int key, int& e, int& m);
// Encode n values read with stride `inc`; codes[i] gets the 8*B-bit code.
bool encode_values(const double* v, int64_t n, int64_t inc, int codec, int key, CodeHdr& hdr,
                   uint64_t* codes);
double decode_value(uint64_t code, const CodeHdr& h);   // host reference decode (FP64)

}  // namespace hm
