// Host H-LU factorisation (Sec. 5, Conclusion: the factors whose triangular
// solves hlu.cu runs): dense elimination without pivoting in the cluster order,
// then the factors cut along the block tree of A, admissible blocks truncated
// by the rule of eqn. epsilon.  No GPU code (the host check links it alone).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

#include "program.h"

namespace hm {

namespace {

// In-place Doolittle elimination without pivoting of the n x n column-major
// array a: afterwards its strict lower part is L (unit diagonal implied) and
// its upper part U.  False if a pivot is zero or not finite.
bool lu_inplace(double* a, int64_t n, int nth) {
  for (int64_t k = 0; k < n; ++k) {
    const double piv = a[k + k * n];
    if (!(std::isfinite(piv) && piv != 0.0)) return false;
    double* col = a + k * n;
    for (int64_t i = k + 1; i < n; ++i) col[i] /= piv;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int64_t j = k + 1; j < n; ++j) {
      double* cj = a + j * n;
      const double u = cj[k];
      if (u == 0.0) continue;
      for (int64_t i = k + 1; i < n; ++i) cj[i] -= col[i] * u;
    }
  }
  return true;
}

void init_factor(HostMatrix& F, const hm_build_params& prm, int64_t n, double kparam, const double* pts,
                 const ClusterTree& ct) {
  F.prm = prm;
  F.n = n;
  F.kparam = kparam;
  F.pts.assign(pts, pts + 3 * n);
  F.ct = ct;
}

}  // namespace

bool lu_factor_host(const hm_build_params& prm, const double* pts, int64_t n, HostMatrix& L, HostMatrix& U) {
  const int nth = prm.nthreads > 0 ? prm.nthreads : (int)std::max(1u, std::thread::hardware_concurrency());
  const double kparam = prm.kparam > 0 ? prm.kparam
                                       : (prm.kernel != HM_KERNEL_MATERN15 ? std::sqrt(4.0 * M_PI / (double)n) : 0.1);
  ClusterTree ct;
  build_cluster_tree(pts, n, prm.leaf_size, ct);
  std::vector<BlockLeaf> blocks;
  build_block_tree(ct, prm.eta, blocks, prm.adm);
  KernelFn f;
  f.kind = prm.kernel;
  f.param = kparam;
  f.pts = pts;
  std::vector<double> a((size_t)(n * n));
#pragma omp parallel for schedule(static) num_threads(nth)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) a[i + j * n] = f(ct.perm[i], ct.perm[j]);
  if (!lu_inplace(a.data(), n, nth)) return false;
  L = HostMatrix();
  U = HostMatrix();
  init_factor(L, prm, n, kparam, pts, ct);
  init_factor(U, prm, n, kparam, pts, ct);
  struct Job {
    HostMatrix* F;
    int64_t slot;
    int row, col;
  };
  std::vector<Job> jobs;
  for (const BlockLeaf& b : blocks) {
    const Cluster& t = ct.cl[b.row];
    const Cluster& s = ct.cl[b.col];
    if (b.row == b.col) {   // diagonal leaf: unit lower triangle to L, upper triangle to U
      for (int side = 0; side < 2; ++side) {
        HostMatrix& Fm = side == 0 ? L : U;
        Fm.blocks.push_back(BlockLeaf{b.row, b.col, false});
        Fm.slot.push_back((int)Fm.dn.size());
        DenseBlock D;
        const int64_t m = t.size();
        D.D.assign((size_t)(m * m), 0.0);
        for (int64_t j = 0; j < m; ++j)
          for (int64_t i = 0; i < m; ++i) {
            const double v = a[(t.start + i) + (t.start + j) * n];
            if (side == 0)
              D.D[i + j * m] = i > j ? v : (i == j ? 1.0 : 0.0);
            else
              D.D[i + j * m] = i <= j ? v : 0.0;
          }
        Fm.dn.push_back(std::move(D));
      }
      continue;
    }
    HostMatrix& Fm = t.start >= s.end ? L : U;   // t after s: L; t before s: U
    Fm.blocks.push_back(b);
    if (b.adm) {
      Fm.slot.push_back((int)Fm.lr.size());
      Fm.lr.emplace_back();
      jobs.push_back(Job{&Fm, (int64_t)Fm.lr.size() - 1, b.row, b.col});
    } else {
      Fm.slot.push_back((int)Fm.dn.size());
      DenseBlock D;
      D.D.resize((size_t)(t.size() * s.size()));
      for (int64_t j = 0; j < s.size(); ++j)
        std::memcpy(&D.D[j * t.size()], &a[t.start + (s.start + j) * n], (size_t)t.size() * 8);
      Fm.dn.push_back(std::move(D));
    }
  }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nth)
  for (int64_t k = 0; k < (int64_t)jobs.size(); ++k) {
    const Job& jb = jobs[k];
    const Cluster& t = ct.cl[jb.row];
    const Cluster& s = ct.cl[jb.col];
    lowrank_dense(&a[t.start + s.start * n], n, t.size(), s.size(), prm.eps_build, jb.F->lr[jb.slot]);
  }
  return true;
}

}  // namespace hm
