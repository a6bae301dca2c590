// Host construction of H-, UH- and H^2-matrices (Sec. 2.2-2.4).
//
// Low-rank blocks: adaptive cross approximation with partial pivoting to
// eps/10 (Frobenius estimate), then recompression U = Q_U R_U, V = Q_V R_V,
// SVD of R_U R_V^T, truncated at the smallest k with sigma_k <= eps*sigma_0
// (eqn. epsilon, spectral reading).  Dense blocks hold the exact entries.
//
// UH (Sec. 2.3): the row basis of cluster t spans the concatenated
// W_b diag(s_b)/||s_b||_2 of its block row (singular values > eps kept); the
// column basis likewise; coupling S_b = (W_t^T W_b) diag(s_b) (X_b^T X_s).
//
// H^2 (Sec. 2.4): the basis of t represents every low-rank block of the block
// rows of t and of its ancestors restricted to t, each scaled to unit
// Frobenius norm; leaves take the SVD of that data, inner clusters the SVD of
// the data projected on the sons' bases, giving the transfer matrices
// E_t,i = Q[rows of son i].  Threshold eps/sqrt(depth+1) per level so the
// errors of all levels add to at most eps per block.  Couplings
// S_b = P_t,b diag(s_b) P_s,b^T with P_t,b = W_t^T W_b[t,:], obtained from the
// leaves upwards as P_t,b = sum_i E_ti^T P_ti,b.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include <omp.h>

#include "hm_internal.h"

namespace hm {

double KernelFn::operator()(int64_t i, int64_t j) const {
  const double* p = pts + 3 * i;
  if (kind == HM_KERNEL_LAPLACE_W)   // row weight w_i = 1 + x_i / 2 times the Laplace entry
    return (1.0 + 0.5 * p[0]) * KernelFn{HM_KERNEL_LAPLACE, param, pts}(i, j);
  if (i == j) return kind == HM_KERNEL_LAPLACE ? 1.0 / (4.0 * M_PI * param) : 1.0;
  const double* q = pts + 3 * j;
  double d0 = p[0] - q[0], d1 = p[1] - q[1], d2 = p[2] - q[2];
  double r = std::sqrt((d0 * d0 + d1 * d1) + d2 * d2);
  if (kind == HM_KERNEL_LAPLACE) return 1.0 / (4.0 * M_PI * r);
  double t = std::sqrt(3.0) * r / param;
  return (1.0 + t) * std::exp(-t);
}

namespace {

// ACA with partial pivoting; returns U (m x k), V (n x k), A ~ U V^T.
// f(i, j): entry of row rows[i], column cols[j] (a kernel function, or a dense array).
template <class Fn>
int aca(const Fn& f, const int64_t* rows, int64_t m, const int64_t* cols, int64_t n,
        double eps, std::vector<double>& U, std::vector<double>& V) {
  const int64_t kmax = std::min(m, n);
  U.clear();
  V.clear();
  std::vector<char> used(m, 0);
  std::vector<double> row(n), col(m);
  double norm2 = 0.0;
  int64_t i = 0;
  int k = 0, small = 0;
  int64_t nused = 0;
  while (k < kmax && nused < m) {
    used[i] = 1;
    ++nused;
    for (int64_t j = 0; j < n; ++j) row[j] = f(rows[i], cols[j]);
    for (int l = 0; l < k; ++l) {
      double u = U[l * m + i];
      if (u == 0.0) continue;
      const double* v = &V[l * n];
      for (int64_t j = 0; j < n; ++j) row[j] -= u * v[j];
    }
    int64_t js = 0;
    double amax = 0.0;
    for (int64_t j = 0; j < n; ++j)
      if (std::fabs(row[j]) > amax) {
        amax = std::fabs(row[j]);
        js = j;
      }
    if (amax == 0.0) {                 // zero residual row: try the next unused row
      int64_t nxt = -1;
      for (int64_t r = 0; r < m; ++r)
        if (!used[r]) {
          nxt = r;
          break;
        }
      if (nxt < 0) break;
      i = nxt;
      continue;
    }
    double piv = row[js];
    for (int64_t j = 0; j < n; ++j) row[j] /= piv;
    for (int64_t r = 0; r < m; ++r) col[r] = f(rows[r], cols[js]);
    for (int l = 0; l < k; ++l) {
      double v = V[l * n + js];
      if (v == 0.0) continue;
      const double* u = &U[l * m];
      for (int64_t r = 0; r < m; ++r) col[r] -= v * u[r];
    }
    double nu2 = 0, nv2 = 0;
    for (int64_t r = 0; r < m; ++r) nu2 += col[r] * col[r];
    for (int64_t j = 0; j < n; ++j) nv2 += row[j] * row[j];
    double cross = 0;
    for (int l = 0; l < k; ++l) {
      const double* u = &U[l * m];
      const double* v = &V[l * n];
      double a = 0, b = 0;
      for (int64_t r = 0; r < m; ++r) a += u[r] * col[r];
      for (int64_t j = 0; j < n; ++j) b += v[j] * row[j];
      cross += a * b;
    }
    norm2 += nu2 * nv2 + 2.0 * cross;
    U.insert(U.end(), col.begin(), col.end());
    V.insert(V.end(), row.begin(), row.end());
    ++k;
    if (nu2 * nv2 <= eps * eps * norm2) {
      if (++small >= 2) break;
    } else {
      small = 0;
    }
    // next pivot row: largest entry of the new column among unused rows
    int64_t nxt = -1;
    double best = -1.0;
    for (int64_t r = 0; r < m; ++r)
      if (!used[r] && std::fabs(col[r]) > best) {
        best = std::fabs(col[r]);
        nxt = r;
      }
    if (nxt < 0) break;
    i = nxt;
  }
  return k;
}

int truncate_rank(const std::vector<double>& s, double eps) {
  if (s.empty() || s[0] == 0.0) return 0;
  int k = 0;
  for (double v : s)
    if (v > eps * s[0]) ++k;
  return k;
}

// C = A^T B with A (m x p), B (m x q), column-major.
void gemm_tn(int64_t m, int64_t p, int64_t q, const double* A, int64_t lda, const double* B,
             int64_t ldb, double* C) {
  for (int64_t j = 0; j < q; ++j)
    for (int64_t i = 0; i < p; ++i) {
      double s = 0;
      const double* a = A + i * lda;
      const double* b = B + j * ldb;
      for (int64_t r = 0; r < m; ++r) s += a[r] * b[r];
      C[i + j * p] = s;
    }
}

// C = A B with A (m x p), B (p x q).
void gemm_nn(int64_t m, int64_t p, int64_t q, const double* A, int64_t lda, const double* B,
             int64_t ldb, double* C, int64_t ldc) {
  for (int64_t j = 0; j < q; ++j) {
    double* c = C + j * ldc;
    for (int64_t r = 0; r < m; ++r) c[r] = 0.0;
    for (int64_t l = 0; l < p; ++l) {
      double b = B[l + j * ldb];
      if (b == 0.0) continue;
      const double* a = A + l * lda;
      for (int64_t r = 0; r < m; ++r) c[r] += a[r] * b;
    }
  }
}

template <class Fn>
void lowrank_block(const Fn& f, const int64_t* rows, int64_t m, const int64_t* cols, int64_t n,
                   double eps, LowRankBlock& out) {
  std::vector<double> U, V;
  int k = aca(f, rows, m, cols, n, eps * 0.1, U, V);
  out.k = 0;
  out.W.clear();
  out.X.clear();
  out.s.clear();
  if (k == 0) return;
  std::vector<double> Qu, Ru, Qv, Rv;
  qr_thin(m, k, U.data(), m, Qu, Ru);
  qr_thin(n, k, V.data(), n, Qv, Rv);
  int64_t ru = std::min<int64_t>(m, k), rv = std::min<int64_t>(n, k);
  // core = Ru (ru x k) * Rv^T (k x rv)
  std::vector<double> core(ru * rv, 0.0);
  for (int64_t j = 0; j < rv; ++j)
    for (int64_t l = 0; l < k; ++l) {
      double b = Rv[j + l * rv];
      if (b == 0.0) continue;
      for (int64_t i = 0; i < ru; ++i) core[i + j * ru] += Ru[i + l * ru] * b;
    }
  std::vector<double> Uc, sc, Vc;
  svd_jacobi(ru, rv, core.data(), ru, Uc, sc, Vc);
  int kk = truncate_rank(sc, eps);
  out.k = kk;
  out.s.assign(sc.begin(), sc.begin() + kk);
  out.W.assign(m * kk, 0.0);
  out.X.assign(n * kk, 0.0);
  gemm_nn(m, ru, kk, Qu.data(), m, Uc.data(), ru, out.W.data(), m);
  gemm_nn(n, rv, kk, Qv.data(), n, Vc.data(), rv, out.X.data(), n);
}

// Orthonormal basis of the columns of R (m x K) with singular values > thr.
void svd_basis(int64_t m, int64_t K, const std::vector<double>& R, double thr, std::vector<double>& B,
               std::vector<double>& sig) {
  B.clear();
  sig.clear();
  if (m == 0 || K == 0) return;
  std::vector<double> U, s, V;
  svd_jacobi(m, K, R.data(), m, U, s, V);
  int k = 0;
  for (double v : s)
    if (v > thr) ++k;
  B.assign(U.begin(), U.begin() + m * k);
  sig.assign(s.begin(), s.begin() + k);
}

}  // namespace

void lowrank_dense(const double* A, int64_t lda, int64_t m, int64_t n, double eps, LowRankBlock& out) {
  std::vector<int64_t> ri(m), ci(n);
  std::iota(ri.begin(), ri.end(), 0);
  std::iota(ci.begin(), ci.end(), 0);
  auto f = [A, lda](int64_t i, int64_t j) { return A[i + j * lda]; };
  lowrank_block(f, ri.data(), m, ci.data(), n, eps, out);
}

void build_lowrank_blocks(HostMatrix& hm, int nthreads) {
  KernelFn f;
  f.kind = hm.prm.kernel;
  f.param = hm.kparam;
  f.pts = hm.pts.data();
  const auto& ct = hm.ct;
  const int64_t nb = (int64_t)hm.blocks.size();
  hm.slot.assign(nb, -1);
  int nlr = 0, nd = 0;
  for (int64_t b = 0; b < nb; ++b) hm.slot[b] = hm.blocks[b].adm ? nlr++ : nd++;
  hm.lr.assign(nlr, LowRankBlock());
  hm.dn.assign(nd, DenseBlock());
  // largest blocks first for load balance
  std::vector<int64_t> order(nb);
  std::iota(order.begin(), order.end(), 0);
  auto area = [&](int64_t b) {
    return ct.cl[hm.blocks[b].row].size() * ct.cl[hm.blocks[b].col].size();
  };
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return area(a) > area(b); });
  const double eps = hm.prm.eps_build;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int64_t oi = 0; oi < nb; ++oi) {
    int64_t b = order[oi];
    const BlockLeaf& bl = hm.blocks[b];
    const Cluster& t = ct.cl[bl.row];
    const Cluster& s = ct.cl[bl.col];
    const int64_t* rows = ct.perm.data() + t.start;
    const int64_t* cols = ct.perm.data() + s.start;
    if (bl.adm) {
      lowrank_block(f, rows, t.size(), cols, s.size(), eps, hm.lr[hm.slot[b]]);
    } else {
      auto& D = hm.dn[hm.slot[b]].D;
      D.resize(t.size() * s.size());
      for (int64_t j = 0; j < s.size(); ++j)
        for (int64_t i = 0; i < t.size(); ++i) D[i + j * t.size()] = f(rows[i], cols[j]);
    }
  }
}

void build_uniform_bases(HostMatrix& hm, int nthreads) {
  const auto& ct = hm.ct;
  const int nc = (int)ct.cl.size();
  const double eps = hm.prm.eps_build;
  std::vector<std::vector<int>> rowl(nc), coll(nc);
  for (size_t b = 0; b < hm.blocks.size(); ++b)
    if (hm.blocks[b].adm && hm.lr[hm.slot[b]].k > 0) {
      rowl[hm.blocks[b].row].push_back((int)b);
      coll[hm.blocks[b].col].push_back((int)b);
    }
  for (Bases* bs : {&hm.rowb, &hm.colb}) {
    bs->B.assign(nc, {});
    bs->sig.assign(nc, {});
    bs->E.clear();
    bs->k.assign(nc, 0);
    bs->tau = eps;
  }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int c = 0; c < 2 * nc; ++c) {
    const bool rowside = c < nc;
    const int cid = rowside ? c : c - nc;
    const auto& lst = rowside ? rowl[cid] : coll[cid];
    const int64_t m = ct.cl[cid].size();
    int64_t K = 0;
    for (int b : lst) K += hm.lr[hm.slot[b]].k;
    std::vector<double> R(m * K);
    int64_t off = 0;
    for (int b : lst) {
      const auto& L = hm.lr[hm.slot[b]];
      double nrm = 0;
      for (double v : L.s) nrm += v * v;
      nrm = std::sqrt(nrm);
      const auto& F = rowside ? L.W : L.X;
      for (int j = 0; j < L.k; ++j)
        for (int64_t i = 0; i < m; ++i) R[i + (off + j) * m] = F[i + j * m] * (L.s[j] / nrm);
      off += L.k;
    }
    Bases& bs = rowside ? hm.rowb : hm.colb;
    svd_basis(m, K, R, eps, bs.B[cid], bs.sig[cid]);
    bs.k[cid] = (int)bs.sig[cid].size();
  }
  // couplings (and, for UH_SEP, their two factors)
  hm.coupling.assign(hm.lr.size(), {});
  const bool sep = hm.prm.format == HM_FMT_UH_SEP;
  hm.coupling_r.assign(sep ? hm.lr.size() : 0, {});
  hm.coupling_ct.assign(sep ? hm.lr.size() : 0, {});
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
  for (int64_t b = 0; b < (int64_t)hm.blocks.size(); ++b) {
    if (!hm.blocks[b].adm) continue;
    const auto& L = hm.lr[hm.slot[b]];
    const int t = hm.blocks[b].row, s = hm.blocks[b].col;
    const int64_t mt = ct.cl[t].size(), ms = ct.cl[s].size();
    const int kt = hm.rowb.k[t], ks = hm.colb.k[s];
    std::vector<double> P(kt * L.k), Q(ks * L.k);
    if (L.k) {
      gemm_tn(mt, kt, L.k, hm.rowb.B[t].data(), mt, L.W.data(), mt, P.data());
      gemm_tn(ms, ks, L.k, hm.colb.B[s].data(), ms, L.X.data(), ms, Q.data());
    }
    auto& S = hm.coupling[hm.slot[b]];
    S.assign(kt * ks, 0.0);
    for (int j = 0; j < ks; ++j)
      for (int l = 0; l < L.k; ++l) {
        double q = Q[j + l * ks] * L.s[l];
        for (int i = 0; i < kt; ++i) S[i + j * kt] += P[i + l * kt] * q;
      }
    if (sep) {   // Sr = (W_t^T W_b) diag(s_b), Sc^T = X_b^T X_s
      auto& R = hm.coupling_r[hm.slot[b]];
      auto& C = hm.coupling_ct[hm.slot[b]];
      R.assign((size_t)kt * L.k, 0.0);
      C.assign((size_t)L.k * ks, 0.0);
      for (int l = 0; l < L.k; ++l)
        for (int i = 0; i < kt; ++i) R[i + (size_t)l * kt] = P[i + (size_t)l * kt] * L.s[l];
      for (int j = 0; j < ks; ++j)
        for (int l = 0; l < L.k; ++l) C[l + (size_t)j * L.k] = Q[j + (size_t)l * ks];
    }
  }
}

namespace {

// Nested bases of one side.  side 0: rows (W_b), side 1: columns (X_b).
// Fills bs and P[b] = W_t^T W_b (k_t x k_b) at the block's own cluster t.
void nested_side(HostMatrix& hm, int side, int nthreads, Bases& bs, std::vector<std::vector<double>>& Pown) {
  const auto& ct = hm.ct;
  const int nc = (int)ct.cl.size();
  const double tau = hm.prm.eps_build / std::sqrt(ct.depth + 1.0);
  std::vector<std::vector<int>> own(nc);
  for (size_t b = 0; b < hm.blocks.size(); ++b)
    if (hm.blocks[b].adm && hm.lr[hm.slot[b]].k > 0)
      own[side == 0 ? hm.blocks[b].row : hm.blocks[b].col].push_back((int)b);
  // contributing blocks of c: own blocks of c and all ancestors
  std::vector<std::vector<int>> contrib(nc);
  for (int c = 0; c < nc; ++c)
    for (int a = c; a >= 0; a = ct.cl[a].parent)
      contrib[c].insert(contrib[c].end(), own[a].begin(), own[a].end());
  bs.B.assign(nc, {});
  bs.sig.assign(nc, {});
  bs.E.assign(nc, {});
  bs.k.assign(nc, 0);
  bs.tau = tau;
  Pown.assign(hm.blocks.size(), {});
  // P[c][i] = W_c^T F_b[c rows] for b = contrib[c][i] (k_c x k_b)
  std::vector<std::vector<std::vector<double>>> P(nc);
  auto factor = [&](int b) -> const std::vector<double>& {
    const auto& L = hm.lr[hm.slot[b]];
    return side == 0 ? L.W : L.X;
  };
  auto bcl = [&](int b) { return side == 0 ? hm.blocks[b].row : hm.blocks[b].col; };
  // Frobenius norm of F_b[c rows] diag(s_b)
  auto rownorm = [&](int c, int b) {
    const auto& L = hm.lr[hm.slot[b]];
    const auto& F = factor(b);
    const Cluster& a = ct.cl[bcl(b)];
    int64_t off = ct.cl[c].start - a.start, m = a.size();
    double s = 0;
    for (int j = 0; j < L.k; ++j) {
      double cs = 0;
      for (int64_t i = 0; i < ct.cl[c].size(); ++i) {
        double v = F[off + i + j * m];
        cs += v * v;
      }
      s += cs * L.s[j] * L.s[j];
    }
    return std::sqrt(s);
  };
  int maxlev = ct.depth;
  for (int lev = maxlev; lev >= 0; --lev) {
    std::vector<int> cs;
    for (int c = 0; c < nc; ++c)
      if (ct.cl[c].level == lev) cs.push_back(c);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (size_t ci = 0; ci < cs.size(); ++ci) {
      const int c = cs[ci];
      const Cluster& cc = ct.cl[c];
      const auto& lst = contrib[c];
      int64_t K = 0;
      for (int b : lst) K += hm.lr[hm.slot[b]].k;
      if (cc.leaf()) {
        const int64_t m = cc.size();
        std::vector<double> R(m * K, 0.0);
        int64_t off = 0;
        for (int b : lst) {
          const auto& L = hm.lr[hm.slot[b]];
          const auto& F = factor(b);
          const Cluster& a = ct.cl[bcl(b)];
          int64_t ro = cc.start - a.start, am = a.size();
          double nr = rownorm(c, b);
          for (int j = 0; j < L.k; ++j)
            for (int64_t i = 0; i < m; ++i)
              R[i + (off + j) * m] = nr > 0 ? F[ro + i + j * am] * L.s[j] / nr : 0.0;
          off += L.k;
        }
        svd_basis(m, K, R, tau, bs.B[c], bs.sig[c]);
        const int kc = (int)bs.sig[c].size();
        bs.k[c] = kc;
        P[c].resize(lst.size());
        for (size_t i = 0; i < lst.size(); ++i) {
          int b = lst[i];
          const auto& L = hm.lr[hm.slot[b]];
          const Cluster& a = ct.cl[bcl(b)];
          P[c][i].assign(kc * L.k, 0.0);
          if (kc && L.k)
            gemm_tn(m, kc, L.k, bs.B[c].data(), m, factor(b).data() + (cc.start - a.start), a.size(),
                    P[c][i].data());
        }
      } else {
        const int s0 = cc.son[0], s1 = cc.son[1];
        const int k0 = bs.k[s0], k1 = bs.k[s1];
        // sons' contrib lists start with the parent's contrib? No: a son's contrib is
        // own(son) followed by contrib(parent); locate the parent's entries by offset.
        const size_t o0 = own[s0].size(), o1 = own[s1].size();
        std::vector<double> R((k0 + k1) * K, 0.0);
        int64_t off = 0;
        for (size_t i = 0; i < lst.size(); ++i) {
          int b = lst[i];
          const auto& L = hm.lr[hm.slot[b]];
          double nr = rownorm(c, b);
          const auto& p0 = P[s0][o0 + i];
          const auto& p1 = P[s1][o1 + i];
          for (int j = 0; j < L.k; ++j) {
            double w = nr > 0 ? L.s[j] / nr : 0.0;
            for (int r = 0; r < k0; ++r) R[r + (off + j) * (k0 + k1)] = p0[r + j * k0] * w;
            for (int r = 0; r < k1; ++r) R[k0 + r + (off + j) * (k0 + k1)] = p1[r + j * k1] * w;
          }
          off += L.k;
        }
        std::vector<double> Q, sig;
        svd_basis(k0 + k1, K, R, tau, Q, sig);
        const int kc = (int)sig.size();
        bs.k[c] = kc;
        bs.sig[c] = sig;
        bs.E[s0].assign(k0 * kc, 0.0);
        bs.E[s1].assign(k1 * kc, 0.0);
        for (int j = 0; j < kc; ++j) {
          for (int r = 0; r < k0; ++r) bs.E[s0][r + j * k0] = Q[r + j * (k0 + k1)];
          for (int r = 0; r < k1; ++r) bs.E[s1][r + j * k1] = Q[k0 + r + j * (k0 + k1)];
        }
        // P[c][i] = E_s0^T P[s0][o0+i] + E_s1^T P[s1][o1+i]
        P[c].resize(lst.size());
        for (size_t i = 0; i < lst.size(); ++i) {
          const auto& L = hm.lr[hm.slot[lst[i]]];
          auto& pc = P[c][i];
          pc.assign(kc * L.k, 0.0);
          const auto& p0 = P[s0][o0 + i];
          const auto& p1 = P[s1][o1 + i];
          for (int j = 0; j < L.k; ++j)
            for (int r = 0; r < kc; ++r) {
              double v = 0;
              for (int q = 0; q < k0; ++q) v += bs.E[s0][q + r * k0] * p0[q + j * k0];
              for (int q = 0; q < k1; ++q) v += bs.E[s1][q + r * k1] * p1[q + j * k1];
              pc[r + j * kc] = v;
            }
        }
      }
    }
    // keep the own-block projections, free the sons' lists
    for (int c : cs) {
      for (size_t i = 0; i < own[c].size(); ++i) Pown[own[c][i]] = P[c][i];
      if (!ct.cl[c].leaf()) {
        P[ct.cl[c].son[0]].clear();
        P[ct.cl[c].son[0]].shrink_to_fit();
        P[ct.cl[c].son[1]].clear();
        P[ct.cl[c].son[1]].shrink_to_fit();
      }
    }
  }
  // inner clusters keep no explicit basis
  for (int c = 0; c < nc; ++c)
    if (!ct.cl[c].leaf()) bs.B[c].clear();
}

}  // namespace

void build_nested_bases(HostMatrix& hm, int nthreads) {
  std::vector<std::vector<double>> PW, PX;
  nested_side(hm, 0, nthreads, hm.rowb, PW);
  nested_side(hm, 1, nthreads, hm.colb, PX);
  hm.coupling.assign(hm.lr.size(), {});
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
  for (int64_t b = 0; b < (int64_t)hm.blocks.size(); ++b) {
    if (!hm.blocks[b].adm) continue;
    const auto& L = hm.lr[hm.slot[b]];
    const int t = hm.blocks[b].row, s = hm.blocks[b].col;
    const int kt = hm.rowb.k[t], ks = hm.colb.k[s];
    auto& S = hm.coupling[hm.slot[b]];
    S.assign(kt * ks, 0.0);
    if (L.k == 0) continue;
    const auto& P = PW[b];
    const auto& Q = PX[b];
    for (int j = 0; j < ks; ++j)
      for (int l = 0; l < L.k; ++l) {
        double q = Q[j + l * ks] * L.s[l];
        for (int i = 0; i < kt; ++i) S[i + j * kt] += P[i + l * kt] * q;
      }
  }
}

// The transpose of an H / UH / H2 matrix on the host: every block (t, s)
// becomes (s, t) with W and X swapped (low rank), D^T (dense), S^T (couplings),
// and the row and column bases (with their transfer matrices) trade places.
// Same cluster tree, same block numbering, same singular values: compressing it
// gives the codes of the original blocks, rearranged.
void transpose_host(const HostMatrix& H, HostMatrix& T) {
  T.prm = H.prm;
  T.n = H.n;
  T.kparam = H.kparam;
  T.pts = H.pts;
  T.ct = H.ct;
  T.blocks = H.blocks;
  for (BlockLeaf& b : T.blocks) std::swap(b.row, b.col);
  T.slot = H.slot;
  T.lr = H.lr;
  for (LowRankBlock& l : T.lr) std::swap(l.W, l.X);
  T.dn.assign(H.dn.size(), DenseBlock());
  T.coupling.assign(H.coupling.size(), std::vector<double>());
  for (size_t b = 0; b < H.blocks.size(); ++b) {
    const int64_t nt = H.ct.cl[H.blocks[b].row].size(), ns = H.ct.cl[H.blocks[b].col].size();
    const int sl = H.slot[b];
    if (!H.blocks[b].adm) {
      const std::vector<double>& D = H.dn[sl].D;   // nt x ns
      std::vector<double>& Dt = T.dn[sl].D;        // ns x nt
      Dt.resize(D.size());
      for (int64_t j = 0; j < ns; ++j)
        for (int64_t i = 0; i < nt; ++i) Dt[(size_t)j + (size_t)i * ns] = D[(size_t)i + (size_t)j * nt];
    } else if ((size_t)sl < H.coupling.size() && !H.coupling[sl].empty()) {
      const int kt = H.rowb.k[H.blocks[b].row], ks = H.colb.k[H.blocks[b].col];
      const std::vector<double>& S = H.coupling[sl];   // kt x ks
      std::vector<double>& St = T.coupling[sl];        // ks x kt
      St.resize(S.size());
      for (int j = 0; j < ks; ++j)
        for (int i = 0; i < kt; ++i) St[(size_t)j + (size_t)i * ks] = S[(size_t)i + (size_t)j * kt];
    }
  }
  // UH_SEP: S^T = Sc Sr^T, so Sr' = (Sc^T)^T and Sc'^T = Sr^T
  T.coupling_r.assign(H.coupling_ct.size(), std::vector<double>());
  T.coupling_ct.assign(H.coupling_r.size(), std::vector<double>());
  for (size_t b = 0; b < H.blocks.size(); ++b) {
    const int sl = H.slot[b];
    if (!H.blocks[b].adm || (size_t)sl >= H.coupling_r.size() || H.coupling_r[sl].empty()) continue;
    const int kt = H.rowb.k[H.blocks[b].row], ks = H.colb.k[H.blocks[b].col];
    const int kb = (int)(H.coupling_r[sl].size() / std::max(kt, 1));
    const std::vector<double>& R = H.coupling_r[sl];    // kt x kb
    const std::vector<double>& C = H.coupling_ct[sl];   // kb x ks
    std::vector<double>& Rt = T.coupling_r[sl];         // ks x kb = C^T
    std::vector<double>& Ct = T.coupling_ct[sl];        // kb x kt = R^T
    Rt.resize(C.size());
    Ct.resize(R.size());
    for (int l = 0; l < kb; ++l) {
      for (int j = 0; j < ks; ++j) Rt[(size_t)j + (size_t)l * ks] = C[(size_t)l + (size_t)j * kb];
      for (int i = 0; i < kt; ++i) Ct[(size_t)l + (size_t)i * kb] = R[(size_t)i + (size_t)l * kt];
    }
  }
  T.rowb = H.colb;
  T.colb = H.rowb;
}

}  // namespace hm
