// Small dense linear algebra for the host builder: Householder QR and
// one-sided Jacobi SVD (Golub & Van Loan, "Matrix Computations", Sec. 5.2 and
// 8.6.3 (Hestenes' method)).  Column-major storage.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "hm_internal.h"

namespace hm {

void qr_thin(int64_t m, int64_t n, const double* A, int64_t lda, std::vector<double>& Q,
             std::vector<double>& R) {
  const int64_t r = std::min(m, n);
  std::vector<double> a(m * n);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) a[i + j * m] = A[i + j * lda];
  std::vector<double> vs(m * r, 0.0), beta(r, 0.0);
  for (int64_t j = 0; j < r; ++j) {
    double* col = &a[j * m];
    double nrm2 = 0;
    for (int64_t i = j; i < m; ++i) nrm2 += col[i] * col[i];
    double nrm = std::sqrt(nrm2);
    double* v = &vs[j * m];
    if (nrm == 0.0) {
      beta[j] = 0.0;
      continue;
    }
    double alpha = col[j] >= 0 ? -nrm : nrm;
    for (int64_t i = j; i < m; ++i) v[i] = col[i];
    v[j] -= alpha;
    double vn2 = 0;
    for (int64_t i = j; i < m; ++i) vn2 += v[i] * v[i];
    beta[j] = vn2 > 0 ? 2.0 / vn2 : 0.0;
    // apply H = I - beta v v^T to columns j..n-1
    for (int64_t c = j; c < n; ++c) {
      double* ac = &a[c * m];
      double d = 0;
      for (int64_t i = j; i < m; ++i) d += v[i] * ac[i];
      d *= beta[j];
      for (int64_t i = j; i < m; ++i) ac[i] -= d * v[i];
    }
  }
  R.assign(r * n, 0.0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i <= std::min(j, r - 1); ++i) R[i + j * r] = a[i + j * m];
  Q.assign(m * r, 0.0);
  for (int64_t j = 0; j < r; ++j) Q[j + j * m] = 1.0;
  for (int64_t j = r - 1; j >= 0; --j) {
    if (beta[j] == 0.0) continue;
    const double* v = &vs[j * m];
    for (int64_t c = 0; c < r; ++c) {
      double* qc = &Q[c * m];
      double d = 0;
      for (int64_t i = j; i < m; ++i) d += v[i] * qc[i];
      d *= beta[j];
      for (int64_t i = j; i < m; ++i) qc[i] -= d * v[i];
    }
  }
}

namespace {

// One-sided Jacobi on the columns of G (m x n, m >= n): G V = U diag(s).
void jacobi_cols(int64_t m, int64_t n, std::vector<double>& G, std::vector<double>& V) {
  V.assign(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i) V[i + i * n] = 1.0;
  const double tol = 1e-15;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int64_t p = 0; p < n - 1; ++p) {
      for (int64_t q = p + 1; q < n; ++q) {
        double* gp = &G[p * m];
        double* gq = &G[q * m];
        double alpha = 0, beta = 0, gamma = 0;
        for (int64_t i = 0; i < m; ++i) {
          alpha += gp[i] * gp[i];
          beta += gq[i] * gq[i];
          gamma += gp[i] * gq[i];
        }
        if (gamma == 0.0 || std::fabs(gamma) <= tol * std::sqrt(alpha * beta)) continue;
        rotated = true;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double c = 1.0 / std::sqrt(1.0 + t * t);
        double s = c * t;
        for (int64_t i = 0; i < m; ++i) {
          double x = gp[i], y = gq[i];
          gp[i] = c * x - s * y;
          gq[i] = s * x + c * y;
        }
        double* vp = &V[p * n];
        double* vq = &V[q * n];
        for (int64_t i = 0; i < n; ++i) {
          double x = vp[i], y = vq[i];
          vp[i] = c * x - s * y;
          vq[i] = s * x + c * y;
        }
      }
    }
    if (!rotated) break;
  }
}

}  // namespace

void svd_jacobi(int64_t m, int64_t n, const double* A, int64_t lda, std::vector<double>& U,
                std::vector<double>& s, std::vector<double>& V) {
  const bool tr = m < n;
  const int64_t mm = tr ? n : m, nn = tr ? m : n;   // work on the tall orientation
  std::vector<double> G(mm * nn);
  for (int64_t j = 0; j < nn; ++j)
    for (int64_t i = 0; i < mm; ++i) G[i + j * mm] = tr ? A[j + i * lda] : A[i + j * lda];
  // precondition with QR when tall: G = Q R, Jacobi on R (nn x nn)
  std::vector<double> Q, R, Vw;
  bool useqr = mm > 2 * nn;
  std::vector<double> W;
  int64_t wm = mm;
  if (useqr) {
    qr_thin(mm, nn, G.data(), mm, Q, R);
    W = R;
    wm = nn;
  } else {
    W = G;
  }
  jacobi_cols(wm, nn, W, Vw);
  std::vector<double> sv(nn);
  for (int64_t j = 0; j < nn; ++j) {
    double a = 0;
    for (int64_t i = 0; i < wm; ++i) a += W[i + j * wm] * W[i + j * wm];
    sv[j] = std::sqrt(a);
  }
  std::vector<int64_t> ord(nn);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return sv[a] > sv[b]; });
  // left vectors of the worked matrix: W(:,j)/s_j, then multiply by Q if used
  std::vector<double> Lw(wm * nn, 0.0);
  for (int64_t jj = 0; jj < nn; ++jj) {
    int64_t j = ord[jj];
    double sj = sv[j];
    for (int64_t i = 0; i < wm; ++i) Lw[i + jj * wm] = sj > 0 ? W[i + j * wm] / sj : 0.0;
  }
  // complete zero columns with orthonormal directions is not needed: they carry s = 0
  std::vector<double> L(mm * nn, 0.0);
  if (useqr) {
    for (int64_t jj = 0; jj < nn; ++jj)
      for (int64_t l = 0; l < nn; ++l) {
        double w = Lw[l + jj * nn];
        if (w == 0.0) continue;
        for (int64_t i = 0; i < mm; ++i) L[i + jj * mm] += Q[i + l * mm] * w;
      }
  } else {
    L = Lw;
  }
  std::vector<double> Rv(nn * nn);
  for (int64_t jj = 0; jj < nn; ++jj)
    for (int64_t i = 0; i < nn; ++i) Rv[i + jj * nn] = Vw[i + ord[jj] * nn];
  s.resize(nn);
  for (int64_t jj = 0; jj < nn; ++jj) s[jj] = sv[ord[jj]];
  if (!tr) {
    U = L;          // m x r
    V = Rv;         // n x r
  } else {
    U = Rv;         // A^T = L S Rv^T  =>  A = Rv S L^T
    V = L;
  }
}

}  // namespace hm
