// Host check of the H-LU solve program (build_lu_program): test code, built by
// tests/test_lu_program.py against the library's host objects; no GPU code.
//
// It factors the Matern (or Laplace) matrix of the given points with the
// library's own host routine (lu_factor_host), packs both factors, and then
//  * checks every packed column against the payload (8-byte aligned, its
//    8-code groups inside the payload with the slack the kernel relies on),
//    every multiplier and coefficient index, and every dependency flag;
//  * replays the work list in list order, as one warp after another would run
//    it, in FP64 with its own decoder of the packed codes, requiring that
//    every dependency is met when its item starts (the GPU's warps take items
//    in list order and wait only for earlier ones: no stall is possible iff
//    this holds);
//  * compares the replayed solution with a dense LU solve of the exact matrix
//    (partial pivoting) and prints the relative difference and the relative
//    residual ||A x - b|| / (||A|| ||x||).
// usage: lu_check <points file> n kernel eps codec leaf
// prints "diff <d>", "residual <r>" and "ok" or "FAILED <count>".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "program.h"

using namespace hm;

namespace {

int g_fails = 0;
#define CHECK(cond, ...)                         \
  do {                                           \
    if (!(cond)) {                               \
      if (g_fails < 20) {                        \
        std::printf("FAIL line %d: ", __LINE__); \
        std::printf(__VA_ARGS__);                \
        std::printf("\n");                       \
      }                                          \
      ++g_fails;                                 \
    }                                            \
  } while (0)

// Value of one code: fb = fmt << 4 | B, em = e | m << 8 (AFLP as +-(s - 1)).
double decode(uint64_t code, uint16_t fb, uint16_t em) {
  const int B = fb & 15, fmt = fb >> 4, e = em & 0xff, m = em >> 8;
  if (fmt == 0) {
    const uint32_t w = (uint32_t)(code << (32 - 8 * B));
    float f;
    std::memcpy(&f, &w, 4);
    return f;
  }
  if (fmt == 1 || fmt == 3) {
    const uint64_t w = code << (64 - 8 * B);
    double d;
    std::memcpy(&d, &w, 8);
    return d;
  }
  const uint64_t sign = (code >> (8 * B - 1)) & 1, f = (code >> m) & ((1ull << e) - 1),
                 mant = code & ((1ull << m) - 1);
  if (f == 0) return sign ? -0.0 : 0.0;
  const uint64_t sb = ((f + 1023) << 52) | (mant << (52 - m));
  double s;
  std::memcpy(&s, &sb, 8);
  return sign ? -(s - 1.0) : s - 1.0;
}

double value(const LuProgram& P, const LuCol& c, int r) {
  const int B = c.fb & 15;
  uint64_t code = 0;
  for (int b = 0; b < B; ++b) code |= (uint64_t)P.pk.pay[c.off + (uint64_t)r * B + b] << (8 * b);
  return decode(code, c.fb, c.em);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 7) {
    std::fprintf(stderr, "usage: %s file n kernel eps codec leaf\n", argv[0]);
    return 2;
  }
  const int64_t n = std::atoll(argv[2]);
  const int kernel = std::atoi(argv[3]), codec = std::atoi(argv[5]), leaf = std::atoi(argv[6]);
  const double eps = std::atof(argv[4]);
  std::vector<double> pts(3 * n), b(n);
  FILE* f = std::fopen(argv[1], "rb");
  if (!f || std::fread(pts.data(), 8, 3 * n, f) != (size_t)(3 * n) || std::fread(b.data(), 8, n, f) != (size_t)n) {
    std::fprintf(stderr, "cannot read %s\n", argv[1]);
    return 2;
  }
  std::fclose(f);
  hm_build_params prm{};
  prm.kernel = kernel;
  prm.leaf_size = leaf;
  prm.eta = 2.0;
  prm.eps_build = eps;
  prm.nthreads = 8;
  HostMatrix L, U;
  if (!lu_factor_host(prm, pts.data(), n, L, U)) {
    std::printf("factorisation failed\n");
    return 1;
  }
  LuProgram P;
  if (!build_lu_program(L, U, codec, eps, 1, P)) {
    std::printf("build_lu_program failed\n");
    return 1;
  }
  const uint64_t psz = P.pk.pay.size();
  for (size_t i = 0; i < P.cols.size(); ++i) {
    const LuCol& c = P.cols[i];
    const int B = c.fb & 15;
    CHECK(c.off % 8 == 0, "column %zu not 8-byte aligned", i);
    CHECK(c.off + (uint64_t)((c.rows + 7) / 8) * 8 * B <= psz, "column %zu: groups past the payload", i);
    CHECK(c.rows >= 1 && c.rows <= (1 << 30), "column %zu rows", i);
    CHECK(B >= 1 && B <= 8 && (c.fb >> 4) <= 3, "column %zu class", i);
  }
  std::vector<int> flags(P.nflags, 0);
  std::vector<double> coef(P.ncoef, 0.0), w(n, 0.0), x(n, 0.0), bz(n);
  const auto& perm = L.ct.perm;
  for (int64_t i = 0; i < n; ++i) bz[i] = b[perm[i]];
  for (size_t ii = 0; ii < P.items.size(); ++ii) {
    const LuItem& it = P.items[ii];
    for (int d = it.d0; d < it.d1; ++d) {
      CHECK(P.deps[d].flag >= 0 && P.deps[d].flag < P.nflags, "item %zu: dependency flag out of range", ii);
      if (P.deps[d].flag >= 0 && P.deps[d].flag < P.nflags)
        CHECK(flags[P.deps[d].flag] >= P.deps[d].target, "item %zu: dependency %d not met in list order", ii, d);
    }
    CHECK(it.flag >= 0 && it.flag < P.nflags, "item %zu: flag out of range", ii);
    CHECK(it.r0 >= 0 && it.nr >= 1 && it.r0 + it.nr <= n, "item %zu: rows out of range", ii);
    if (it.kind == LU_ROW_L || it.kind == LU_ROW_U) {
      const bool fwd = it.kind == LU_ROW_L;
      const int R = it.nr;
      CHECK(R <= CHUNK_ROWS, "item %zu: %d rows", ii, R);
      std::vector<double> r(R);
      for (int k = 0; k < R; ++k) r[k] = (fwd ? bz : w)[it.r0 + k];
      for (int j = it.c0; j < it.c1; ++j) {
        const LuCol& c = P.cols[j];
        CHECK(c.rows == R, "item %zu: column rows %d != %d", ii, c.rows, R);
        const bool cf = (c.flags & LC_COEF) != 0;
        CHECK(c.mult >= 0 && c.mult < (cf ? P.ncoef : n), "item %zu: multiplier index", ii);
        const double m = (cf ? coef[c.mult] : (fwd ? w : x)[c.mult]) * c.scale;
        for (int k = 0; k < R; ++k) r[k] -= value(P, c, k) * m;
      }
      if (fwd) {
        for (int j = 0; j < R; ++j) {
          const LuCol& c = P.cols[it.tri + j];
          for (int i = j + 1; i < R; ++i) r[i] -= value(P, c, i) * c.scale * r[j];
        }
      } else {
        for (int j = R - 1; j >= 0; --j) {
          const LuCol& c = P.cols[it.tri + j];
          r[j] /= value(P, c, j) * c.scale;
          for (int i = 0; i < j; ++i) r[i] -= value(P, c, i) * c.scale * r[j];
        }
      }
      for (int k = 0; k < R; ++k) (fwd ? w : x)[it.r0 + k] = r[k];
      flags[it.flag] += 1;
    } else {
      const std::vector<double>& vin = it.kind == LU_COL_L ? w : x;
      for (int j = it.c0; j < it.c1; ++j) {
        const LuCol& c = P.cols[j];
        CHECK(c.rows == it.nr, "item %zu: column rows", ii);
        CHECK(c.mult >= 0 && c.mult < P.ncoef, "item %zu: coefficient index", ii);
        double s = 0;
        for (int k = 0; k < it.nr; ++k) s += value(P, c, k) * vin[it.r0 + k];
        coef[c.mult] = s * c.scale;
      }
      flags[it.flag] += it.c1 - it.c0;
    }
  }
  for (int64_t l = 0; l < 2 * P.nleaves; ++l) CHECK(flags[l] == 1, "leaf flag %ld = %d", (long)l, flags[l]);
  std::vector<double> xo(n);
  for (int64_t i = 0; i < n; ++i) xo[perm[i]] = x[i];
  // dense reference: A x* = b by Gaussian elimination with partial pivoting
  KernelFn kf;
  kf.kind = kernel;
  kf.param = L.kparam;
  kf.pts = pts.data();
  std::vector<double> A(n * n), a2;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) A[i + j * n] = kf(i, j);
  a2 = A;
  std::vector<double> xs = b;
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = k;
    for (int64_t i = k + 1; i < n; ++i)
      if (std::fabs(a2[i + k * n]) > std::fabs(a2[p + k * n])) p = i;
    if (p != k) {
      for (int64_t j = 0; j < n; ++j) std::swap(a2[k + j * n], a2[p + j * n]);
      std::swap(xs[k], xs[p]);
    }
    for (int64_t i = k + 1; i < n; ++i) {
      const double l = a2[i + k * n] / a2[k + k * n];
      a2[i + k * n] = l;
      for (int64_t j = k + 1; j < n; ++j) a2[i + j * n] -= l * a2[k + j * n];
      xs[i] -= l * xs[k];
    }
  }
  for (int64_t k = n - 1; k >= 0; --k) {
    double s = xs[k];
    for (int64_t j = k + 1; j < n; ++j) s -= a2[k + j * n] * xs[j];
    xs[k] = s / a2[k + k * n];
  }
  double dn = 0, xn = 0, rn = 0, an = 0;
  for (int64_t i = 0; i < n; ++i) {
    dn += (xo[i] - xs[i]) * (xo[i] - xs[i]);
    xn += xs[i] * xs[i];
    double ri = -b[i];
    for (int64_t j = 0; j < n; ++j) ri += A[i + j * n] * xo[j];
    rn += ri * ri;
  }
  for (double v : A) an += v * v;
  double xon = 0;
  for (double v : xo) xon += v * v;
  std::printf("items %zu columns %zu payload %lu\n", P.items.size(), P.cols.size(), (unsigned long)psz);
  std::printf("diff %.6e\n", std::sqrt(dn / xn));
  std::printf("residual %.6e\n", std::sqrt(rn) / (std::sqrt(an) * std::sqrt(xon)));
  if (g_fails) {
    std::printf("FAILED %d\n", g_fails);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
