// Cluster tree (Def. Cluster Tree) and block tree (Def. Block Tree), Sec. 2.2.
//
// Geometric bisection: a cluster with more than `leaf` points is cut at the
// midpoint 0.5*(lo+hi) of the longest edge of its tight bounding box (lowest
// axis on ties); points below the midpoint form the first son.  A degenerate
// cut (one side empty) splits the cluster into its first floor(n/2) and
// remaining points.  Standard admissibility in squared form:
//   adm(t,s) <=> dist^2 > 0 and min(diam_t^2, diam_s^2) <= eta^2 * dist^2.
// Built with -ffp-contract=off so the sums are evaluated as written.
#include <algorithm>
#include <functional>

#include "hm_internal.h"

namespace hm {

namespace {

void bbox(const double* pts, const int64_t* idx, int64_t n, double lo[3], double hi[3]) {
  for (int d = 0; d < 3; ++d) {
    lo[d] = pts[3 * idx[0] + d];
    hi[d] = lo[d];
  }
  for (int64_t i = 1; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      double v = pts[3 * idx[i] + d];
      if (v < lo[d]) lo[d] = v;
      if (v > hi[d]) hi[d] = v;
    }
}

double diam2(const Cluster& c) {
  double d0 = c.hi[0] - c.lo[0], d1 = c.hi[1] - c.lo[1], d2 = c.hi[2] - c.lo[2];
  return (d0 * d0 + d1 * d1) + d2 * d2;
}

double dist2(const Cluster& a, const Cluster& b) {
  double g[3];
  for (int d = 0; d < 3; ++d) {
    double u = b.lo[d] - a.hi[d];
    double w = a.lo[d] - b.hi[d];
    double m = u > w ? u : w;
    g[d] = m > 0.0 ? m : 0.0;
  }
  return (g[0] * g[0] + g[1] * g[1]) + g[2] * g[2];
}

}  // namespace

void build_cluster_tree(const double* pts, int64_t n, int leaf, ClusterTree& ct) {
  ct.cl.clear();
  ct.perm.resize(n);
  std::vector<int64_t> idx(n), tmp(n);
  for (int64_t i = 0; i < n; ++i) idx[i] = i;
  ct.depth = 0;
  // idx[start..end) holds the cluster's points in the current order
  std::function<int(int64_t, int64_t, int, int)> rec = [&](int64_t start, int64_t end, int level,
                                                           int parent) -> int {
    int id = (int)ct.cl.size();
    ct.cl.emplace_back();
    Cluster c;
    c.start = start;
    c.end = end;
    c.level = level;
    c.parent = parent;
    int64_t cnt = end - start;
    bbox(pts, idx.data() + start, cnt, c.lo, c.hi);
    if (level > ct.depth) ct.depth = level;
    if (cnt <= leaf) {
      ct.cl[id] = c;
      return id;
    }
    int axis = 0;
    double ext = c.hi[0] - c.lo[0];
    for (int d = 1; d < 3; ++d) {
      double e = c.hi[d] - c.lo[d];
      if (e > ext) {
        ext = e;
        axis = d;
      }
    }
    double mid = 0.5 * (c.lo[axis] + c.hi[axis]);
    int64_t nl = 0, nr = 0;
    for (int64_t i = start; i < end; ++i)
      if (pts[3 * idx[i] + axis] < mid) ++nl;
    nr = cnt - nl;
    if (nl > 0 && nr > 0) {
      int64_t a = start, b = start + nl;
      for (int64_t i = start; i < end; ++i) {
        int64_t p = idx[i];
        if (pts[3 * p + axis] < mid)
          tmp[a++] = p;
        else
          tmp[b++] = p;
      }
      std::copy(tmp.begin() + start, tmp.begin() + end, idx.begin() + start);
    } else {
      nl = cnt / 2;
    }
    ct.cl[id] = c;
    int s0 = rec(start, start + nl, level + 1, id);
    int s1 = rec(start + nl, end, level + 1, id);
    ct.cl[id].son[0] = s0;
    ct.cl[id].son[1] = s1;
    ct.cl[id].nsons = 2;
    return id;
  };
  rec(0, n, 0, -1);
  ct.perm = idx;
}

void build_block_tree(const ClusterTree& ct, double eta, std::vector<BlockLeaf>& out, int mode) {
  out.clear();
  const double eta2 = eta * eta;
  std::function<void(int, int)> rec = [&](int t, int s) {
    const Cluster& a = ct.cl[t];
    const Cluster& b = ct.cl[s];
    double d2 = dist2(a, b);
    double da = diam2(a), db = diam2(b);
    const bool std_adm = d2 > 0.0 && (da < db ? da : db) <= eta2 * d2;
    // admissibility modes (the remark after Def. H-Matrix): standard, off-diagonal
    // (HODLR: inadmissible only on the diagonal), single level (BLR: only blocks
    // of leaf clusters are tested)
    bool adm = std_adm;
    if (mode == HM_ADM_HODLR) adm = t != s;
    if (mode == HM_ADM_BLR) adm = (a.leaf() || b.leaf()) && std_adm;
    if (adm) {
      out.push_back({t, s, true});
    } else if (a.leaf() || b.leaf()) {
      out.push_back({t, s, false});
    } else {
      for (int i = 0; i < a.nsons; ++i)
        for (int j = 0; j < b.nsons; ++j) rec(a.son[i], b.son[j]);
    }
  };
  rec(0, 0);
}

}  // namespace hm
