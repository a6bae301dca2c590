// Packed layout of compressed H / UH / H^2 matrices and the launch program of
// one product (Sec. 3 algorithms mapped onto the GPU kernels).
//
// Layout (one payload buffer, every column 8-byte aligned):
//  * column dots (phase A: X factors of H blocks, UH column bases, H^2 leaf
//    column bases, transfer matrices for the up-sweep) are stored
//    segment-major: for each run of <= 128 rows, the rows of every column of
//    the set.  An item is one such segment (all columns of the set).
//  * row chunks (phase C; couplings; down-sweep): each output chunk (a leaf
//    cluster, or <= 128 coefficients) reads
//      - uniform tiles: the chunk's rows of every column of one directly
//        compressed matrix (dense leaf, coupling, transfer), contiguous;
//      - merged columns: the chunk's rows of every VALR-compressed column
//        that reaches it (W factors of all low-rank blocks of its ancestors'
//        block rows, or row bases), stored contiguously per chunk and sorted
//        by format, with one (format word, multiplier index) per column.
// A leaf chunk owns its rows of y and gathers the contributions of all its
// ancestors' block rows itself: the race freedom of Alg. 3 without a
// root-to-leaf traversal.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <functional>
#include <numeric>

#include "program.h"

namespace hm {

namespace {

constexpr int SEG_ROWS = 128;    // rows of a column-dot segment (16 lanes x 8 rows)
constexpr int CHUNK_ROWS = 128;  // rows of a coefficient chunk

struct Enc {
  CodeHdr h;
  std::vector<uint64_t> codes;
  uint32_t fw() const { return fmt_word(h.B, h.fmt, h.e, h.m); }
  double scale() const { return h.fmt == FMT_AFLP ? h.vmin : 1.0; }
};

bool kernel_decodable(const CodeHdr& h, const double* v, int64_t n) {
  if (h.fmt == FMT_AFLP && h.e > 7) return false;
  if (h.fmt == FMT_FPX11 || h.fmt == FMT_RAW)
    for (int64_t i = 0; i < n; ++i)
      if (std::fabs(v[i]) >= 0x1p127) return false;
  return true;
}

bool encode(const double* v, int64_t n, int codec, int key, Enc& out) {
  out.codes.resize(std::max<int64_t>(n, 1));
  if (!encode_values(v, n, 1, codec, key, out.h, out.codes.data())) return false;
  return kernel_decodable(out.h, v, n);
}

struct Ctx {
  const HostMatrix& H;
  Program& P;
  int codec;
  double eps;
  int valr;
  int key_eps;
};

// ---------------------------------------------------------------- VALR keys
std::vector<int> keys_lowrank(const Ctx& cx, const std::vector<double>& s) {
  std::vector<int> k(s.size(), cx.key_eps);
  if (cx.codec == HM_CODEC_NONE || !cx.valr || s.empty()) return k;
  double nrm = 0;
  for (double v : s) nrm += v * v;
  const double delta = cx.eps * std::sqrt(nrm) / (1.0 + 2.0 * (double)s.size());
  for (size_t i = 0; i < s.size(); ++i) k[i] = valr_key(s[i], delta);
  return k;
}

std::vector<int> keys_basis(const Ctx& cx, const std::vector<double>& sig, double tau) {
  std::vector<int> k(sig.size(), cx.key_eps);
  if (cx.codec == HM_CODEC_NONE || !cx.valr || sig.empty()) return k;
  const double delta = tau / (double)sig.size();
  for (size_t i = 0; i < sig.size(); ++i) k[i] = valr_key(sig[i], delta);
  return k;
}

// A column set: one Enc per column (VALR) or one for the whole matrix (direct).
struct ColSet {
  std::vector<Enc> enc;
  bool direct = false;
  int64_t m = 0;
  int n = 0;
  int B(int j) const { return direct ? enc[0].h.B : enc[j].h.B; }
  uint32_t fw(int j) const { return direct ? enc[0].fw() : enc[j].fw(); }
  const uint64_t* col(int j) const { return direct ? enc[0].codes.data() + (int64_t)j * m : enc[j].codes.data(); }
  double scale(int j) const { return direct ? enc[0].scale() : enc[j].scale(); }
};

bool make_cols(const Ctx& cx, const double* A, int64_t m, int n, const std::vector<int>& keys, ColSet& cs) {
  cs.direct = false;
  cs.m = m;
  cs.n = n;
  cs.enc.assign(n, Enc());
  for (int j = 0; j < n; ++j)
    if (!encode(A + (int64_t)j * m, m, cx.codec, keys[j], cs.enc[j])) return false;
  return true;
}

bool make_direct(const Ctx& cx, const double* A, int64_t m, int n, ColSet& cs) {
  cs.direct = true;
  cs.m = m;
  cs.n = n;
  cs.enc.assign(1, Enc());
  return encode(A, m * n, cx.codec, cx.key_eps, cs.enc[0]);
}

// format kind and byte width: columns with equal keys can share an item
uint32_t kind_width(uint32_t fw) { return fw & 0xffffu; }

// ---------------------------------------------------------------- column-dot items
// Segment-major layout of a column set (one item per segment of <= 128 rows);
// input vector index of row 0 is vin.  A set that fits one segment writes its
// coefficients v[out0 + j] = scale[j] * (alpha if use_alpha) * sum directly
// (final = true, segp untouched); otherwise segp[j] receives the partial
// index of column j in every segment.
void pack_cdot(Program& P, const ColSet& cs, int32_t vin, int64_t& pbase, std::vector<std::vector<int32_t>>& segp,
               bool allow_final, int64_t out0, const std::vector<double>* scale, bool use_alpha, bool& final_out) {
  segp.assign(cs.n, {});
  const int32_t fbase = (int32_t)P.pk.fmts.size();
  for (int j = 0; j < cs.n; ++j) {
    P.pk.fmts.push_back(cs.fw(j));
    P.pk.cscale.push_back(split_ff(scale ? (*scale)[j] : 1.0));
  }
  final_out = allow_final && cs.m <= SEG_ROWS;
  for (int64_t r0 = 0; r0 < cs.m; r0 += SEG_ROWS) {
    const int64_t r1 = std::min<int64_t>(cs.m, r0 + SEG_ROWS);
    uint64_t off0 = 0;
    for (int j = 0; j < cs.n; ++j) {
      const uint64_t o = P.pk.put(cs.col(j) + r0, r1 - r0, cs.B(j));
      if (j == 0) off0 = o;
    }
    Item it{};
    it.off = off0;
    it.fmt = fbase;
    it.ncols = cs.n;
    it.nrows = (int32_t)(r1 - r0);
    it.vin = (int32_t)(vin + r0);
    if (final_out) {
      it.out = (int32_t)out0;
      it.flags = ITEM_FINAL | (use_alpha ? ITEM_ALPHA : 0);
    } else {
      it.out = (int32_t)pbase;
      for (int j = 0; j < cs.n; ++j) segp[j].push_back((int32_t)(pbase + j));
      pbase += cs.n;
    }
    P.items.push_back(it);
  }
}

// ---------------------------------------------------------------- row-chunk pieces
// Uniform tile: rows [r0, r1) of every column of a direct column set.
Tile pack_tile(Program& P, const ColSet& cs, int64_t r0, int64_t r1, int32_t vin, int32_t flags) {
  Tile T{};
  for (int j = 0; j < cs.n; ++j) {
    const uint64_t o = P.pk.put(cs.col(j) + r0, r1 - r0, cs.B(j));
    if (j == 0) T.off = o;
  }
  T.ncols = cs.n;
  T.fw = cs.fw(0);
  T.vin = vin;
  T.flags = flags;
  T.scale = split_ff(cs.scale(0));
  return T;
}

// One column of a VALR set restricted to rows [r0, r1), with its multiplier.
struct ColRef {
  const ColSet* cs;
  int j;
  int64_t r0;
  int32_t vin;
};

struct ChunkWork {
  Chunk c{};
  std::vector<Tile> t;
  std::vector<ColRef> cols;
};

void add_launch(Program& P, Launch::Kind k, int64_t off, int64_t n, int mode = 0, bool rs = false) {
  Launch L;
  L.kind = k;
  L.off = off;
  L.n = n;
  L.mode = mode;
  L.use_rowscale = rs;
  P.launches.push_back(L);
}

// Pack the merged columns of every chunk (sorted by format, contiguous), append
// the chunks (largest first) and one RGEMV launch.
void add_rgemv(Ctx& cx, std::vector<ChunkWork>& cw, int mode, bool rowscale) {
  Program& P = cx.P;
  std::vector<int64_t> w(cw.size());
  for (size_t i = 0; i < cw.size(); ++i) {
    ChunkWork& c = cw[i];
    const int64_t R = c.c.nrows;
    int64_t b = 64;
    for (const Tile& t : c.t) b += R * (int64_t)(t.fw & 0xff) * t.ncols;
    for (const ColRef& r : c.cols) b += R * r.cs->B(r.j) + 16;
    w[i] = b;
  }
  std::vector<int64_t> order(cw.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return w[a] > w[b]; });
  const int64_t first = (int64_t)P.chunks.size();
  for (int64_t i : order) {
    ChunkWork& c = cw[i];
    const int64_t R = c.c.nrows;
    c.c.t0 = (int32_t)P.tiles.size();
    P.tiles.insert(P.tiles.end(), c.t.begin(), c.t.end());
    c.c.t1 = (int32_t)P.tiles.size();
    std::stable_sort(c.cols.begin(), c.cols.end(), [](const ColRef& a, const ColRef& b) {
      return kind_width(a.cs->fw(a.j)) < kind_width(b.cs->fw(b.j));
    });
    c.c.c0 = (int32_t)P.cols.size();
    c.c.coff = P.pk.align8();
    for (const ColRef& r : c.cols) {
      P.pk.put(r.cs->col(r.j) + r.r0, R, r.cs->B(r.j));
      P.cols.push_back(ColMeta{r.cs->fw(r.j), r.vin});
    }
    c.c.c1 = (int32_t)P.cols.size();
    P.chunks.push_back(c.c);
  }
  Launch L;
  L.kind = Launch::RGEMV;
  L.mode = mode;
  L.off = first;
  L.n = (int64_t)cw.size();
  L.use_rowscale = rowscale;
  P.launches.push_back(L);
}

std::vector<std::vector<int>> leaves_under(const ClusterTree& ct) {
  std::vector<int> leaves;
  for (size_t c = 0; c < ct.cl.size(); ++c)
    if (ct.cl[c].leaf()) leaves.push_back((int)c);
  std::sort(leaves.begin(), leaves.end(), [&](int a, int b) { return ct.cl[a].start < ct.cl[b].start; });
  std::vector<std::vector<int>> out(ct.cl.size());
  for (size_t c = 0; c < ct.cl.size(); ++c) {
    const Cluster& cc = ct.cl[c];
    auto lo = std::lower_bound(leaves.begin(), leaves.end(), cc.start,
                               [&](int a, int64_t s) { return ct.cl[a].start < s; });
    for (auto it = lo; it != leaves.end() && ct.cl[*it].start < cc.end; ++it) out[c].push_back(*it);
  }
  return out;
}

std::vector<int> ancestors_root_first(const ClusterTree& ct, int c) {
  std::vector<int> anc;
  for (int a = c; a >= 0; a = ct.cl[a].parent) anc.push_back(a);
  std::reverse(anc.begin(), anc.end());
  return anc;
}

// Dense blocks: direct compression, one uniform tile per leaf of the row cluster.
// dt[b][i] = tile for the i-th leaf under the block's row cluster.
bool pack_dense(Ctx& cx, const std::vector<std::vector<int>>& lv, std::vector<std::vector<Tile>>& dt) {
  const HostMatrix& H = cx.H;
  const auto& ct = H.ct;
  const int64_t nb = (int64_t)H.blocks.size();
  std::vector<ColSet> cs(nb);
  std::atomic<bool> ok{true};
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nb; ++b) {
    if (H.blocks[b].adm) continue;
    const auto& D = H.dn[H.slot[b]].D;
    if (!make_direct(cx, D.data(), ct.cl[H.blocks[b].row].size(), (int)ct.cl[H.blocks[b].col].size(), cs[b]))
      ok = false;
  }
  if (!ok) return false;
  dt.assign(nb, {});
  for (int64_t b = 0; b < nb; ++b) {
    if (H.blocks[b].adm) continue;
    const Cluster& t = ct.cl[H.blocks[b].row];
    const Cluster& s = ct.cl[H.blocks[b].col];
    for (int l : lv[H.blocks[b].row])
      dt[b].push_back(pack_tile(cx.P, cs[b], ct.cl[l].start - t.start, ct.cl[l].end - t.start, (int32_t)s.start, 1));
    cx.P.fp64_dense += (int64_t)H.dn[H.slot[b]].D.size() * 8;
    cs[b] = ColSet();
  }
  return true;
}

size_t leaf_index(const ClusterTree& ct, const std::vector<int>& leaves, int c) {
  auto it = std::lower_bound(leaves.begin(), leaves.end(), ct.cl[c].start,
                             [&](int a, int64_t s) { return ct.cl[a].start < s; });
  return (size_t)(it - leaves.begin());
}

// Leaf chunks producing y: merged VALR columns from `rowcols(c, out)` and the
// dense tiles of c's ancestors' block rows (root first, as Alg. 3).
void leaf_chunks(Ctx& cx, const std::vector<std::vector<int>>& lv, const std::vector<std::vector<Tile>>& dt,
                 const std::function<void(int, std::vector<ColRef>&)>& rowcols) {
  const HostMatrix& H = cx.H;
  const auto& ct = H.ct;
  std::vector<std::vector<int>> rowdense(ct.cl.size());
  for (size_t b = 0; b < H.blocks.size(); ++b)
    if (!H.blocks[b].adm) rowdense[H.blocks[b].row].push_back((int)b);
  std::vector<ChunkWork> cw;
  for (int c : lv[0]) {
    ChunkWork w;
    w.c.row0 = (int32_t)ct.cl[c].start;
    w.c.nrows = (int32_t)ct.cl[c].size();
    rowcols(c, w.cols);
    for (int a : ancestors_root_first(ct, c))
      for (int b : rowdense[a]) w.t.push_back(dt[b][leaf_index(ct, lv[a], c)]);
    cw.push_back(std::move(w));
  }
  add_rgemv(cx, cw, MODE_Y, false);
}

void gsum_outputs(Program& P, int64_t out0, const std::vector<std::vector<int32_t>>& segp,
                  const std::vector<double>& scale, int flags) {
  for (size_t j = 0; j < segp.size(); ++j) {
    GsumOut o{};
    o.out = (int32_t)(out0 + (int64_t)j);
    o.p0 = (int32_t)P.plist.size();
    for (int32_t p : segp[j]) {
      P.plist.push_back(p);
      P.pscale.push_back(split_ff(1.0));
    }
    o.p1 = (int32_t)P.plist.size();
    o.flags = flags;
    o.scale = split_ff(scale[j]);
    P.gouts.push_back(o);
  }
}

// ---------------------------------------------------------------- H (Alg. 1 / 3)
bool program_h(Ctx& cx) {
  const HostMatrix& H = cx.H;
  Program& P = cx.P;
  const auto& ct = H.ct;
  const int64_t N = H.n;
  const auto lv = leaves_under(ct);
  std::vector<std::vector<Tile>> dt;
  if (!pack_dense(cx, lv, dt)) return false;
  const int64_t nb = (int64_t)H.blocks.size();
  std::vector<ColSet> csx(nb), csw(nb);
  std::atomic<bool> ok{true};
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t b = 0; b < nb; ++b) {
    if (!H.blocks[b].adm) continue;
    const auto& L = H.lr[H.slot[b]];
    if (L.k == 0) continue;
    const auto keys = keys_lowrank(cx, L.s);
    if (!make_cols(cx, L.X.data(), ct.cl[H.blocks[b].col].size(), L.k, keys, csx[b])) ok = false;
    if (!make_cols(cx, L.W.data(), ct.cl[H.blocks[b].row].size(), L.k, keys, csw[b])) ok = false;
  }
  if (!ok) return false;
  add_launch(P, Launch::GATHER, 0, N);
  std::vector<int64_t> toff(nb, -1);
  int64_t vec = N, pbase = 0;
  const int64_t i0 = (int64_t)P.items.size(), g0 = (int64_t)P.gouts.size();
  for (int64_t b = 0; b < nb; ++b) {
    if (!H.blocks[b].adm) continue;
    const auto& L = H.lr[H.slot[b]];
    if (L.k == 0) continue;
    const Cluster& t = ct.cl[H.blocks[b].row];
    const Cluster& s = ct.cl[H.blocks[b].col];
    P.fp64_lowrank += (t.size() + s.size()) * L.k * 8;
    std::vector<std::vector<int32_t>> segp;
    std::vector<double> sc(L.k);
    for (int j = 0; j < L.k; ++j) sc[j] = L.s[j] * csx[b].scale(j) * csw[b].scale(j);
    bool fin = false;
    pack_cdot(P, csx[b], (int32_t)s.start, pbase, segp, true, vec, &sc, true, fin);
    if (!fin) gsum_outputs(P, vec, segp, sc, 1);
    toff[b] = vec;
    vec += L.k;
    csx[b] = ColSet();
  }
  P.npartial = std::max(P.npartial, pbase);
  add_launch(P, Launch::CDOT, i0, (int64_t)P.items.size() - i0);
  add_launch(P, Launch::GSUM, g0, (int64_t)P.gouts.size() - g0);
  std::vector<std::vector<int>> rowlr(ct.cl.size());
  for (int64_t b = 0; b < nb; ++b)
    if (toff[b] >= 0) rowlr[H.blocks[b].row].push_back((int)b);
  leaf_chunks(cx, lv, dt, [&](int c, std::vector<ColRef>& out) {
    for (int a : ancestors_root_first(ct, c))
      for (int b : rowlr[a]) {
        const int64_t r0 = ct.cl[c].start - ct.cl[a].start;
        for (int j = 0; j < csw[b].n; ++j) out.push_back(ColRef{&csw[b], j, r0, (int32_t)(toff[b] + j)});
      }
  });
  P.nvec = vec;
  return true;
}

// coupling chunks of every row cluster with k > 0: t_tau = sum_b S_b s_sigma(b)
bool coupling_chunks(Ctx& cx, const std::vector<int64_t>& soff, const std::vector<int64_t>& toff,
                     std::vector<ChunkWork>& cw, int flags) {
  const HostMatrix& H = cx.H;
  const auto& ct = H.ct;
  const int nc = (int)ct.cl.size();
  std::vector<std::vector<int>> rowlr(nc);
  for (size_t b = 0; b < H.blocks.size(); ++b)
    if (H.blocks[b].adm) rowlr[H.blocks[b].row].push_back((int)b);
  std::vector<ColSet> enc(H.blocks.size());
  std::atomic<bool> ok{true};
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t b = 0; b < (int64_t)H.blocks.size(); ++b) {
    if (!H.blocks[b].adm) continue;
    const int kt = H.rowb.k[H.blocks[b].row], ks = H.colb.k[H.blocks[b].col];
    if (kt == 0 || ks == 0) continue;
    if (!make_direct(cx, H.coupling[H.slot[b]].data(), kt, ks, enc[b])) ok = false;
  }
  if (!ok) return false;
  for (int t = 0; t < nc; ++t) {
    const int kt = H.rowb.k[t];
    if (kt == 0) continue;
    const int nsplit = (kt + CHUNK_ROWS - 1) / CHUNK_ROWS;
    std::vector<ChunkWork> per(nsplit);
    for (int b : rowlr[t]) {
      const int s = H.blocks[b].col;
      if (H.colb.k[s] == 0) continue;
      for (int i = 0; i < nsplit; ++i) {
        const int64_t r0 = (int64_t)i * CHUNK_ROWS, r1 = std::min<int64_t>(kt, r0 + CHUNK_ROWS);
        per[i].t.push_back(pack_tile(cx.P, enc[b], r0, r1, (int32_t)soff[s], 0));
      }
      cx.P.fp64_lowrank += (int64_t)enc[b].m * enc[b].n * 8;
      enc[b] = ColSet();
    }
    for (int i = 0; i < nsplit; ++i) {
      per[i].c.row0 = (int32_t)(toff[t] + (int64_t)i * CHUNK_ROWS);
      per[i].c.nrows = std::min(CHUNK_ROWS, kt - i * CHUNK_ROWS);
      per[i].c.flags = flags;
      cw.push_back(std::move(per[i]));
    }
  }
  return true;
}

// column-basis forward (Alg. 4 / leaves of Alg. 6): s = vmin * X^T x
bool forward_bases(Ctx& cx, const std::vector<int>& which, const std::vector<int64_t>& soff, int64_t& pbase) {
  const HostMatrix& H = cx.H;
  const auto& ct = H.ct;
  std::vector<ColSet> enc(ct.cl.size());
  std::atomic<bool> ok{true};
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < (int64_t)which.size(); ++i) {
    const int c = which[i];
    const auto keys = keys_basis(cx, H.colb.sig[c], H.colb.tau);
    if (!make_cols(cx, H.colb.B[c].data(), ct.cl[c].size(), H.colb.k[c], keys, enc[c])) ok = false;
  }
  if (!ok) return false;
  for (int c : which) {
    const int k = H.colb.k[c];
    cx.P.fp64_lowrank += ct.cl[c].size() * k * 8;
    std::vector<std::vector<int32_t>> segp;
    std::vector<double> sc(k);
    for (int j = 0; j < k; ++j) sc[j] = enc[c].scale(j);
    bool fin = false;
    pack_cdot(cx.P, enc[c], (int32_t)ct.cl[c].start, pbase, segp, true, soff[c], &sc, false, fin);
    if (!fin) gsum_outputs(cx.P, soff[c], segp, sc, 0);
    enc[c] = ColSet();
  }
  return true;
}

// row bases (VALR); rowscale of the t' entries = vmin of each column
bool row_bases(Ctx& cx, const std::vector<int>& which, const std::vector<int64_t>& toff, std::vector<ColSet>& enc) {
  const HostMatrix& H = cx.H;
  const auto& ct = H.ct;
  enc.assign(ct.cl.size(), ColSet());
  std::atomic<bool> ok{true};
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < (int64_t)which.size(); ++i) {
    const int c = which[i];
    const auto keys = keys_basis(cx, H.rowb.sig[c], H.rowb.tau);
    if (!make_cols(cx, H.rowb.B[c].data(), ct.cl[c].size(), H.rowb.k[c], keys, enc[c])) ok = false;
  }
  if (!ok) return false;
  for (int c : which) {
    cx.P.fp64_lowrank += ct.cl[c].size() * H.rowb.k[c] * 8;
    for (int j = 0; j < H.rowb.k[c]; ++j) cx.P.rowscale[toff[c] + j] = enc[c].scale(j);
  }
  return true;
}

// ---------------------------------------------------------------- UH (Alg. 4 + 5)
bool program_uh(Ctx& cx) {
  const HostMatrix& H = cx.H;
  Program& P = cx.P;
  const auto& ct = H.ct;
  const int64_t N = H.n;
  const int nc = (int)ct.cl.size();
  const auto lv = leaves_under(ct);
  std::vector<std::vector<Tile>> dt;
  if (!pack_dense(cx, lv, dt)) return false;
  std::vector<int64_t> soff(nc, -1), toff(nc, -1);
  int64_t vec = N;
  std::vector<int> xs, ws;
  for (int c = 0; c < nc; ++c)
    if (H.colb.k[c]) {
      soff[c] = vec;
      vec += H.colb.k[c];
      xs.push_back(c);
    }
  for (int c = 0; c < nc; ++c)
    if (H.rowb.k[c]) {
      toff[c] = vec;
      vec += H.rowb.k[c];
      ws.push_back(c);
    }
  P.rowscale.assign(vec, 1.0);
  add_launch(P, Launch::GATHER, 0, N);
  int64_t pbase = 0;
  const int64_t i0 = (int64_t)P.items.size(), g0 = (int64_t)P.gouts.size();
  if (!forward_bases(cx, xs, soff, pbase)) return false;
  P.npartial = std::max(P.npartial, pbase);
  add_launch(P, Launch::CDOT, i0, (int64_t)P.items.size() - i0);
  add_launch(P, Launch::GSUM, g0, (int64_t)P.gouts.size() - g0);
  std::vector<ColSet> wb;
  if (!row_bases(cx, ws, toff, wb)) return false;
  std::vector<ChunkWork> cw;
  if (!coupling_chunks(cx, soff, toff, cw, 1)) return false;
  add_rgemv(cx, cw, MODE_VEC, true);
  leaf_chunks(cx, lv, dt, [&](int c, std::vector<ColRef>& out) {
    for (int a : ancestors_root_first(ct, c)) {
      if (H.rowb.k[a] == 0) continue;
      const int64_t r0 = ct.cl[c].start - ct.cl[a].start;
      for (int j = 0; j < wb[a].n; ++j) out.push_back(ColRef{&wb[a], j, r0, (int32_t)(toff[a] + j)});
    }
  });
  P.nvec = vec;
  return true;
}

// ---------------------------------------------------------------- H^2 (Alg. 6 + 7)
bool program_h2(Ctx& cx) {
  const HostMatrix& H = cx.H;
  Program& P = cx.P;
  const auto& ct = H.ct;
  const int64_t N = H.n;
  const int nc = (int)ct.cl.size();
  for (int c = 0; c < nc; ++c)
    if (H.rowb.k[c] > CHUNK_ROWS) return false;      // a down-sweep chunk holds <= 128 coefficients
  const auto lv = leaves_under(ct);
  std::vector<std::vector<Tile>> dt;
  if (!pack_dense(cx, lv, dt)) return false;
  std::vector<int64_t> soff(nc, -1), toff(nc, -1);
  int64_t vec = N;
  for (int c = 0; c < nc; ++c)
    if (H.colb.k[c]) {
      soff[c] = vec;
      vec += H.colb.k[c];
    }
  for (int c = 0; c < nc; ++c)
    if (H.rowb.k[c]) {
      toff[c] = vec;
      vec += H.rowb.k[c];
    }
  P.rowscale.assign(vec, 1.0);
  add_launch(P, Launch::GATHER, 0, N);
  std::vector<int> xl, wl;
  for (int c = 0; c < nc; ++c) {
    if (!ct.cl[c].leaf()) continue;
    if (H.colb.k[c]) xl.push_back(c);
    if (H.rowb.k[c]) wl.push_back(c);
  }
  int64_t pbase = 0;
  int64_t i0 = (int64_t)P.items.size(), g0 = (int64_t)P.gouts.size();
  if (!forward_bases(cx, xl, soff, pbase)) return false;
  P.npartial = std::max(P.npartial, pbase);
  add_launch(P, Launch::CDOT, i0, (int64_t)P.items.size() - i0);
  add_launch(P, Launch::GSUM, g0, (int64_t)P.gouts.size() - g0);
  // transfer matrices, direct compression
  std::vector<ColSet> ex(nc), ew(nc);
  for (int c = 0; c < nc; ++c) {
    const int p = ct.cl[c].parent;
    if (p < 0) continue;
    if (H.colb.k[c] && H.colb.k[p]) {
      if (!make_direct(cx, H.colb.E[c].data(), H.colb.k[c], H.colb.k[p], ex[c])) return false;
      P.fp64_lowrank += (int64_t)H.colb.E[c].size() * 8;
    }
    if (H.rowb.k[c] && H.rowb.k[p]) {
      if (!make_direct(cx, H.rowb.E[c].data(), H.rowb.k[c], H.rowb.k[p], ew[c])) return false;
      P.fp64_lowrank += (int64_t)H.rowb.E[c].size() * 8;
    }
  }
  // up-sweep by height: s_sigma = sum_i vmin_i * E_i^T s_i (Alg. 6)
  std::vector<int> height(nc, 0);
  int maxh = 0;
  for (int c = nc - 1; c >= 0; --c) {
    if (!ct.cl[c].leaf()) height[c] = 1 + std::max(height[ct.cl[c].son[0]], height[ct.cl[c].son[1]]);
    maxh = std::max(maxh, height[c]);
  }
  for (int h = 1; h <= maxh; ++h) {
    i0 = (int64_t)P.items.size();
    g0 = (int64_t)P.gouts.size();
    int64_t pb = 0;
    for (int c = 0; c < nc; ++c) {
      if (height[c] != h || H.colb.k[c] == 0) continue;
      const int kp = H.colb.k[c];
      std::vector<std::vector<int32_t>> all(kp);
      std::vector<std::vector<double>> scl(kp);
      for (int i = 0; i < 2; ++i) {
        const int sc = ct.cl[c].son[i];
        if (H.colb.k[sc] == 0) continue;
        std::vector<std::vector<int32_t>> segp;
        bool fin = false;
        pack_cdot(P, ex[sc], (int32_t)soff[sc], pb, segp, false, 0, nullptr, false, fin);
        for (int j = 0; j < kp; ++j)
          for (int32_t q : segp[j]) {
            all[j].push_back(q);
            scl[j].push_back(ex[sc].scale(0));
          }
      }
      for (int j = 0; j < kp; ++j) {
        GsumOut o{};
        o.out = (int32_t)(soff[c] + j);
        o.p0 = (int32_t)P.plist.size();
        for (size_t q = 0; q < all[j].size(); ++q) {
          P.plist.push_back(all[j][q]);
          P.pscale.push_back(split_ff(scl[j][q]));
        }
        o.p1 = (int32_t)P.plist.size();
        o.scale = split_ff(1.0);
        P.gouts.push_back(o);
      }
    }
    P.npartial = std::max(P.npartial, pb);
    add_launch(P, Launch::CDOT, i0, (int64_t)P.items.size() - i0);
    add_launch(P, Launch::GSUM, g0, (int64_t)P.gouts.size() - g0);
  }
  std::vector<ColSet> wb;
  if (!row_bases(cx, wl, toff, wb)) return false;
  // coupling (unscaled t)
  std::vector<ChunkWork> cw;
  if (!coupling_chunks(cx, soff, toff, cw, 0)) return false;
  add_rgemv(cx, cw, MODE_VEC, false);
  // down-sweep by level: t_c += vmin * E_c t_parent; leaves scaled by alpha * vminW (Alg. 7)
  for (int lev = 1; lev <= ct.depth; ++lev) {
    std::vector<ChunkWork> dw;
    for (int c = 0; c < nc; ++c) {
      if (ct.cl[c].level != lev || H.rowb.k[c] == 0) continue;
      const int p = ct.cl[c].parent;
      ChunkWork w;
      w.c.row0 = (int32_t)toff[c];
      w.c.nrows = H.rowb.k[c];
      w.c.flags = ct.cl[c].leaf() ? 1 : 0;
      if (H.rowb.k[p] > 0) w.t.push_back(pack_tile(P, ew[c], 0, H.rowb.k[c], (int32_t)toff[p], 0));
      dw.push_back(std::move(w));
    }
    if (!dw.empty()) add_rgemv(cx, dw, MODE_VEC_ADD, true);
  }
  // backward at the leaves plus dense blocks
  leaf_chunks(cx, lv, dt, [&](int c, std::vector<ColRef>& out) {
    for (int j = 0; j < wb[c].n; ++j) out.push_back(ColRef{&wb[c], j, 0, (int32_t)(toff[c] + j)});
  });
  P.nvec = vec;
  return true;
}

// Algorithmic bytes of every launch: packed values (no padding), format
// words, descriptors, vector reads and writes.
void launch_bytes(Program& P) {
  for (Launch& L : P.launches) {
    int64_t b = 0;
    switch (L.kind) {
      case Launch::GATHER:
        b = L.n * (4 + 8 + 8);
        break;
      case Launch::CDOT:
        for (int64_t i = L.off; i < L.off + L.n; ++i) {
          const Item& t = P.items[i];
          for (int j = 0; j < t.ncols; ++j) b += (int64_t)t.nrows * (P.pk.fmts[t.fmt + j] & 0xff);
          b += 4 * (int64_t)t.ncols + (int64_t)sizeof(Item) + 8 * (int64_t)t.nrows + 8 * (int64_t)t.ncols;
        }
        break;
      case Launch::GSUM:
        for (int64_t i = L.off; i < L.off + L.n; ++i) {
          const GsumOut& o = P.gouts[i];
          b += (int64_t)(o.p1 - o.p0) * (4 + 8 + 8) + (int64_t)sizeof(GsumOut) + 8;
        }
        break;
      case Launch::RGEMV:
        for (int64_t i = L.off; i < L.off + L.n; ++i) {
          const Chunk& c = P.chunks[i];
          b += (int64_t)sizeof(Chunk);
          for (int32_t k = c.t0; k < c.t1; ++k) {
            const Tile& t = P.tiles[k];
            b += (int64_t)sizeof(Tile) + (int64_t)c.nrows * (t.fw & 0xff) * t.ncols + 8 * (int64_t)t.ncols;
          }
          for (int32_t k = c.c0; k < c.c1; ++k)
            b += (int64_t)sizeof(ColMeta) + (int64_t)c.nrows * (P.cols[k].fw & 0xff) + 8;
          if (L.mode == MODE_Y)
            b += (int64_t)c.nrows * (4 + 8 + 8);
          else
            b += (int64_t)c.nrows * ((L.mode == MODE_VEC_ADD ? 16 : 8) + (L.use_rowscale ? 8 : 0));
        }
        break;
    }
    L.bytes = b;
  }
}

}  // namespace

bool build_program(const HostMatrix& H, int codec, double eps, int valr, int nsm, Program& P) {
  (void)nsm;
  P = Program();
  P.tier = (codec == HM_CODEC_NONE || eps <= 0x1p-22) ? TIER_FF : TIER_F32;
  Ctx cx{H, P, codec, eps, valr ? 1 : 0, m_eps(eps)};
  bool ok;
  switch (H.prm.format) {
    case HM_FMT_H: ok = program_h(cx); break;
    case HM_FMT_UH: ok = program_uh(cx); break;
    default: ok = program_h2(cx); break;
  }
  if (!ok) {
    P = Program();
    return false;
  }
  P.pk.align8();
  P.pk.pay.resize(P.pk.pay.size() + 128, 0);   // tail reads of the last column stay in bounds
  if (P.rowscale.empty()) P.rowscale.assign(1, 1.0);
  launch_bytes(P);
  return true;
}

}  // namespace hm
