// libhm: C ABI (include/hm.h), device layout of compressed H / UH / H^2
// matrices, and the launch program of one product.
//
// Layout in HBM (one payload buffer, every column 4-byte aligned):
//  * phase A (column dots): X factors of low-rank blocks (H), column bases
//    (UH), leaf column bases (H^2) and transfer matrices, column-major, one
//    format word per column (VALR) or per matrix (direct compression);
//  * phase C (row chunks): the row-side data of every block -- dense leaves,
//    W factors, row bases -- split into tiles by leaf cluster ("tile-major"):
//    for each leaf c under the block's row cluster, the rows c of every column.
//    A leaf chunk then reads contiguous tiles only and owns its rows of y
//    (race-free in the sense of Alg. 3: clusters of one level are disjoint,
//    and a leaf gathers the contributions of all its ancestors itself).
//  * couplings (UH / H^2) and transfer matrices are tiles of <= 128 rows.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <functional>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>

#include <cuda_runtime.h>

#include "dev_types.h"
#include "hm_internal.h"

namespace hm {
cudaError_t launch_gather(const double* x, const int32_t* perm, int n, float2* xo, cudaStream_t st);
cudaError_t launch_cdot(int tier, const CdotItem* items, int nitems, const uint8_t* pay,
                        const uint32_t* fmts, const float2* vin, double* partial, int* err, int grid,
                        cudaStream_t st);
cudaError_t launch_gsum(const GsumOut* outs, int nouts, const int32_t* plist, const double* pscale,
                        const double* partial, double alpha, float2* vout, cudaStream_t st);
cudaError_t launch_rgemv(int tier, int mode, const Chunk* chunks, int nchunks, const Tile* tiles,
                         const uint8_t* pay, const uint32_t* fmts, const float2* vin, double alpha,
                         double beta, double* y, const int32_t* perm, float2* vout,
                         const double* rowscale, int* err, int grid, cudaStream_t st);
cudaError_t launch_decode(const uint8_t* p, int64_t n, int B, int fmt, int e, int m, double vmin,
                          double* out, cudaStream_t st);
}  // namespace hm

using namespace hm;

namespace {

// ---------------------------------------------------------------- host-side packing
struct Packer {
  std::vector<uint8_t> pay;
  std::vector<uint32_t> fmts;
  int64_t value_bytes = 0;
  bool unsupported = false;

  uint64_t align4() {
    while (pay.size() & 3) pay.push_back(0);
    return pay.size();
  }
  // append n codes of B bytes (little-endian), column padded to 4 bytes
  uint64_t put(const uint64_t* codes, int64_t n, int64_t inc, int B) {
    uint64_t off = align4();
    pay.resize(off + (uint64_t)(n * B));
    uint8_t* dst = pay.data() + off;
    for (int64_t i = 0; i < n; ++i) {
      uint64_t c = codes[i * inc];
      for (int b = 0; b < B; ++b) dst[i * B + b] = (uint8_t)(c >> (8 * b));
    }
    value_bytes += n * B;
    align4();
    return off;
  }
};

// Encoded array (one header) with its codes.
struct Enc {
  CodeHdr h;
  std::vector<uint64_t> codes;
  uint32_t fw() const { return fmt_word(h.B, h.fmt, h.e, h.m); }
  double scale() const { return h.fmt == FMT_AFLP ? h.vmin : 1.0; }
};

bool kernel_decodable(const CodeHdr& h, const double* v, int64_t n, int64_t inc) {
  if (h.fmt == FMT_AFLP && h.e > 7) return false;
  if (h.fmt == FMT_FPX11 || h.fmt == FMT_RAW) {
    for (int64_t i = 0; i < n; ++i)
      if (std::fabs(v[i * inc]) >= 0x1p127) return false;
  }
  return true;
}

bool encode(const double* v, int64_t n, int64_t inc, int codec, int key, Enc& out) {
  out.codes.resize(std::max<int64_t>(n, 1));
  if (!encode_values(v, n, inc, codec, key, out.h, out.codes.data())) return false;
  return kernel_decodable(out.h, v, n, inc);
}

int64_t pad4(int64_t x) { return (x + 3) & ~int64_t(3); }

// ---------------------------------------------------------------- device program
struct Launch {
  enum Kind { GATHER, CDOT, GSUM, RGEMV } kind;
  int mode = 0;
  int64_t off = 0, n = 0;        // range in the item / out / chunk array
  bool use_pscale = false;
  bool use_rowscale = false;
  int64_t bytes = 0;             // algorithmic bytes of the launch
};

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

struct Program {
  int tier = TIER_F32;
  std::vector<Launch> launches;
  std::vector<CdotItem> items;
  std::vector<GsumOut> gouts;
  std::vector<int32_t> plist;
  std::vector<double> pscale;
  std::vector<Tile> tiles;
  std::vector<Chunk> chunks;
  std::vector<double> rowscale;
  int64_t nvec = 0;          // float2 vector workspace (x first)
  int64_t npartial = 0;      // max partials of one cdot launch
  Packer pk;
  int64_t fp64_lowrank = 0, fp64_dense = 0;
};

}  // namespace

struct hm_matrix {
  HostMatrix H;
  bool compressed = false;
  int codec = 0, valr = 0;
  double eps = 0;
  Program prog;
  // device
  DevArr<uint8_t> d_pay;
  DevArr<uint32_t> d_fmt;
  DevArr<CdotItem> d_items;
  DevArr<GsumOut> d_gout;
  DevArr<int32_t> d_plist;
  DevArr<double> d_pscale;
  DevArr<Tile> d_tiles;
  DevArr<Chunk> d_chunks;
  DevArr<double> d_rowscale;
  DevArr<int32_t> d_perm;
  float2* d_vec = nullptr;
  double* d_part = nullptr;
  int* d_err = nullptr;
  double* d_hx = nullptr;      // host-path staging (hm_matvec_host)
  double* d_hy = nullptr;
  int64_t d_h_cap = 0;
  int grid_cdot = 0, grid_rg = 0;
  std::mutex mu;
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
    d_pay.release();
    d_fmt.release();
    d_items.release();
    d_gout.release();
    d_plist.release();
    d_pscale.release();
    d_tiles.release();
    d_chunks.release();
    d_rowscale.release();
    d_perm.release();
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

namespace {

// leaves (pre-order ids) under each cluster, in position order
std::vector<std::vector<int>> leaves_under(const ClusterTree& ct) {
  std::vector<int> leaves;
  for (size_t c = 0; c < ct.cl.size(); ++c)
    if (ct.cl[c].leaf()) leaves.push_back((int)c);
  std::sort(leaves.begin(), leaves.end(),
            [&](int a, int b) { return ct.cl[a].start < ct.cl[b].start; });
  std::vector<std::vector<int>> out(ct.cl.size());
  for (size_t c = 0; c < ct.cl.size(); ++c) {
    const Cluster& cc = ct.cl[c];
    auto lo = std::lower_bound(leaves.begin(), leaves.end(), cc.start,
                               [&](int a, int64_t s) { return ct.cl[a].start < s; });
    for (auto it = lo; it != leaves.end() && ct.cl[*it].start < cc.end; ++it) out[c].push_back(*it);
  }
  return out;
}

// Pack a column-major m x n matrix whose column j is encoded by enc[j] (VALR,
// one Enc per column) or by enc[0] (direct), tile-major over row splits.
// Returns the payload offset of each split's tile.
std::vector<uint64_t> pack_tiled(Packer& pk, const std::vector<Enc>& enc, bool direct, int64_t m,
                                 int64_t n, const std::vector<std::pair<int64_t, int64_t>>& splits) {
  std::vector<uint64_t> offs;
  for (auto [r0, r1] : splits) {
    uint64_t first = 0;
    for (int64_t j = 0; j < n; ++j) {
      const Enc& e = direct ? enc[0] : enc[j];
      const uint64_t* codes = direct ? e.codes.data() + j * m : e.codes.data();
      uint64_t o = pk.put(codes + r0, r1 - r0, 1, e.h.B);
      if (j == 0) first = o;
    }
    if (n == 0) first = pk.align4();
    offs.push_back(first);
  }
  return offs;
}

// Pack columns (column-major, full length), return the offset of column 0.
uint64_t pack_cols(Packer& pk, const std::vector<Enc>& enc, bool direct, int64_t m, int64_t n) {
  uint64_t first = pk.align4();
  for (int64_t j = 0; j < n; ++j) {
    const Enc& e = direct ? enc[0] : enc[j];
    const uint64_t* codes = direct ? e.codes.data() + j * m : e.codes.data();
    uint64_t o = pk.put(codes, m, 1, e.h.B);
    if (j == 0) first = o;
  }
  return first;
}

int32_t push_fmts(Packer& pk, const std::vector<Enc>& enc) {
  int32_t idx = (int32_t)pk.fmts.size();
  for (const auto& e : enc) pk.fmts.push_back(e.fw());
  return idx;
}

struct Ctx {
  hm_matrix* M;
  int codec;
  double eps;
  int valr;
  int key_eps;
  bool ok = true;
};

// Encode one column at key (codec NONE: raw)
bool enc_col(Ctx& cx, const double* v, int64_t n, int key, Enc& e) {
  return encode(v, n, 1, cx.codec, key, e);
}

// cdot items over the columns of a packed matrix, segments of <= 512 rows
void add_cdot_items(Program& P, uint64_t off, int32_t fmt, int ncols, int64_t nrows, int32_t vin,
                    int64_t& pbase, std::vector<std::vector<int32_t>>* seg_partials) {
  for (int64_t r0 = 0; r0 < nrows; r0 += 512) {
    CdotItem it{};
    it.off = off;
    it.fmt = fmt;
    it.ncols = ncols;
    it.nrows = (int32_t)nrows;
    it.row0 = (int32_t)r0;
    it.seg = (int32_t)std::min<int64_t>(512, nrows - r0);
    it.vin = vin;
    it.pout = (int32_t)pbase;
    P.items.push_back(it);
    if (seg_partials)
      for (int j = 0; j < ncols; ++j) (*seg_partials)[j].push_back((int32_t)(pbase + j));
    pbase += ncols;
  }
}

void add_launch(Program& P, Launch::Kind k, int64_t off, int64_t n, int mode = 0, bool ps = false,
                bool rs = false) {
  Launch L;
  L.kind = k;
  L.off = off;
  L.n = n;
  L.mode = mode;
  L.use_pscale = ps;
  L.use_rowscale = rs;
  P.launches.push_back(L);
}

// split rows [0, m) into chunks of <= 128
std::vector<std::pair<int64_t, int64_t>> row_splits(int64_t m) {
  std::vector<std::pair<int64_t, int64_t>> s;
  for (int64_t r = 0; r < m; r += 128) s.push_back({r, std::min<int64_t>(m, r + 128)});
  if (m == 0) s.push_back({0, 0});
  return s;
}

// -------------------------------------------------------------- dense tiles shared by all formats
struct DenseTiles {
  // per dense block: tile offset per leaf under the row cluster, and the encoding
  std::vector<std::vector<uint64_t>> off;
  std::vector<int32_t> fidx;     // direct format index (~ index into the format words)
  std::vector<double> scale;
};

int32_t direct_fmt(Packer& pk, uint32_t fw);

// position of leaf c in the position-ordered leaf list of a cluster
size_t leaf_index(const ClusterTree& ct, const std::vector<int>& leaves, int c) {
  auto it = std::lower_bound(leaves.begin(), leaves.end(), ct.cl[c].start,
                             [&](int a, int64_t s) { return ct.cl[a].start < s; });
  return (size_t)(it - leaves.begin());
}

bool pack_dense(Ctx& cx, Program& P, const std::vector<std::vector<int>>& lv, DenseTiles& dt) {
  HostMatrix& H = cx.M->H;
  const auto& ct = H.ct;
  dt.off.assign(H.blocks.size(), {});
  dt.fidx.assign(H.blocks.size(), 0);
  dt.scale.assign(H.blocks.size(), 1.0);
  const int64_t nb = (int64_t)H.blocks.size();
  std::vector<std::vector<Enc>> encs(nb);
  std::atomic<bool> ok{true};
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nb; ++b) {
    if (H.blocks[b].adm) continue;
    const auto& D = H.dn[H.slot[b]].D;
    encs[b].resize(1);
    if (!encode(D.data(), (int64_t)D.size(), 1, cx.codec, cx.key_eps, encs[b][0])) ok = false;
  }
  if (!ok) return false;
  for (size_t b = 0; b < H.blocks.size(); ++b) {
    if (H.blocks[b].adm) continue;
    const Cluster& t = ct.cl[H.blocks[b].row];
    const Cluster& s = ct.cl[H.blocks[b].col];
    const auto& D = H.dn[H.slot[b]].D;
    std::vector<Enc> enc = std::move(encs[b]);
    std::vector<std::pair<int64_t, int64_t>> sp;
    for (int c : lv[H.blocks[b].row]) sp.push_back({ct.cl[c].start - t.start, ct.cl[c].end - t.start});
    dt.off[b] = pack_tiled(P.pk, enc, true, t.size(), s.size(), sp);
    dt.fidx[b] = direct_fmt(P.pk, enc[0].fw());
    dt.scale[b] = enc[0].scale();
    P.fp64_dense += (int64_t)D.size() * 8;
  }
  return true;
}

int32_t direct_fmt(Packer& pk, uint32_t fw) {
  pk.fmts.push_back(fw);
  return ~(int32_t)(pk.fmts.size() - 1);
}

// Leaf chunks producing y: tiles from `rowtiles(c)` then dense tiles; sorted by bytes.
void add_leaf_chunks(Ctx& cx, Program& P, const std::vector<std::vector<int>>& lv, const DenseTiles& dt,
                     const std::function<void(int, std::vector<Tile>&)>& rowtiles) {
  HostMatrix& H = cx.M->H;
  const auto& ct = H.ct;
  std::vector<std::vector<int>> rowblocks(ct.cl.size());
  for (size_t b = 0; b < H.blocks.size(); ++b)
    if (!H.blocks[b].adm) rowblocks[H.blocks[b].row].push_back((int)b);
  struct CW {
    Chunk c;
    std::vector<Tile> t;
    int64_t bytes;
  };
  std::vector<CW> cws;
  for (int c : lv[0]) {
    CW w;
    w.c.row0 = (int32_t)ct.cl[c].start;
    w.c.nrows = (int32_t)ct.cl[c].size();
    w.c.flags = 0;
    w.c.pad = 0;
    rowtiles(c, w.t);
    // dense tiles from the block rows of c's ancestors (root first, Alg. 3 order)
    std::vector<int> anc;
    for (int a = c; a >= 0; a = ct.cl[a].parent) anc.push_back(a);
    std::reverse(anc.begin(), anc.end());
    for (int a : anc)
      for (int b : rowblocks[a]) {
        size_t li = leaf_index(ct, lv[a], c);
        Tile T{};
        T.off = dt.off[b][li];
        T.fmt = dt.fidx[b];
        T.ncols = (int32_t)ct.cl[H.blocks[b].col].size();
        T.vin = (int32_t)ct.cl[H.blocks[b].col].start;
        T.flags = 1;
        T.scale = dt.scale[b];
        w.t.push_back(T);
      }
    w.bytes = 0;
    for (auto& t : w.t) w.bytes += t.ncols;
    cws.push_back(std::move(w));
  }
  std::stable_sort(cws.begin(), cws.end(), [](const CW& a, const CW& b) { return a.bytes > b.bytes; });
  int64_t off = (int64_t)P.chunks.size();
  for (auto& w : cws) {
    w.c.t0 = (int32_t)P.tiles.size();
    P.tiles.insert(P.tiles.end(), w.t.begin(), w.t.end());
    w.c.t1 = (int32_t)P.tiles.size();
    P.chunks.push_back(w.c);
  }
  add_launch(P, Launch::RGEMV, off, (int64_t)cws.size(), MODE_Y);
}

// VALR keys
std::vector<int> keys_lowrank(const Ctx& cx, const std::vector<double>& s) {
  std::vector<int> k(s.size(), cx.key_eps);
  if (cx.codec == HM_CODEC_NONE) return k;
  if (!cx.valr) return k;
  double nrm = 0;
  for (double v : s) nrm += v * v;
  double delta = cx.eps * std::sqrt(nrm) / (1.0 + 2.0 * (double)s.size());
  for (size_t i = 0; i < s.size(); ++i) k[i] = valr_key(s[i], delta);
  return k;
}

std::vector<int> keys_basis(const Ctx& cx, const std::vector<double>& sig, double tau) {
  std::vector<int> k(sig.size(), cx.key_eps);
  if (cx.codec == HM_CODEC_NONE || !cx.valr || sig.empty()) return k;
  double delta = tau / (double)sig.size();
  for (size_t i = 0; i < sig.size(); ++i) k[i] = valr_key(sig[i], delta);
  return k;
}

bool enc_matrix_cols(Ctx& cx, const std::vector<double>& A, int64_t m, int64_t n, const std::vector<int>& keys,
                     std::vector<Enc>& enc) {
  enc.assign(n, Enc());
  for (int64_t j = 0; j < n; ++j)
    if (!enc_col(cx, A.data() + j * m, m, keys[j], enc[j])) return false;
  return true;
}

// ---------------------------------------------------------------- H program
bool program_h(Ctx& cx) {
  hm_matrix* M = cx.M;
  HostMatrix& H = M->H;
  Program& P = M->prog;
  const auto& ct = H.ct;
  const int64_t N = H.n;
  auto lv = leaves_under(ct);
  DenseTiles dt;
  if (!pack_dense(cx, P, lv, dt)) return false;
  // low-rank blocks
  const size_t nb = H.blocks.size();
  std::vector<int64_t> toff(nb, -1);
  std::vector<std::vector<uint64_t>> wtile(nb);
  std::vector<int32_t> wfmt(nb, 0);
  int64_t vec = N;
  int64_t pbase = 0;
  int64_t items0 = (int64_t)P.items.size();
  int64_t g0 = (int64_t)P.gouts.size();
  std::vector<std::vector<Enc>> encx(nb), encw(nb);
  std::atomic<bool> ok{true};
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t b = 0; b < (int64_t)nb; ++b) {
    if (!H.blocks[b].adm) continue;
    const auto& L = H.lr[H.slot[b]];
    if (L.k == 0) continue;
    auto keys = keys_lowrank(cx, L.s);
    if (!enc_matrix_cols(cx, L.X, ct.cl[H.blocks[b].col].size(), L.k, keys, encx[b])) ok = false;
    if (!enc_matrix_cols(cx, L.W, ct.cl[H.blocks[b].row].size(), L.k, keys, encw[b])) ok = false;
  }
  if (!ok) return false;
  for (size_t b = 0; b < nb; ++b) {
    if (!H.blocks[b].adm) continue;
    const auto& L = H.lr[H.slot[b]];
    if (L.k == 0) continue;
    const Cluster& t = ct.cl[H.blocks[b].row];
    const Cluster& s = ct.cl[H.blocks[b].col];
    std::vector<Enc> ex = std::move(encx[b]), ew = std::move(encw[b]);
    P.fp64_lowrank += (t.size() + s.size()) * L.k * 8;
    int32_t fx = push_fmts(P.pk, ex);
    uint64_t xo = pack_cols(P.pk, ex, false, s.size(), L.k);
    std::vector<std::vector<int32_t>> segp(L.k);
    add_cdot_items(P, xo, fx, L.k, s.size(), (int32_t)s.start, pbase, &segp);
    wfmt[b] = push_fmts(P.pk, ew);
    std::vector<std::pair<int64_t, int64_t>> sp;
    for (int c : lv[H.blocks[b].row]) sp.push_back({ct.cl[c].start - t.start, ct.cl[c].end - t.start});
    wtile[b] = pack_tiled(P.pk, ew, false, t.size(), L.k, sp);
    toff[b] = vec;
    for (int j = 0; j < L.k; ++j) {
      GsumOut o{};
      o.out = (int32_t)(vec + j);
      o.p0 = (int32_t)P.plist.size();
      for (int32_t p : segp[j]) {
        P.plist.push_back(p);
        P.pscale.push_back(1.0);
      }
      o.p1 = (int32_t)P.plist.size();
      o.flags = 1;
      o.scale = L.s[j] * ex[j].scale() * ew[j].scale();
      P.gouts.push_back(o);
    }
    vec += L.k;
  }
  P.npartial = std::max(P.npartial, pbase);
  add_launch(P, Launch::GATHER, 0, N);
  add_launch(P, Launch::CDOT, items0, (int64_t)P.items.size() - items0);
  add_launch(P, Launch::GSUM, g0, (int64_t)P.gouts.size() - g0);
  // low-rank row tiles of leaf c: blocks of the block rows of c's ancestors
  std::vector<std::vector<int>> rowlr(ct.cl.size());
  for (size_t b = 0; b < nb; ++b)
    if (toff[b] >= 0) rowlr[H.blocks[b].row].push_back((int)b);
  add_leaf_chunks(cx, P, lv, dt, [&](int c, std::vector<Tile>& out) {
    std::vector<int> anc;
    for (int a = c; a >= 0; a = ct.cl[a].parent) anc.push_back(a);
    std::reverse(anc.begin(), anc.end());
    for (int a : anc)
      for (int b : rowlr[a]) {
        size_t li = leaf_index(ct, lv[a], c);
        Tile T{};
        T.off = wtile[b][li];
        T.fmt = wfmt[b];
        T.ncols = H.lr[H.slot[b]].k;
        T.vin = (int32_t)toff[b];
        T.flags = 0;
        T.scale = 1.0;
        out.push_back(T);
      }
  });
  P.nvec = vec;
  return true;
}

// ---------------------------------------------------------------- UH program
bool program_uh(Ctx& cx) {
  hm_matrix* M = cx.M;
  HostMatrix& H = M->H;
  Program& P = M->prog;
  const auto& ct = H.ct;
  const int64_t N = H.n;
  const int nc = (int)ct.cl.size();
  auto lv = leaves_under(ct);
  DenseTiles dt;
  if (!pack_dense(cx, P, lv, dt)) return false;
  int64_t vec = N, pbase = 0;
  int64_t items0 = (int64_t)P.items.size(), g0 = (int64_t)P.gouts.size();
  // forward: s_sigma = X_sigma^T x (Alg. 4) for every column basis
  std::vector<int64_t> soff(nc, -1), toff(nc, -1);
  for (int c = 0; c < nc; ++c) {
    int k = H.colb.k[c];
    if (k == 0) continue;
    const int64_t m = ct.cl[c].size();
    auto keys = keys_basis(cx, H.colb.sig[c], H.colb.tau);
    std::vector<Enc> ex;
    if (!enc_matrix_cols(cx, H.colb.B[c], m, k, keys, ex)) return false;
    P.fp64_lowrank += m * k * 8;
    int32_t fx = push_fmts(P.pk, ex);
    uint64_t xo = pack_cols(P.pk, ex, false, m, k);
    std::vector<std::vector<int32_t>> segp(k);
    add_cdot_items(P, xo, fx, k, m, (int32_t)ct.cl[c].start, pbase, &segp);
    soff[c] = vec;
    for (int j = 0; j < k; ++j) {
      GsumOut o{};
      o.out = (int32_t)(vec + j);
      o.p0 = (int32_t)P.plist.size();
      for (int32_t p : segp[j]) {
        P.plist.push_back(p);
        P.pscale.push_back(1.0);
      }
      o.p1 = (int32_t)P.plist.size();
      o.flags = 0;
      o.scale = ex[j].scale();
      P.gouts.push_back(o);
    }
    vec += k;
  }
  P.npartial = std::max(P.npartial, pbase);
  add_launch(P, Launch::GATHER, 0, N);
  add_launch(P, Launch::CDOT, items0, (int64_t)P.items.size() - items0);
  add_launch(P, Launch::GSUM, g0, (int64_t)P.gouts.size() - g0);
  // row bases (tiles per leaf) and their column scales
  std::vector<std::vector<uint64_t>> wtile(nc);
  std::vector<int32_t> wfmt(nc, 0);
  P.rowscale.assign(0, 0.0);
  std::vector<double> wscale;   // per t' entry
  for (int c = 0; c < nc; ++c) {
    int k = H.rowb.k[c];
    if (k == 0) continue;
    const int64_t m = ct.cl[c].size();
    auto keys = keys_basis(cx, H.rowb.sig[c], H.rowb.tau);
    std::vector<Enc> ew;
    if (!enc_matrix_cols(cx, H.rowb.B[c], m, k, keys, ew)) return false;
    P.fp64_lowrank += m * k * 8;
    wfmt[c] = push_fmts(P.pk, ew);
    std::vector<std::pair<int64_t, int64_t>> sp;
    for (int l : lv[c]) sp.push_back({ct.cl[l].start - ct.cl[c].start, ct.cl[l].end - ct.cl[c].start});
    wtile[c] = pack_tiled(P.pk, ew, false, m, k, sp);
    toff[c] = vec;
    for (int j = 0; j < k; ++j) wscale.push_back(ew[j].scale());
    vec += k;
  }
  // rowscale indexed by vector position: fill for t' entries
  P.rowscale.assign(vec, 1.0);
  {
    size_t wi = 0;
    for (int c = 0; c < nc; ++c)
      for (int j = 0; j < H.rowb.k[c]; ++j) P.rowscale[toff[c] + j] = wscale[wi++];
  }
  // coupling chunks (eq. sumcoup): t'_tau = alpha * vminW * sum S s
  std::vector<std::vector<int>> rowlr(nc);
  for (size_t b = 0; b < H.blocks.size(); ++b)
    if (H.blocks[b].adm) rowlr[H.blocks[b].row].push_back((int)b);
  int64_t c0 = (int64_t)P.chunks.size();
  for (int t = 0; t < nc; ++t) {
    const int kt = H.rowb.k[t];
    if (kt == 0) continue;
    // encode couplings of the row once, tiles by 128-row splits
    auto sp = row_splits(kt);
    std::vector<std::vector<Tile>> per(sp.size());
    for (int b : rowlr[t]) {
      const int s = H.blocks[b].col;
      const int ks = H.colb.k[s];
      if (ks == 0) continue;
      const auto& S = H.coupling[H.slot[b]];
      std::vector<Enc> enc(1);
      if (!encode(S.data(), (int64_t)S.size(), 1, cx.codec, cx.key_eps, enc[0])) return false;
      P.fp64_lowrank += (int64_t)S.size() * 8;
      auto offs = pack_tiled(P.pk, enc, true, kt, ks, sp);
      int32_t f = direct_fmt(P.pk, enc[0].fw());
      for (size_t i = 0; i < sp.size(); ++i) {
        Tile T{};
        T.off = offs[i];
        T.fmt = f;
        T.ncols = ks;
        T.vin = (int32_t)soff[s];
        T.flags = 0;
        T.scale = enc[0].scale();
        per[i].push_back(T);
      }
    }
    for (size_t i = 0; i < sp.size(); ++i) {
      Chunk C{};
      C.row0 = (int32_t)(toff[t] + sp[i].first);
      C.nrows = (int32_t)(sp[i].second - sp[i].first);
      C.flags = 1;
      C.t0 = (int32_t)P.tiles.size();
      P.tiles.insert(P.tiles.end(), per[i].begin(), per[i].end());
      C.t1 = (int32_t)P.tiles.size();
      P.chunks.push_back(C);
    }
  }
  add_launch(P, Launch::RGEMV, c0, (int64_t)P.chunks.size() - c0, MODE_VEC, false, true);
  // backward (Alg. 5): y|c += sum over ancestors W_tau[c,:] t'_tau, plus dense
  add_leaf_chunks(cx, P, lv, dt, [&](int c, std::vector<Tile>& out) {
    std::vector<int> anc;
    for (int a = c; a >= 0; a = ct.cl[a].parent) anc.push_back(a);
    std::reverse(anc.begin(), anc.end());
    for (int a : anc) {
      if (H.rowb.k[a] == 0) continue;
      size_t li = leaf_index(ct, lv[a], c);
      Tile T{};
      T.off = wtile[a][li];
      T.fmt = wfmt[a];
      T.ncols = H.rowb.k[a];
      T.vin = (int32_t)toff[a];
      T.flags = 0;
      T.scale = 1.0;
      out.push_back(T);
    }
  });
  P.nvec = vec;
  return true;
}

// ---------------------------------------------------------------- H^2 program
bool program_h2(Ctx& cx) {
  hm_matrix* M = cx.M;
  HostMatrix& H = M->H;
  Program& P = M->prog;
  const auto& ct = H.ct;
  const int64_t N = H.n;
  const int nc = (int)ct.cl.size();
  for (int c = 0; c < nc; ++c)
    if (H.rowb.k[c] > 128 || H.colb.k[c] > 128) return false;   // transfer tiles hold <= 128 rows
  auto lv = leaves_under(ct);
  DenseTiles dt;
  if (!pack_dense(cx, P, lv, dt)) return false;
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
  add_launch(P, Launch::GATHER, 0, N);
  // leaf forward (Alg. 6, leaves)
  int64_t pbase = 0;
  int64_t items0 = (int64_t)P.items.size(), g0 = (int64_t)P.gouts.size();
  for (int c = 0; c < nc; ++c) {
    const int k = H.colb.k[c];
    if (!ct.cl[c].leaf() || k == 0) continue;
    const int64_t m = ct.cl[c].size();
    auto keys = keys_basis(cx, H.colb.sig[c], H.colb.tau);
    std::vector<Enc> ex;
    if (!enc_matrix_cols(cx, H.colb.B[c], m, k, keys, ex)) return false;
    P.fp64_lowrank += m * k * 8;
    int32_t fx = push_fmts(P.pk, ex);
    uint64_t xo = pack_cols(P.pk, ex, false, m, k);
    std::vector<std::vector<int32_t>> segp(k);
    add_cdot_items(P, xo, fx, k, m, (int32_t)ct.cl[c].start, pbase, &segp);
    for (int j = 0; j < k; ++j) {
      GsumOut o{};
      o.out = (int32_t)(soff[c] + j);
      o.p0 = (int32_t)P.plist.size();
      for (int32_t p : segp[j]) {
        P.plist.push_back(p);
        P.pscale.push_back(1.0);
      }
      o.p1 = (int32_t)P.plist.size();
      o.flags = 0;
      o.scale = ex[j].scale();
      P.gouts.push_back(o);
    }
  }
  P.npartial = std::max(P.npartial, pbase);
  add_launch(P, Launch::CDOT, items0, (int64_t)P.items.size() - items0);
  add_launch(P, Launch::GSUM, g0, (int64_t)P.gouts.size() - g0, 0, true);
  // transfer matrices (direct compression), one tile each (k_child x k_parent)
  std::vector<uint64_t> exoff(nc, 0), ewoff(nc, 0);
  std::vector<int32_t> exf(nc, 0), ewf(nc, 0);
  std::vector<double> exs(nc, 1.0), ews(nc, 1.0);
  for (int c = 0; c < nc; ++c) {
    int p = ct.cl[c].parent;
    if (p < 0) continue;
    for (int side = 0; side < 2; ++side) {
      const Bases& bs = side ? H.colb : H.rowb;
      int kc = bs.k[c], kp = bs.k[p];
      if (kc == 0 || kp == 0) continue;
      std::vector<Enc> enc(1);
      if (!encode(bs.E[c].data(), (int64_t)bs.E[c].size(), 1, cx.codec, cx.key_eps, enc[0])) return false;
      P.fp64_lowrank += (int64_t)bs.E[c].size() * 8;
      uint64_t o = pack_cols(P.pk, enc, true, kc, kp);
      int32_t f = direct_fmt(P.pk, enc[0].fw());
      if (side) {
        exoff[c] = o; exf[c] = f; exs[c] = enc[0].scale();
      } else {
        ewoff[c] = o; ewf[c] = f; ews[c] = enc[0].scale();
      }
    }
  }
  // up-sweep by height: s_sigma = sum_i E_i^T s_i (Alg. 6)
  std::vector<int> height(nc, 0);
  int maxh = 0;
  for (int c = nc - 1; c >= 0; --c) {   // pre-order ids: sons after parents
    if (!ct.cl[c].leaf()) height[c] = 1 + std::max(height[ct.cl[c].son[0]], height[ct.cl[c].son[1]]);
    maxh = std::max(maxh, height[c]);
  }
  for (int h = 1; h <= maxh; ++h) {
    int64_t i0 = (int64_t)P.items.size(), o0 = (int64_t)P.gouts.size();
    int64_t pb = 0;
    for (int c = 0; c < nc; ++c) {
      if (height[c] != h || H.colb.k[c] == 0) continue;
      const int kp = H.colb.k[c];
      std::vector<std::pair<int32_t, double>> parts[128];
      for (int i = 0; i < 2; ++i) {
        int sc = ct.cl[c].son[i];
        int ks = H.colb.k[sc];
        if (ks == 0) continue;
        std::vector<std::vector<int32_t>> segp(kp);
        add_cdot_items(P, exoff[sc], exf[sc], kp, ks, (int32_t)soff[sc], pb, &segp);
        for (int j = 0; j < kp; ++j)
          for (int32_t p : segp[j]) parts[j].push_back({p, exs[sc]});
      }
      for (int j = 0; j < kp; ++j) {
        GsumOut o{};
        o.out = (int32_t)(soff[c] + j);
        o.p0 = (int32_t)P.plist.size();
        for (auto& pr : parts[j]) {
          P.plist.push_back(pr.first);
          P.pscale.push_back(pr.second);
        }
        o.p1 = (int32_t)P.plist.size();
        o.flags = 0;
        o.scale = 1.0;
        P.gouts.push_back(o);
      }
    }
    P.npartial = std::max(P.npartial, pb);
    add_launch(P, Launch::CDOT, i0, (int64_t)P.items.size() - i0);
    add_launch(P, Launch::GSUM, o0, (int64_t)P.gouts.size() - o0, 0, true);
  }
  // leaf row bases, tile per leaf
  std::vector<uint64_t> wleaf(nc, 0);
  std::vector<int32_t> wleaff(nc, 0);
  P.rowscale.assign(vec, 1.0);
  for (int c = 0; c < nc; ++c) {
    const int k = H.rowb.k[c];
    if (!ct.cl[c].leaf() || k == 0) continue;
    const int64_t m = ct.cl[c].size();
    auto keys = keys_basis(cx, H.rowb.sig[c], H.rowb.tau);
    std::vector<Enc> ew;
    if (!enc_matrix_cols(cx, H.rowb.B[c], m, k, keys, ew)) return false;
    P.fp64_lowrank += m * k * 8;
    wleaff[c] = push_fmts(P.pk, ew);
    wleaf[c] = pack_tiled(P.pk, ew, false, m, k, {{0, m}})[0];
    for (int j = 0; j < k; ++j) P.rowscale[toff[c] + j] = ew[j].scale();
  }
  // coupling: t_tau = sum S s (unscaled)
  std::vector<std::vector<int>> rowlr(nc);
  for (size_t b = 0; b < H.blocks.size(); ++b)
    if (H.blocks[b].adm) rowlr[H.blocks[b].row].push_back((int)b);
  int64_t c0 = (int64_t)P.chunks.size();
  for (int t = 0; t < nc; ++t) {
    const int kt = H.rowb.k[t];
    if (kt == 0) continue;
    auto sp = row_splits(kt);
    std::vector<std::vector<Tile>> per(sp.size());
    for (int b : rowlr[t]) {
      const int s = H.blocks[b].col;
      const int ks = H.colb.k[s];
      if (ks == 0) continue;
      const auto& S = H.coupling[H.slot[b]];
      std::vector<Enc> enc(1);
      if (!encode(S.data(), (int64_t)S.size(), 1, cx.codec, cx.key_eps, enc[0])) return false;
      P.fp64_lowrank += (int64_t)S.size() * 8;
      auto offs = pack_tiled(P.pk, enc, true, kt, ks, sp);
      int32_t f = direct_fmt(P.pk, enc[0].fw());
      for (size_t i = 0; i < sp.size(); ++i) {
        Tile T{};
        T.off = offs[i];
        T.fmt = f;
        T.ncols = ks;
        T.vin = (int32_t)soff[s];
        T.flags = 0;
        T.scale = enc[0].scale();
        per[i].push_back(T);
      }
    }
    for (size_t i = 0; i < sp.size(); ++i) {
      Chunk C{};
      C.row0 = (int32_t)(toff[t] + sp[i].first);
      C.nrows = (int32_t)(sp[i].second - sp[i].first);
      C.flags = 0;
      C.t0 = (int32_t)P.tiles.size();
      P.tiles.insert(P.tiles.end(), per[i].begin(), per[i].end());
      C.t1 = (int32_t)P.tiles.size();
      P.chunks.push_back(C);
    }
  }
  // a root-level leaf (no parent) still needs its scaling: handled by the
  // down-sweep pass below only for level >= 1; a leaf root has no low-rank data.
  add_launch(P, Launch::RGEMV, c0, (int64_t)P.chunks.size() - c0, MODE_VEC, false, false);
  // down-sweep by level: t_child += E_child t_parent; leaves scaled by alpha * vminW
  for (int lev = 1; lev <= ct.depth; ++lev) {
    int64_t k0 = (int64_t)P.chunks.size();
    for (int c = 0; c < nc; ++c) {
      if (ct.cl[c].level != lev || H.rowb.k[c] == 0) continue;
      int p = ct.cl[c].parent;
      Chunk C{};
      C.row0 = (int32_t)toff[c];
      C.nrows = H.rowb.k[c];
      C.flags = ct.cl[c].leaf() ? 1 : 0;
      C.t0 = (int32_t)P.tiles.size();
      if (H.rowb.k[p] > 0) {
        Tile T{};
        T.off = ewoff[c];
        T.fmt = ewf[c];
        T.ncols = H.rowb.k[p];
        T.vin = (int32_t)toff[p];
        T.flags = 0;
        T.scale = ews[c];
        P.tiles.push_back(T);
      }
      C.t1 = (int32_t)P.tiles.size();
      P.chunks.push_back(C);
    }
    add_launch(P, Launch::RGEMV, k0, (int64_t)P.chunks.size() - k0, MODE_VEC_ADD, false, true);
  }
  // backward at the leaves (Alg. 7) plus dense blocks
  add_leaf_chunks(cx, P, lv, dt, [&](int c, std::vector<Tile>& out) {
    if (H.rowb.k[c] == 0) return;
    Tile T{};
    T.off = wleaf[c];
    T.fmt = wleaff[c];
    T.ncols = H.rowb.k[c];
    T.vin = (int32_t)toff[c];
    T.flags = 0;
    T.scale = 1.0;
    out.push_back(T);
  });
  P.nvec = vec;
  return true;
}

// Algorithmic bytes of every launch (values without padding, format words,
// descriptors, vector reads / writes).
void launch_bytes(Program& P) {
  auto colbytes = [&](int32_t fmt, int ncols, int64_t rows) {
    int64_t b = 0;
    if (fmt < 0) {
      b = rows * (int64_t)(P.pk.fmts[~fmt] & 0xff) * ncols + 4;
    } else {
      for (int j = 0; j < ncols; ++j) b += rows * (int64_t)(P.pk.fmts[fmt + j] & 0xff) + 4;
    }
    return b;
  };
  for (Launch& L : P.launches) {
    int64_t b = 0;
    switch (L.kind) {
      case Launch::GATHER:
        b = L.n * (4 + 8 + 8);
        break;
      case Launch::CDOT:
        for (int64_t i = L.off; i < L.off + L.n; ++i) {
          const CdotItem& it = P.items[i];
          int64_t vb = colbytes(it.fmt, it.ncols, it.seg);
          if (it.fmt >= 0) vb -= 0;   // format words counted once per item
          b += vb + (int64_t)sizeof(CdotItem) + 8 * (int64_t)it.seg + 8 * (int64_t)it.ncols;
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
          for (int32_t t = c.t0; t < c.t1; ++t) {
            const Tile& T = P.tiles[t];
            b += (int64_t)sizeof(Tile) + colbytes(T.fmt, T.ncols, c.nrows) + 8 * (int64_t)T.ncols;
          }
          if (L.mode == MODE_Y) b += (int64_t)c.nrows * (4 + 8 + 8);
          else b += (int64_t)c.nrows * ((L.mode == MODE_VEC_ADD ? 16 : 8) + (L.use_rowscale ? 8 : 0));
        }
        break;
    }
    L.bytes = b;
  }
}

hm_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HM_OK;
  if (e == cudaErrorMemoryAllocation) return HM_ERR_OOM;
  return HM_ERR_CUDA;
}

hm_status upload(hm_matrix* M) {
  Program& P = M->prog;
  cudaError_t e;
#define UP(arr, vec) \
  if ((e = M->arr.upload(vec)) != cudaSuccess) return cuda_status(e);
  UP(d_pay, P.pk.pay)
  UP(d_fmt, P.pk.fmts)
  UP(d_items, P.items)
  UP(d_gout, P.gouts)
  UP(d_plist, P.plist)
  UP(d_pscale, P.pscale)
  UP(d_tiles, P.tiles)
  UP(d_chunks, P.chunks)
  UP(d_rowscale, P.rowscale)
#undef UP
  std::vector<int32_t> perm(M->H.n);
  for (int64_t i = 0; i < M->H.n; ++i) perm[i] = (int32_t)M->H.ct.perm[i];
  if ((e = M->d_perm.upload(perm)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMalloc(&M->d_vec, std::max<int64_t>(P.nvec, 1) * sizeof(float2))) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMalloc(&M->d_part, std::max<int64_t>(P.npartial, 1) * sizeof(double))) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMalloc(&M->d_err, sizeof(int))) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemset(M->d_err, 0, sizeof(int))) != cudaSuccess) return cuda_status(e);
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  M->grid_cdot = sms * 8;
  M->grid_rg = sms * 12;
  (void)occ;
  return HM_OK;
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
    case HM_ERR_CAPACITY: return "request exceeds the fixed device scratch of hm_matvec_host_noalloc";
  }
  return "unknown status";
}

hm_status hm_build(const hm_build_params* prm, const double* pts, int64_t n, hm_matrix** out) {
  if (!prm || !pts || !out || n < 1 || n > (int64_t)INT32_MAX / 2) return HM_ERR_ARG;
  if (prm->leaf_size < 1 || prm->leaf_size > 128) return HM_ERR_ARG;
  if (!(prm->eta > 0) || !(prm->eps_build > 0 && prm->eps_build < 1)) return HM_ERR_ARG;
  if (prm->format < HM_FMT_H || prm->format > HM_FMT_H2) return HM_ERR_ARG;
  if (prm->kernel != HM_KERNEL_LAPLACE && prm->kernel != HM_KERNEL_MATERN15) return HM_ERR_ARG;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(pts[i])) return HM_ERR_ARG;
  std::unique_ptr<hm_matrix> M;
  try {
    M.reset(new hm_matrix());
    HostMatrix& H = M->H;
    H.prm = *prm;
    H.n = n;
    H.kparam = prm->kparam > 0 ? prm->kparam
                               : (prm->kernel == HM_KERNEL_LAPLACE ? std::sqrt(4.0 * M_PI / (double)n) : 0.1);
    H.pts.assign(pts, pts + 3 * n);
    int nth = prm->nthreads > 0 ? prm->nthreads : (int)std::max(1u, std::thread::hardware_concurrency());
    build_cluster_tree(H.pts.data(), n, prm->leaf_size, H.ct);
    build_block_tree(H.ct, prm->eta, H.blocks);
    build_lowrank_blocks(H, nth);
    if (prm->format == HM_FMT_UH) build_uniform_bases(H, nth);
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
  cudaDeviceSynchronize();
  M->release_device();
  M->prog = Program();
  Ctx cx{M, codec, eps, valr ? 1 : 0, m_eps(eps)};
  Program& P = M->prog;
  P.tier = (codec == HM_CODEC_NONE || eps <= 0x1p-22) ? TIER_FF : TIER_F32;
  bool ok;
  try {
    switch (M->H.prm.format) {
      case HM_FMT_H: ok = program_h(cx); break;
      case HM_FMT_UH: ok = program_uh(cx); break;
      default: ok = program_h2(cx); break;
    }
  } catch (const std::bad_alloc&) {
    return HM_ERR_OOM;
  }
  if (!ok) {
    M->prog = Program();
    return HM_ERR_UNSUPPORTED;
  }
  P.pk.pay.resize(P.pk.pay.size() + 64, 0);   // tail reads of the last column stay in bounds
  launch_bytes(P);
  hm_status s = upload(M);
  if (s != HM_OK) {
    M->release_device();
    return s;
  }
  M->codec = codec;
  M->valr = valr ? 1 : 0;
  M->eps = eps;
  M->compressed = true;
  return HM_OK;
}

static hm_status run_program(hm_matrix* M, double alpha, const double* x, double beta, double* y,
                             cudaStream_t st) {
  Program& P = M->prog;
  cudaError_t e = cudaSuccess;
  for (const Launch& L : P.launches) {
    hm_matrix::Rec rec{(int)L.kind, nullptr, nullptr, L.bytes};
    if (M->prof) {
      rec.e0 = M->take_event();
      rec.e1 = M->take_event();
      cudaEventRecord(rec.e0, st);
    }
    switch (L.kind) {
      case Launch::GATHER:
        e = launch_gather(x, M->d_perm.p, (int)L.n, M->d_vec, st);
        break;
      case Launch::CDOT:
        e = launch_cdot(P.tier, M->d_items.p + L.off, (int)L.n, M->d_pay.p, M->d_fmt.p, M->d_vec,
                        M->d_part, M->d_err, M->grid_cdot, st);
        break;
      case Launch::GSUM:
        e = launch_gsum(M->d_gout.p + L.off, (int)L.n, M->d_plist.p, M->d_pscale.p, M->d_part, alpha,
                        M->d_vec, st);
        break;
      case Launch::RGEMV:
        e = launch_rgemv(P.tier, L.mode, M->d_chunks.p + L.off, (int)L.n, M->d_tiles.p, M->d_pay.p,
                         M->d_fmt.p, M->d_vec, alpha, beta, y, M->d_perm.p, M->d_vec,
                         L.use_rowscale ? M->d_rowscale.p : nullptr, M->d_err, M->grid_rg, st);
        break;
    }
    if (e != cudaSuccess) return HM_ERR_CUDA;
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
  for (int64_t r = 0; r < nrhs; ++r) {
    hm_status s = run_program(M, alpha, x + r * ldx, beta, y + r * ldy, st);
    if (s != HM_OK) return s;
  }
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
  if (cudaMemcpyAsync(M->d_hx, x, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return HM_ERR_CUDA;
  if (beta != 0.0 && cudaMemcpyAsync(M->d_hy, y, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HM_ERR_CUDA;
  hm_status s = hm_matvec(M, alpha, M->d_hx, n, beta, M->d_hy, n, nrhs, stream);
  if (s != HM_OK) return s;
  if (cudaMemcpyAsync(y, M->d_hy, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HM_ERR_CUDA;
  return HM_OK;
}

hm_status hm_profile(hm_matrix* M, int32_t enable) {
  if (!M) return HM_ERR_ARG;
  M->prof = enable != 0;
  return HM_OK;
}

hm_status hm_profile_read(hm_matrix* M, hm_kernel_stat* out, int32_t nout) {
  if (!M || !out || nout < 0 || nout > 4) return HM_ERR_ARG;
  hm_kernel_stat acc[4];
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
  o->bytes_meta = (int64_t)(P.pk.fmts.size() * 4 + P.items.size() * sizeof(CdotItem) +
                            P.gouts.size() * sizeof(GsumOut) + P.plist.size() * 12 +
                            P.tiles.size() * sizeof(Tile) + P.chunks.size() * sizeof(Chunk) +
                            P.rowscale.size() * 8 + H.n * 4);
  o->bytes_workspace = P.nvec * 8 + P.npartial * 8;
  o->nlaunches = (int64_t)P.launches.size();
  o->tier = P.tier;
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

}  // extern "C"
