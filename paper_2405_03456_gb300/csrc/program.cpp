// Packed layout of compressed H / UH / H^2 matrices and the launch program of
// one product (Sec. 3 algorithms mapped onto the GPU kernels).
//
// Layout (one payload buffer; every unit a warp copies into shared memory
// starts 16-byte aligned with an inline header, every column is 8-byte aligned):
//  * column dots (phase A: X factors of H blocks, UH column bases, H^2 leaf
//    column bases, transfer matrices for the up-sweep) are stored
//    segment-major: for each run of <= 128 rows, the rows of every column of
//    the set.  An item is one such segment of a group of columns (<= one
//    stage of bytes), with the columns' format words (and output scales).
//  * row chunks (phase C; couplings; down-sweep): each output chunk (a leaf
//    cluster, or <= 128 coefficients) reads
//      - uniform tiles: the chunk's rows of every column of one directly
//        compressed matrix (dense leaf, coupling, transfer);
//      - merged columns: the chunk's rows of every VALR-compressed column
//        that reaches it (W factors of all low-rank blocks of its ancestors'
//        block rows, or row bases), sorted by decode class, with one
//        (e, m, multiplier index) per column.
//    A chunk's data is cut into pieces (one decode class, <= 64 columns,
//    <= one stage of bytes) stored contiguously in chunk order.
// Every launch's items / pieces are split into contiguous ranges of about
// equal bytes, one per warp.  A leaf chunk owns its rows of y and gathers the
// contributions of all its ancestors' block rows itself: the race freedom of
// Alg. 3 without a root-to-leaf traversal.  A chunk that straddles two warp
// ranges is finished by whichever of its parts ends last (fixed summation
// order, so results stay bitwise reproducible).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <numeric>

#include "program.h"

namespace hm {

namespace {


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

// Packed rows [r0, r1) of every column of a direct column set, columns
// pad8(rows * B) apart: a uniform tile of a row chunk before it is cut into pieces.
struct TileData {
  std::vector<uint8_t> bytes;
  int ncols = 0;
  int64_t R = 0;
  uint32_t fw = 0;
  int32_t vin = 0;       // multiplier index of column 0
  int32_t flags = 0;     // bit 0: multiply by alpha
  F2 scale{1.0f, 0.0f};  // AFLP vmin of the matrix
};

struct Ctx {
  const HostMatrix& H;
  Program& P;
  int codec;
  double eps;
  int valr;
  int key_eps;
  int nsm;
  std::deque<TileData> tiles;   // storage of every tile until the program is laid out
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

int64_t pad8(int64_t x) { return (x + 7) & ~int64_t(7); }
uint16_t class_of(uint32_t fw) { return (uint16_t)((((fw >> 8) & 0xff) << 4) | (fw & 0xff)); }
uint16_t em_of(uint32_t fw) { return (uint16_t)(((fw >> 16) & 0xff) | ((fw >> 24) << 8)); }

// BF16 limbs that hold a decoded FP32 value of format word fw exactly (the
// multi-RHS tensor-core path): AFLP +-(s - 1) with s = 2^f (1 + k 2^-m'),
// f < 2^e, has at most max(f, m') + 1 significant bits; FPX e8 m+1; e11 / raw
// values are FP32-truncated (24).  Each limb carries 8 significant bits.
int limbs_of(uint32_t fw) {
  const int f = (int)((fw >> 8) & 0xff), e = (int)((fw >> 16) & 0xff), m = (int)(fw >> 24);
  int bits = 24;
  if (f == FMT_AFLP) bits = std::min(24, std::max((1 << e) - 1, m) + 1);
  if (f == FMT_FPX8) bits = std::min(24, m + 1);
  return (bits + 7) / 8;
}

// ---------------------------------------------------------------- warp ranges
// Split units (items / pieces) [0, n) of `bytes` into nw contiguous ranges of
// about equal bytes: unit i goes to the warp holding the midpoint of its
// bytes.  Appends nw + 1 absolute range starts (base + index) to wbeg.
int partition(const std::vector<int64_t>& bytes, int64_t base, int nw_max, std::vector<int32_t>& wbeg) {
  int64_t total = 0;
  for (int64_t b : bytes) total += b;
  const int64_t n = (int64_t)bytes.size();
  int nw = (int)std::min<int64_t>(nw_max, std::max<int64_t>(1, (total + MIN_WARP_BYTES - 1) / MIN_WARP_BYTES));
  nw = (int)std::max<int64_t>(1, std::min<int64_t>(nw, n));
  std::vector<int32_t> start(nw + 1, (int32_t)(base + n));
  int64_t cum = 0;
  int w = 0;
  start[0] = (int32_t)base;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t mid = cum + bytes[i] / 2;
    const int wi = (int)std::min<int64_t>(nw - 1, (__int128)mid * nw / std::max<int64_t>(total, 1));
    while (w < wi) start[++w] = (int32_t)(base + i);
    cum += bytes[i];
  }
  while (w < nw) start[++w] = (int32_t)(base + n);
  wbeg.insert(wbeg.end(), start.begin(), start.end());
  return nw;
}

// ---------------------------------------------------------------- column-dot pieces
// One column of a column set that takes part in a column dot, with where a
// single-segment result goes (out_final, scaled by scale_final).
struct CdotCol {
  const ColSet* cs;
  int j;
  int64_t out_final;
  double scale_final;
};

int64_t nseg_of(int64_t m) { return (m + SEG_ROWS - 1) / SEG_ROWS; }

// Pieces of the column dots of `cols` (all over the same m rows, input vector
// index of row 0 = vin): segments of <= SEG_ROWS rows, columns sorted by
// decode class, <= CPIECE_MAX_COLS columns and <= STAGE_BYTES bytes per piece.
// If m fits one segment and allow_final, the results go straight to
// v[out_final] (final_out = true); otherwise segment s of column c writes
// partial[pout[c] + s].
void pack_cdot(Program& P, const std::vector<CdotCol>& cols, int64_t m, int32_t vin, bool allow_final,
               bool use_alpha, const std::vector<int64_t>& pout, bool& final_out) {
  final_out = allow_final && m <= SEG_ROWS;
  std::vector<int> ord(cols.size());
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    return class_of(cols[a].cs->fw(cols[a].j)) < class_of(cols[b].cs->fw(cols[b].j));
  });
  for (int64_t r0 = 0; r0 < m; r0 += SEG_ROWS) {
    const int64_t R = std::min<int64_t>(m, r0 + SEG_ROWS) - r0, R8 = (R + 15) & ~int64_t(15);
    for (size_t k = 0; k < ord.size();) {
      const uint32_t fw = cols[ord[k]].cs->fw(cols[ord[k]].j);
      const uint16_t cls = class_of(fw);
      size_t k1 = k;
      while (k1 < ord.size() && class_of(cols[ord[k1]].cs->fw(cols[ord[k1]].j)) == cls) ++k1;
      const int B = (int)(fw & 0xff);
      const int64_t stride = R8 * B;
      const int64_t percol = stride + (int64_t)sizeof(CColMeta) + (final_out ? 8 : 0);
      const int per = (int)std::min<int64_t>(CPIECE_MAX_COLS, (STAGE_BYTES - (int64_t)sizeof(CPieceHdr)) / percol);
      for (size_t a = k; a < k1; a += per) {
        const int nc = (int)std::min<size_t>(per, k1 - a);
        const uint64_t off = P.pk.align(16);
        CPieceHdr h{};
        h.vin = (int32_t)(vin + r0);
        h.nrows = (uint16_t)R;
        h.ncols = (uint16_t)nc;
        h.fb = cls;
        h.flags = (uint16_t)(final_out ? (ITEM_FINAL | (use_alpha ? ITEM_ALPHA : 0)) : 0);
        for (int t = 0; t < nc; ++t) {
          const CdotCol& cc = cols[ord[a + t]];
          h.limbs = std::max(h.limbs, (int32_t)limbs_of(cc.cs->fw(cc.j)));
        }
        P.pk.raw(&h, sizeof h);
        std::vector<CColMeta> cm(nc);
        std::vector<F2> sc;
        for (int t = 0; t < nc; ++t) {
          const int c = ord[a + t];
          cm[t].em = em_of(cols[c].cs->fw(cols[c].j));
          if (final_out) {
            cm[t].out = (int32_t)cols[c].out_final;
            sc.push_back(split_ff(cols[c].scale_final));
          } else {
            cm[t].out = (int32_t)(pout[c] + r0 / SEG_ROWS);
          }
        }
        P.pk.raw(cm.data(), cm.size() * sizeof(CColMeta));
        if (final_out) P.pk.raw(sc.data(), sc.size() * sizeof(F2));
        for (int t = 0; t < nc; ++t) {
          const CdotCol& cc = cols[ord[a + t]];
          P.pk.put_rows(cc.cs->col(cc.j) + r0, R, R8, B);
        }
        const uint64_t end = P.pk.align(8);
        P.items.push_back(ItemCopy{(uint32_t)(off >> 4), (uint32_t)(end - off), h.vin, (int32_t)R});
        // values, header, column metadata, scales, input rows, outputs, copy descriptor
        P.item_alg.push_back(R * B * nc + (int64_t)sizeof(CPieceHdr) + (8 + 8 + (final_out ? 8 : 0)) * nc + 8 * R +
                             (int64_t)sizeof(ItemCopy));
      }
      k = k1;
    }
  }
}

// coefficient out = scale * (alpha if flags & 1) * sum_p w_p partial[p], p in [p0, p1)
// (w_p = pscale[p - p0] when given, else 1)
void gsum_one(Program& P, int64_t out, int64_t p0, int64_t p1, const std::vector<double>& pscale, double scale,
              int flags) {
  GsumOut o{};
  o.out = (int32_t)out;
  o.p0 = (int32_t)p0;
  o.p1 = (int32_t)p1;
  o.flags = flags;
  o.ps = -1;
  if (!pscale.empty()) {
    o.flags |= 2;
    o.ps = (int32_t)P.pscale.size();
    for (double w : pscale) P.pscale.push_back(split_ff(w));
  }
  o.scale = split_ff(scale);
  P.gouts.push_back(o);
}

// ---------------------------------------------------------------- row-chunk pieces
// Uniform tile: rows [r0, r1) of every column of a direct column set.
const TileData* pack_tile(Ctx& cx, const ColSet& cs, int64_t r0, int64_t r1, int32_t vin, int32_t flags) {
  cx.tiles.emplace_back();
  TileData& T = cx.tiles.back();
  const int B = cs.B(0);
  const int64_t R = r1 - r0, stride = pad8(R * B);
  T.bytes.assign((size_t)(stride * cs.n), 0);
  for (int j = 0; j < cs.n; ++j) {
    const uint64_t* c = cs.col(j) + r0;
    uint8_t* dst = T.bytes.data() + j * stride;
    for (int64_t i = 0; i < R; ++i)
      for (int b = 0; b < B; ++b) dst[i * B + b] = (uint8_t)(c[i] >> (8 * b));
  }
  T.ncols = cs.n;
  T.R = R;
  T.fw = cs.fw(0);
  T.vin = vin;
  T.flags = flags;
  T.scale = split_ff(cs.scale(0));
  return &T;
}

// One column of a VALR set restricted to rows [r0, r1), with its multiplier.
struct ColRef {
  const ColSet* cs;
  int j;
  int64_t r0;
  int32_t vin;
};

struct ChunkWork {
  int32_t row0 = 0, nrows = 0, flags = 0;   // flags bit 0: multiply the result by alpha
  std::vector<const TileData*> t;
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

// Cut the chunks of one output launch into pieces, split the pieces into
// per-warp ranges, lay them out (headers, column metadata, columns) and append
// one RGEMV launch.
void add_rgemv(Ctx& cx, std::vector<ChunkWork>& cw, int mode, bool rowscale) {
  Program& P = cx.P;
  struct PW {
    int32_t chunk;
    const TileData* t;   // tile piece, or nullptr for merged columns
    int32_t j0;          // tile: first column; merged: first entry of the chunk's sorted list
    int32_t ncols;
    uint16_t cls;
    int64_t bytes;
  };
  std::vector<PW> pw;
  for (size_t ci = 0; ci < cw.size(); ++ci) {
    ChunkWork& c = cw[ci];
    const int64_t R = c.nrows;
    for (const TileData* t : c.t) {
      const int64_t stride = pad8(R * (int64_t)(t->fw & 0xff));
      const int per = (int)std::min<int64_t>(PIECE_MAX_COLS, (STAGE_BYTES - (int64_t)sizeof(PieceHdr)) / stride);
      for (int j0 = 0; j0 < t->ncols; j0 += per) {
        const int nc = std::min(per, t->ncols - j0);
        pw.push_back(PW{(int32_t)ci, t, j0, nc, class_of(t->fw), (int64_t)sizeof(PieceHdr) + nc * stride});
      }
    }
    std::stable_sort(c.cols.begin(), c.cols.end(), [](const ColRef& a, const ColRef& b) {
      return class_of(a.cs->fw(a.j)) < class_of(b.cs->fw(b.j));
    });
    for (size_t k = 0; k < c.cols.size();) {
      const uint32_t fw = c.cols[k].cs->fw(c.cols[k].j);
      const uint16_t cls = class_of(fw);
      size_t k1 = k;
      while (k1 < c.cols.size() && class_of(c.cols[k1].cs->fw(c.cols[k1].j)) == cls) ++k1;
      const int64_t stride = pad8(R * (int64_t)(fw & 0xff));
      const int per = (int)std::min<int64_t>(PIECE_MAX_COLS,
                                             (STAGE_BYTES - (int64_t)sizeof(PieceHdr) - 8) / (stride + 2));
      for (size_t a = k; a < k1; a += per) {
        const int nc = (int)std::min<size_t>(per, k1 - a);
        pw.push_back(PW{(int32_t)ci, nullptr, (int32_t)a, nc, cls,
                        (int64_t)sizeof(PieceHdr) + pad8(2 * nc) + nc * stride});
      }
      k = k1;
    }
    if (c.t.empty() && c.cols.empty())   // nothing to add: the chunk still writes its (zero / scaled) rows
      pw.push_back(PW{(int32_t)ci, nullptr, 0, 0, (uint16_t)((FMT_AFLP << 4) | 3), (int64_t)sizeof(PieceHdr)});
  }
  Launch L;
  L.kind = Launch::RGEMV;
  L.mode = mode;
  L.use_rowscale = rowscale;
  L.off = P.npieces;
  L.n = (int64_t)pw.size();
  for (const ChunkWork& c : cw) L.maxrows = std::max<int>(L.maxrows, (int)c.nrows);
  const int64_t fan0 = (int64_t)P.fan_src.size();
  // lay out (partition-independent headers, decode parameters, columns)
  std::vector<PieceCopy> base(pw.size());
  for (size_t i = 0; i < pw.size(); ++i) {
    const PW& p = pw[i];
    const ChunkWork& c = cw[p.chunk];
    const int64_t R = c.nrows;
    const uint64_t off = P.pk.align(16);
    PieceHdr h{};
    h.row0 = c.row0;
    h.nrows = (uint16_t)R;
    h.flags = (c.flags & 1) ? PH_CALPHA : 0;
    h.fb = p.cls;
    h.ncols = (uint16_t)p.ncols;
    h.scale = F2{1.0f, 0.0f};
    h.limbs = 1;
    if (p.t) {
      h.limbs = (uint16_t)limbs_of(p.t->fw);
    } else {
      for (int k = 0; k < p.ncols; ++k) {
        const ColRef& r = c.cols[p.j0 + k];
        h.limbs = (uint16_t)std::max<int>(h.limbs, limbs_of(r.cs->fw(r.j)));
      }
    }
    int64_t vals = 0, meta = (int64_t)sizeof(PieceHdr) + (int64_t)sizeof(PieceCopy);
    int64_t moff = 0;
    if (p.t) {
      const TileData& t = *p.t;
      const int B = (int)(t.fw & 0xff);
      const int64_t stride = pad8(R * B);
      h.flags |= PH_TILE | ((t.flags & 1) ? PH_TALPHA : 0);
      h.em = em_of(t.fw);
      h.vin0 = t.vin + p.j0;
      h.scale = t.scale;
      moff = h.vin0;
      P.pk.raw(&h, sizeof h);
      P.pk.align(8);
      P.pk.pay.insert(P.pk.pay.end(), t.bytes.begin() + p.j0 * stride, t.bytes.begin() + (p.j0 + p.ncols) * stride);
      vals = R * B * p.ncols;
      P.pk.value_bytes += vals;
      meta += 8 * p.ncols;   // multipliers
    } else {
      P.pk.raw(&h, sizeof h);
      std::vector<uint16_t> em(p.ncols);
      bool consecutive = true;
      for (int k = 0; k < p.ncols; ++k) {
        const ColRef& r = c.cols[p.j0 + k];
        em[k] = em_of(r.cs->fw(r.j));
        consecutive = consecutive && r.vin == c.cols[p.j0].vin + k;
      }
      if (p.ncols == 0) consecutive = false;
      P.pk.raw(em.data(), em.size() * sizeof(uint16_t));
      for (int k = 0; k < p.ncols; ++k) {
        const ColRef& r = c.cols[p.j0 + k];
        P.pk.put(r.cs->col(r.j) + r.r0, R, r.cs->B(r.j));
        vals += R * r.cs->B(r.j);
      }
      if (p.ncols == 0) {
        moff = 0;
      } else if (consecutive) {
        moff = c.cols[p.j0].vin;
      } else {   // a run of fan-out slots (resolved to vector indices at the end)
        moff = -1 - (int64_t)P.fan_src.size();
        for (int k = 0; k < p.ncols; ++k) P.fan_src.push_back(c.cols[p.j0 + k].vin);
      }
      meta += (2 + 8) * p.ncols;   // decode parameters + multipliers
    }
    const uint64_t end = P.pk.align(8);
    base[i] = PieceCopy{(uint32_t)(off >> 4), (uint32_t)(end - off) | ((uint32_t)p.ncols << 24), (int32_t)moff, -1};
    int64_t alg = vals + meta;
    const bool last_of_chunk = (i + 1 == pw.size()) || pw[i + 1].chunk != p.chunk;
    if (last_of_chunk) {   // output rows of the chunk
      if (mode == MODE_Y)
        alg += R * (4 + 8 + 8);
      else
        alg += R * ((mode == MODE_VEC_ADD ? 16 : 8) + (rowscale ? 8 : 0));
    }
    P.piece_alg.push_back(alg);
  }
  if ((int64_t)P.fan_src.size() > fan0)   // the slots of this launch are filled right before it
    add_launch(P, Launch::FANOUT, fan0, (int64_t)P.fan_src.size() - fan0);
  // per launch shape: warp ranges, range flags, shared chunks
  std::vector<int64_t> pb(pw.size());
  for (size_t i = 0; i < pw.size(); ++i) {
    const bool last_of_chunk = (i + 1 == pw.size()) || pw[i + 1].chunk != pw[i].chunk;
    pb[i] = pw[i].bytes + 8 * pw[i].ncols + PIECE_COST + (last_of_chunk ? EMIT_COST : 0);
  }
  int64_t nfix = 0;
  int64_t nfix_mr = 0;
  for (int cf = 0; cf < NSHAPES; ++cf) {
    L.woff[cf] = (int64_t)P.wbeg.size();
    if (pw.empty()) {
      L.nw[cf] = 0;
      continue;
    }
    L.nw[cf] = partition(pb, L.off, cx.nsm * (cf == MR_SHAPE ? MP_PAIRS : RS_CFG_WARPS[cf]), P.wbeg);
    std::vector<PieceCopy> d = base;
    std::vector<int32_t> nparts(cw.size(), 0), partof(pw.size(), 0);
    const int32_t* wb = P.wbeg.data() + L.woff[cf];
    for (int w = 0; w < L.nw[cf]; ++w) {
      const int64_t a = wb[w] - L.off, b = wb[w + 1] - L.off;
      for (int64_t i = a; i < b; ++i) {
        const int32_t ch = pw[i].chunk;
        const bool first = (i == a) || pw[i - 1].chunk != ch;
        const bool last = (i == b - 1) || pw[i + 1].chunk != ch;
        if (first) {
          d[i].bytes_flags |= PD_FIRST << 16;
          partof[i] = nparts[ch]++;
        } else {
          partof[i] = partof[i - 1];
        }
        if (last) d[i].bytes_flags |= PD_LAST << 16;
      }
    }
    std::vector<int32_t> splitof(cw.size(), -1);
    // fix-up slots: reused by the next launch, except in the persistent shape,
    // whose launches may run concurrently as phases of one launch
    const int64_t fix0 = cf == SEQ_SHAPE ? P.nfix_seq : 0;
    int64_t fix = fix0;
    for (size_t ch = 0; ch < cw.size(); ++ch)
      if (nparts[ch] > 1) {
        splitof[ch] = (int32_t)P.splits.size();
        P.splits.push_back(Split{(int32_t)fix, nparts[ch]});
        fix += nparts[ch];
      }
    if (cf == SEQ_SHAPE) P.nfix_seq = fix;
    if (cf == MR_SHAPE)
      nfix_mr = std::max(nfix_mr, fix);
    else
      nfix = std::max(nfix, fix);
    for (size_t i = 0; i < pw.size(); ++i)
      if (splitof[pw[i].chunk] >= 0) {
        d[i].bytes_flags |= PD_SPLIT << 16;
        d[i].split_part = (splitof[pw[i].chunk] << 8) | partof[i];
      }
    P.pdesc[cf].insert(P.pdesc[cf].end(), d.begin(), d.end());
  }
  P.nfix = std::max(P.nfix, nfix);
  P.nfix_mr = std::max(P.nfix_mr, nfix_mr);
  P.npieces += (int64_t)pw.size();
  P.nchunks += (int64_t)cw.size();
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
bool pack_dense(Ctx& cx, const std::vector<std::vector<int>>& lv, std::vector<std::vector<const TileData*>>& dt) {
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
      dt[b].push_back(pack_tile(cx, cs[b], ct.cl[l].start - t.start, ct.cl[l].end - t.start, (int32_t)s.start, 1));
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
void leaf_chunks(Ctx& cx, const std::vector<std::vector<int>>& lv,
                 const std::vector<std::vector<const TileData*>>& dt,
                 const std::function<void(int, std::vector<ColRef>&)>& rowcols) {
  const HostMatrix& H = cx.H;
  const auto& ct = H.ct;
  std::vector<std::vector<int>> rowdense(ct.cl.size());
  for (size_t b = 0; b < H.blocks.size(); ++b)
    if (!H.blocks[b].adm) rowdense[H.blocks[b].row].push_back((int)b);
  std::vector<ChunkWork> cw;
  for (int c : lv[0]) {
    ChunkWork w;
    w.row0 = (int32_t)ct.cl[c].start;
    w.nrows = (int32_t)ct.cl[c].size();
    rowcols(c, w.cols);
    for (int a : ancestors_root_first(ct, c))
      for (int b : rowdense[a]) w.t.push_back(dt[b][leaf_index(ct, lv[a], c)]);
    cw.push_back(std::move(w));
  }
  add_rgemv(cx, cw, MODE_Y, false);
}

// ---------------------------------------------------------------- H (Alg. 1 / 3)
bool program_h(Ctx& cx) {
  const HostMatrix& H = cx.H;
  Program& P = cx.P;
  const auto& ct = H.ct;
  const int64_t N = H.n;
  const auto lv = leaves_under(ct);
  std::vector<std::vector<const TileData*>> dt;
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
  // t_b = alpha * sigma_b * (X_b^T x|sigma): coefficient vectors after x; the
  // column dots of all blocks of one block column share the input segment
  std::vector<int64_t> toff(nb, -1);
  int64_t vec = N, pbase = 0;
  std::vector<std::vector<int>> collr(ct.cl.size());
  for (int64_t b = 0; b < nb; ++b) {
    if (!H.blocks[b].adm) continue;
    const auto& L = H.lr[H.slot[b]];
    if (L.k == 0) continue;
    P.fp64_lowrank += (ct.cl[H.blocks[b].row].size() + ct.cl[H.blocks[b].col].size()) * L.k * 8;
    toff[b] = vec;
    vec += L.k;
    collr[H.blocks[b].col].push_back((int)b);
  }
  const int64_t i0 = (int64_t)P.items.size(), g0 = (int64_t)P.gouts.size();
  for (size_t sg = 0; sg < ct.cl.size(); ++sg) {
    if (collr[sg].empty()) continue;
    std::vector<CdotCol> cols;
    for (int b : collr[sg]) {
      const auto& L = H.lr[H.slot[b]];
      for (int j = 0; j < L.k; ++j)
        cols.push_back(CdotCol{&csx[b], j, toff[b] + j, L.s[j] * csx[b].scale(j) * csw[b].scale(j)});
    }
    const int64_t ns = nseg_of(ct.cl[sg].size());
    std::vector<int64_t> pout(cols.size());
    for (size_t c = 0; c < cols.size(); ++c) pout[c] = pbase + (int64_t)c * ns;
    bool fin = false;
    pack_cdot(P, cols, ct.cl[sg].size(), (int32_t)ct.cl[sg].start, true, true, pout, fin);
    if (!fin) {
      for (size_t c = 0; c < cols.size(); ++c)
        gsum_one(P, cols[c].out_final, pout[c], pout[c] + ns, {}, cols[c].scale_final, 1);
      pbase += (int64_t)cols.size() * ns;
    }
    for (int b : collr[sg]) csx[b] = ColSet();
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
        per[i].t.push_back(pack_tile(cx, enc[b], r0, r1, (int32_t)soff[s], 0));
      }
      cx.P.fp64_lowrank += (int64_t)enc[b].m * enc[b].n * 8;
      enc[b] = ColSet();
    }
    for (int i = 0; i < nsplit; ++i) {
      per[i].row0 = (int32_t)(toff[t] + (int64_t)i * CHUNK_ROWS);
      per[i].nrows = std::min(CHUNK_ROWS, kt - i * CHUNK_ROWS);
      per[i].flags = flags;
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
    std::vector<CdotCol> cols;
    for (int j = 0; j < k; ++j) cols.push_back(CdotCol{&enc[c], j, soff[c] + j, enc[c].scale(j)});
    const int64_t ns = nseg_of(ct.cl[c].size());
    std::vector<int64_t> pout(k);
    for (int j = 0; j < k; ++j) pout[j] = pbase + (int64_t)j * ns;
    bool fin = false;
    pack_cdot(cx.P, cols, ct.cl[c].size(), (int32_t)ct.cl[c].start, true, false, pout, fin);
    if (!fin) {
      for (int j = 0; j < k; ++j) gsum_one(cx.P, soff[c] + j, pout[j], pout[j] + ns, {}, enc[c].scale(j), 0);
      pbase += (int64_t)k * ns;
    }
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
// UH with separate couplings (the variant discussed after Alg. 5): first stage
// u_b = Sc_b^T s_sigma, one chunk (of <= 128 rows) per low-rank block with the
// tile Sc_b^T; second stage t_tau = alpha sum_b Sr_b u_b, one chunk per row
// cluster with the tiles Sr_b (rows scaled as the single-coupling t_tau).  Both
// factors are compressed directly at eps.
bool separate_coupling_chunks(Ctx& cx, const std::vector<int64_t>& soff, const std::vector<int64_t>& toff,
                              const std::vector<int64_t>& uoff) {
  const HostMatrix& H = cx.H;
  const auto& ct = H.ct;
  const int nc = (int)ct.cl.size();
  const int64_t nb = (int64_t)H.blocks.size();
  std::vector<ColSet> encr(nb), encc(nb);
  std::atomic<bool> ok{true};
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t b = 0; b < nb; ++b) {
    if (uoff[b] < 0) continue;
    const int kt = H.rowb.k[H.blocks[b].row], ks = H.colb.k[H.blocks[b].col], kb = H.lr[H.slot[b]].k;
    if (!make_direct(cx, H.coupling_r[H.slot[b]].data(), kt, kb, encr[b])) ok = false;
    if (!make_direct(cx, H.coupling_ct[H.slot[b]].data(), kb, ks, encc[b])) ok = false;
  }
  if (!ok) return false;
  std::vector<ChunkWork> first, second;
  std::vector<std::vector<int>> rowlr(nc);
  for (int64_t b = 0; b < nb; ++b) {
    if (uoff[b] < 0) continue;
    rowlr[H.blocks[b].row].push_back((int)b);
    const int kb = H.lr[H.slot[b]].k;
    for (int64_t r0 = 0; r0 < kb; r0 += CHUNK_ROWS) {
      const int64_t r1 = std::min<int64_t>(kb, r0 + CHUNK_ROWS);
      ChunkWork w;
      w.row0 = (int32_t)(uoff[b] + r0);
      w.nrows = (int32_t)(r1 - r0);
      w.t.push_back(pack_tile(cx, encc[b], r0, r1, (int32_t)soff[H.blocks[b].col], 0));
      first.push_back(std::move(w));
    }
    cx.P.fp64_lowrank += (int64_t)(encc[b].m * encc[b].n + encr[b].m * encr[b].n) * 8;
  }
  for (int t = 0; t < nc; ++t) {
    const int kt = H.rowb.k[t];
    if (kt == 0) continue;
    for (int64_t r0 = 0; r0 < kt; r0 += CHUNK_ROWS) {
      const int64_t r1 = std::min<int64_t>(kt, r0 + CHUNK_ROWS);
      ChunkWork w;
      w.row0 = (int32_t)(toff[t] + r0);
      w.nrows = (int32_t)(r1 - r0);
      w.flags = 1;
      for (int b : rowlr[t]) w.t.push_back(pack_tile(cx, encr[b], r0, r1, (int32_t)uoff[b], 0));
      second.push_back(std::move(w));
    }
  }
  if (!first.empty()) add_rgemv(cx, first, MODE_VEC, false);
  add_rgemv(cx, second, MODE_VEC, true);
  return true;
}

bool program_uh(Ctx& cx) {
  const HostMatrix& H = cx.H;
  Program& P = cx.P;
  const auto& ct = H.ct;
  const int64_t N = H.n;
  const int nc = (int)ct.cl.size();
  const auto lv = leaves_under(ct);
  std::vector<std::vector<const TileData*>> dt;
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
  // UH_SEP: one coefficient vector u_b = Sc_b^T s_sigma per low-rank block
  const bool sep = H.prm.format == HM_FMT_UH_SEP;
  std::vector<int64_t> uoff(H.blocks.size(), -1);
  if (sep)
    for (size_t b = 0; b < H.blocks.size(); ++b) {
      if (!H.blocks[b].adm) continue;
      const int kb = H.lr[H.slot[b]].k;
      if (kb == 0 || H.rowb.k[H.blocks[b].row] == 0 || H.colb.k[H.blocks[b].col] == 0) continue;
      uoff[b] = vec;
      vec += kb;
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
  if (!sep) {
    if (!coupling_chunks(cx, soff, toff, cw, 1)) return false;
    add_rgemv(cx, cw, MODE_VEC, true);
  } else if (!separate_coupling_chunks(cx, soff, toff, uoff)) {
    return false;
  }
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
  for (int c = 0; c < nc; ++c)   // an up- or down-sweep chunk holds <= 128 coefficients
    if (H.rowb.k[c] > CHUNK_ROWS || H.colb.k[c] > CHUNK_ROWS) {
      P.too_large = true;
      return false;
    }
  const auto lv = leaves_under(ct);
  std::vector<std::vector<const TileData*>> dt;
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
  // transfer matrices, direct compression; the column-basis ones are stored
  // transposed (k_parent rows x k_son columns): the up-sweep is a row-chunk
  // product per parent, s_parent = sum over sons of vmin E_son^T s_son
  std::vector<ColSet> ext(nc), ew(nc);
  for (int c = 0; c < nc; ++c) {
    const int p = ct.cl[c].parent;
    if (p < 0) continue;
    if (H.colb.k[c] && H.colb.k[p]) {
      const int kc = H.colb.k[c], kp = H.colb.k[p];
      std::vector<double> et((size_t)kc * kp);
      for (int j = 0; j < kp; ++j)
        for (int i = 0; i < kc; ++i) et[(size_t)j + (size_t)i * kp] = H.colb.E[c][(size_t)i + (size_t)j * kc];
      if (!make_direct(cx, et.data(), kp, kc, ext[c])) return false;
      P.fp64_lowrank += (int64_t)H.colb.E[c].size() * 8;
    }
    if (H.rowb.k[c] && H.rowb.k[p]) {
      if (!make_direct(cx, H.rowb.E[c].data(), H.rowb.k[c], H.rowb.k[p], ew[c])) return false;
      P.fp64_lowrank += (int64_t)H.rowb.E[c].size() * 8;
    }
  }
  // up-sweep by height: s_sigma = sum over sons i of vmin_i E_i^T s_i (Alg. 6),
  // one row-chunk launch per height (chunk = s_sigma, one tile per son)
  std::vector<int> height(nc, 0);
  int maxh = 0;
  for (int c = nc - 1; c >= 0; --c) {
    if (!ct.cl[c].leaf()) height[c] = 1 + std::max(height[ct.cl[c].son[0]], height[ct.cl[c].son[1]]);
    maxh = std::max(maxh, height[c]);
  }
  for (int h = 1; h <= maxh; ++h) {
    std::vector<ChunkWork> uw;
    for (int c = 0; c < nc; ++c) {
      if (height[c] != h || H.colb.k[c] == 0) continue;
      ChunkWork w;
      w.row0 = (int32_t)soff[c];
      w.nrows = H.colb.k[c];
      for (int i = 0; i < 2; ++i) {
        const int sc = ct.cl[c].son[i];
        if (H.colb.k[sc]) w.t.push_back(pack_tile(cx, ext[sc], 0, H.colb.k[c], (int32_t)soff[sc], 0));
      }
      uw.push_back(std::move(w));
    }
    if (!uw.empty()) add_rgemv(cx, uw, MODE_VEC, false);
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
      w.row0 = (int32_t)toff[c];
      w.nrows = H.rowb.k[c];
      w.flags = ct.cl[c].leaf() ? 1 : 0;
      if (H.rowb.k[p] > 0) w.t.push_back(pack_tile(cx, ew[c], 0, H.rowb.k[c], (int32_t)toff[p], 0));
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

// Algorithmic bytes of every launch (packed values without padding, inline
// metadata, descriptors, vector reads and writes) and the warp ranges of the
// column-dot launches.
// A fan-out launch right after a segment-sum launch (which follows its column
// dots) is folded into the segment sums when every slot takes a coefficient that
// one of the two wrote: each segment-sum output also writes its own slots, and
// the slots of one-segment column-dot outputs become copy entries run by the
// same launch.  The slot values are the same; the launch goes.  A fan-out of
// coefficients that a row-chunk launch writes stays.
void fold_fanouts(Program& P) {
  std::vector<int32_t> by_gsum((size_t)P.fan_base, -1);   // coefficient -> its GsumOut, or -2: one-segment dot
  std::vector<char> gone(P.launches.size(), 0);
  for (size_t li = 2; li < P.launches.size(); ++li) {
    const Launch& F = P.launches[li];
    Launch& G = P.launches[li - 1];
    const Launch& C = P.launches[li - 2];
    if (F.kind != Launch::FANOUT || G.kind != Launch::GSUM || C.kind != Launch::CDOT || G.scatter) continue;
    std::vector<int32_t> marks;
    for (int64_t it = C.off; it < C.off + C.n; ++it) {
      const uint8_t* p = P.pk.pay.data() + (uint64_t)P.items[it].off16 * 16;
      CPieceHdr h;
      std::memcpy(&h, p, sizeof h);
      if (!(h.flags & ITEM_FINAL)) continue;
      for (int j = 0; j < h.ncols; ++j) {
        CColMeta m;
        std::memcpy(&m, p + sizeof h + (size_t)j * sizeof m, sizeof m);
        if (m.out >= 0 && m.out < P.fan_base && by_gsum[m.out] == -1) {
          by_gsum[m.out] = -2;
          marks.push_back(m.out);
        }
      }
    }
    for (int64_t i = G.off; i < G.off + G.n; ++i) {
      const int32_t o = P.gouts[i].out;
      if (o >= 0 && o < P.fan_base && by_gsum[o] == -1) {
        by_gsum[o] = (int32_t)i;
        marks.push_back(o);
      }
    }
    bool all = true;
    for (int64_t i = F.off; i < F.off + F.n && all; ++i)
      all = P.fan_src[i] >= 0 && P.fan_src[i] < P.fan_base && by_gsum[P.fan_src[i]] != -1;
    if (all) {
      // slots per segment-sum output, in slot order; copy entries in slot order
      std::vector<std::vector<int32_t>> lists((size_t)G.n);
      G.copy_off = (int64_t)P.fan_copy_src.size();
      for (int64_t i = F.off; i < F.off + F.n; ++i) {
        const int32_t src = P.fan_src[i], dst = (int32_t)(P.fan_base + i);
        if (by_gsum[src] >= 0) {
          lists[(size_t)(by_gsum[src] - G.off)].push_back(dst);
        } else {
          P.fan_copy_src.push_back(src);
          P.fan_copy_dst.push_back(dst);
        }
      }
      G.copy_n = (int64_t)P.fan_copy_src.size() - G.copy_off;
      for (int64_t i = G.off; i < G.off + G.n; ++i) {
        GsumOut& o = P.gouts[i];
        const auto& l = lists[(size_t)(i - G.off)];
        o.pad = (int32_t)P.fan_dst.size();
        o.flags = (o.flags & 0xff) | (int32_t)(l.size() << 8);
        P.fan_dst.insert(P.fan_dst.end(), l.begin(), l.end());
        G.xbytes += 12 * (int64_t)l.size();   // slot index read, value written
      }
      G.xbytes += 24 * G.copy_n;                // source and slot index, value read and written
      G.scatter = true;
      gone[li] = 1;
    }
    for (int32_t o : marks) by_gsum[o] = -1;
  }
  std::vector<Launch> keep;
  for (size_t li = 0; li < P.launches.size(); ++li)
    if (!gone[li]) keep.push_back(P.launches[li]);
  P.launches.swap(keep);
}

void finish_launches(Ctx& cx) {
  Program& P = cx.P;
  for (Launch& L : P.launches) {
    int64_t b = 0;
    switch (L.kind) {
      case Launch::GATHER:
        b = L.n * (4 + 8 + 8);
        break;
      case Launch::CDOT: {
        std::vector<int64_t> ib((size_t)L.n);
        for (int64_t i = 0; i < L.n; ++i) {
          ib[i] = P.items[L.off + i].bytes + CPIECE_COST;
          b += P.item_alg[L.off + i];
        }
        for (int cf = 0; cf < NSHAPES; ++cf) {
          L.woff[cf] = (int64_t)P.wbeg.size();
          const int nmax = cx.nsm * (cf == MR_SHAPE ? MR_CDOT_RANGES : CS_CFG_WARPS[cf]);
          L.nw[cf] = L.n > 0 ? partition(ib, L.off, nmax, P.wbeg) : 0;
        }
        break;
      }
      case Launch::GSUM:
        for (int64_t i = L.off; i < L.off + L.n; ++i) {
          const GsumOut& o = P.gouts[i];
          b += (int64_t)(o.p1 - o.p0) * ((o.flags & 2) ? 16 : 8) + (int64_t)sizeof(GsumOut) + 8;
        }
        break;
      case Launch::RGEMV:
        for (int64_t i = L.off; i < L.off + L.n; ++i) b += P.piece_alg[i];
        break;
      case Launch::FANOUT:
        b = L.n * (4 + 8 + 8);
        break;
    }
    L.bytes = b + L.xbytes;
  }
}

}  // namespace

bool build_program(const HostMatrix& H, int codec, double eps, int valr, int nsm, Program& P) {
  P = Program();
  P.tier = (codec == HM_CODEC_NONE || eps <= 0x1p-22) ? TIER_FF : TIER_F32;
  Ctx cx{H, P, codec, eps, valr ? 1 : 0, m_eps(eps), std::max(1, nsm), {}};
  bool ok;
  switch (H.prm.format) {
    case HM_FMT_H: ok = program_h(cx); break;
    case HM_FMT_UH:
    case HM_FMT_UH_SEP: ok = program_uh(cx); break;
    default: ok = program_h2(cx); break;
  }
  cx.tiles.clear();
  if (ok && P.pk.pay.size() >= (1ull << 36)) {   // copy descriptors hold offset / 16 in 32 bits
    ok = false;
    P.too_large = true;
  }
  if (!ok) {
    const bool big = P.too_large;   // set by an addressing or layout limit
    P = Program();
    P.too_large = big;
    return false;
  }
  P.pk.align(16);
  P.pk.pay.resize(P.pk.pay.size() + 256, 0);   // 16-byte rounded copies and lane over-reads stay in bounds
  // fan-out slots follow every other vector entry
  P.fan_base = P.nvec;
  P.nvec += (int64_t)P.fan_src.size();
  for (int cf = 0; cf < NSHAPES; ++cf)
    for (PieceCopy& d : P.pdesc[cf])
      if (d.moff < 0) d.moff = (int32_t)(P.fan_base + (-1 - (int64_t)d.moff));
  if (P.rowscale.size() > 1) P.rowscale.resize(P.nvec, 1.0);
  if (P.rowscale.empty()) P.rowscale.assign(1, 1.0);
  if (P.nvec >= INT32_MAX) {
    P = Program();
    P.too_large = true;
    return false;
  }
  fold_fanouts(P);
  finish_launches(cx);
  // levels without work (empty top levels of the sweeps) launch nothing
  P.launches.erase(std::remove_if(P.launches.begin(), P.launches.end(),
                                  [](const Launch& L) {
                                    return L.n == 0 && !(L.kind == Launch::RGEMV && L.mode == MODE_Y) &&
                                           !(L.kind == Launch::GSUM && L.copy_n > 0);
                                  }),
                   P.launches.end());
  return true;
}

// Dependencies of the pieces of launches [first, last) run as the phases of one
// persistent launch.  Coefficient chunks are the output rows [row0, row0 + nrows)
// of the MODE_VEC / MODE_VEC_ADD chunks of the run; a chunk's version counts the
// phases that have emitted it.  Each piece waits for the chunk holding its
// multipliers at the version reached before its phase, and for its own chunk
// at its current version (read-modify-write, or ordered overwrite).  Returns
// false (run stays per launch) if a multiplier run straddles chunks, or a
// chunk is written after a phase that reads it (a reader could see the later
// value).  deps is sized to the pieces and filled for the run's pieces.
bool seq_dependencies(const Program& P, size_t first, size_t last, std::vector<SeqDep>& deps, int& nchunks) {
  const auto& Ls = P.launches;
  const auto& pd = P.pdesc[SEQ_SHAPE];
  auto hdr = [&](int64_t i, int32_t& row0, int& nrows) {
    const uint8_t* h = P.pk.pay.data() + (size_t)pd[i].off16 * 16;
    std::memcpy(&row0, h, 4);
    uint16_t nr;
    std::memcpy(&nr, h + 4, 2);
    nrows = nr;
  };
  std::map<int32_t, std::pair<int, int>> chunk;   // row0 -> (id, nrows)
  for (size_t k = first; k < last; ++k) {
    if (Ls[k].mode == MODE_Y) continue;
    for (int64_t i = Ls[k].off; i < Ls[k].off + Ls[k].n; ++i) {
      int32_t r0;
      int nr;
      hdr(i, r0, nr);
      if (!chunk.count(r0)) chunk[r0] = {(int)chunk.size(), nr};
    }
  }
  nchunks = (int)chunk.size();
  std::vector<int> ver(nchunks, 0), last_read(nchunks, -1);
  auto find = [&](int64_t m0, int64_t nc) -> int {   // chunk holding [m0, m0 + nc), -1 none, -2 straddles
    auto it = chunk.upper_bound((int32_t)m0);
    if (it != chunk.begin()) {
      --it;
      if (m0 < (int64_t)it->first + it->second.second)
        return m0 + nc <= (int64_t)it->first + it->second.second ? it->second.first : -2;
    }
    auto nx = chunk.lower_bound((int32_t)m0);
    return (nx != chunk.end() && nx->first < m0 + nc) ? -2 : -1;
  };
  if (deps.size() < (size_t)P.npieces) deps.resize((size_t)P.npieces, SeqDep{-1, 0, -1, 0});
  for (size_t k = first; k < last; ++k) {
    const Launch& L = Ls[k];
    std::vector<int> wrote;
    for (int64_t i = L.off; i < L.off + L.n; ++i) {   // reads of this phase first
      const int nc = (int)(pd[i].bytes_flags >> 24);
      SeqDep d{-1, 0, -1, 0};
      if (nc > 0) {
        const int c = find(pd[i].moff, nc);
        if (c == -2) return false;
        if (c >= 0) {
          if (ver[c] > 0) d = SeqDep{c, ver[c], -1, 0};
          last_read[c] = (int)k;
        }
      }
      deps[(size_t)i] = d;
    }
    for (int64_t i = L.off; i < L.off + L.n; ++i) {   // then its writes
      if (L.mode == MODE_Y) continue;
      int32_t r0;
      int nr;
      hdr(i, r0, nr);
      const int c = chunk[r0].first;
      if (last_read[c] >= 0) return false;   // read as multipliers in this or an earlier phase, now written
      deps[(size_t)i].c1 = c;
      deps[(size_t)i].v1 = ver[c];
      wrote.push_back(c);
    }
    std::sort(wrote.begin(), wrote.end());
    wrote.erase(std::unique(wrote.begin(), wrote.end()), wrote.end());
    for (int c : wrote) ++ver[c];
  }
  return true;
}

// ---------------------------------------------------------------- H-LU triangular solves
// Work list of x = U^-1 L^-1 b (block forward substitution with L, then block
// backward substitution with U, leaf by leaf).  For a leaf c the forward row
// item computes
//   w_c = L_cc^-1 (b_c - sum_{(t, s) in L, t >= c} L_ts|_c z_s)
// where a dense block contributes its rows of c times the solved entries of s,
// and a low-rank block W S X^T contributes W|_c t_b with t_b = S X^T w_s, formed
// by the block's column items once every leaf of s is solved.  The backward
// pass is the same with U, leaves in reverse order, the upper triangle U_cc.
bool build_lu_program(const HostMatrix& Lf, const HostMatrix& Uf, int codec, double eps, int valr,
                      LuProgram& P) {
  P = LuProgram();
  const ClusterTree& ct = Lf.ct;
  const auto lv = leaves_under(ct);
  const std::vector<int>& leaves = lv[0];
  const int64_t nl = (int64_t)leaves.size();
  P.nleaves = nl;
  std::vector<int> leaf_of(ct.cl.size(), -1);
  for (int64_t i = 0; i < nl; ++i) leaf_of[leaves[i]] = (int)i;
  auto first_leaf = [&](int c) { return leaf_of[lv[c].front()]; };
  auto last_leaf = [&](int c) { return leaf_of[lv[c].back()]; };
  const int64_t fwd0 = 0, bwd0 = nl;
  int64_t ncounter = 0;
  for (int f = 0; f < 2; ++f) {
    const HostMatrix& H = f == 0 ? Lf : Uf;
    Program dummy;
    Ctx cx{H, dummy, codec, eps, valr ? 1 : 0, m_eps(eps), 1, {}};
    const int64_t nb = (int64_t)H.blocks.size();
    std::vector<ColSet> csd(nb), csw(nb), csx(nb);
    std::atomic<bool> ok{true};
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < nb; ++b) {
      const BlockLeaf& B = H.blocks[b];
      const int64_t m = ct.cl[B.row].size(), n = ct.cl[B.col].size();
      if (!B.adm) {
        if (!make_direct(cx, H.dn[H.slot[b]].D.data(), m, (int)n, csd[b])) ok = false;
        continue;
      }
      const LowRankBlock& R = H.lr[H.slot[b]];
      if (R.k == 0) continue;
      const auto keys = keys_lowrank(cx, R.s);
      if (!make_cols(cx, R.W.data(), m, R.k, keys, csw[b]) || !make_cols(cx, R.X.data(), n, R.k, keys, csx[b]))
        ok = false;
    }
    if (!ok) return false;
    // per leaf: the blocks whose row cluster contains it; per block: coefficient base and counter
    std::vector<std::vector<int64_t>> rowblocks(nl);
    std::vector<int64_t> cbase(nb, -1), cnt(nb, -1), diag(nl, -1);
    for (int64_t b = 0; b < nb; ++b) {
      const BlockLeaf& B = H.blocks[b];
      if (B.row == B.col) {
        diag[leaf_of[B.row]] = b;
        continue;
      }
      if (B.adm && H.lr[H.slot[b]].k == 0) continue;
      for (int c : lv[B.row]) rowblocks[leaf_of[c]].push_back(b);
      if (B.adm) {
        cbase[b] = P.ncoef;
        P.ncoef += H.lr[H.slot[b]].k;
        cnt[b] = 2 * nl + ncounter++;
      }
      P.bytes_fp64 += 8 * (B.adm ? (ct.cl[B.row].size() + ct.cl[B.col].size()) * H.lr[H.slot[b]].k
                                 : ct.cl[B.row].size() * ct.cl[B.col].size());
    }
    auto put_col = [&](const ColSet& cs, int j, int64_t r0, int64_t R, double scale, int32_t mult, int32_t flags) {
      const int B = cs.B(j);
      const uint64_t off = P.pk.put(cs.col(j) + r0, R, B);
      const uint32_t fw = cs.fw(j);
      P.cols.push_back(LuCol{off, scale, (int32_t)R, mult, class_of(fw), em_of(fw), flags});
    };
    auto add_deps = [&](std::vector<LuDep>& d, int s, int64_t base) {
      for (int c : lv[s]) d.push_back(LuDep{(int32_t)(base + leaf_of[c]), 1});
    };
    // column items of the low-rank blocks whose column cluster ends (forward) or
    // starts (backward) with a given leaf
    std::vector<std::vector<int64_t>> colitems(nl);
    for (int64_t b = 0; b < nb; ++b)
      if (cbase[b] >= 0) colitems[f == 0 ? last_leaf(H.blocks[b].col) : first_leaf(H.blocks[b].col)].push_back(b);
    const int64_t done0 = f == 0 ? fwd0 : bwd0;
    for (int64_t k = 0; k < nl; ++k) {
      const int64_t i = f == 0 ? k : nl - 1 - k;
      const Cluster& c = ct.cl[leaves[i]];
      const int64_t R = c.size();
      if (diag[i] < 0) return false;   // every leaf has its diagonal block
      LuItem it{};
      it.kind = f == 0 ? LU_ROW_L : LU_ROW_U;
      it.r0 = (int32_t)c.start;
      it.nr = (int32_t)R;
      it.c0 = (int32_t)P.cols.size();
      std::vector<LuDep> d;
      if (f == 1) d.push_back(LuDep{(int32_t)(fwd0 + i), 1});   // the forward result of this leaf
      for (int64_t b : rowblocks[i]) {
        const BlockLeaf& B = H.blocks[b];
        const Cluster& t = ct.cl[B.row];
        const Cluster& s = ct.cl[B.col];
        const int64_t r0 = c.start - t.start;
        if (!B.adm) {
          for (int j = 0; j < csd[b].n; ++j)
            put_col(csd[b], j, r0, R, csd[b].scale(0), (int32_t)(s.start + j), 0);
          add_deps(d, B.col, done0);
        } else {
          for (int j = 0; j < csw[b].n; ++j) put_col(csw[b], j, r0, R, 1.0, (int32_t)(cbase[b] + j), LC_COEF);
          d.push_back(LuDep{(int32_t)cnt[b], H.lr[H.slot[b]].k});
        }
      }
      it.c1 = (int32_t)P.cols.size();
      it.tri = (int32_t)P.cols.size();
      const ColSet& dt = csd[diag[i]];
      for (int j = 0; j < dt.n; ++j) put_col(dt, j, 0, R, dt.scale(0), 0, 0);
      std::sort(d.begin(), d.end(), [](const LuDep& a, const LuDep& b) {
        return a.flag != b.flag ? a.flag < b.flag : a.target < b.target;
      });
      d.erase(std::unique(d.begin(), d.end(), [](const LuDep& a, const LuDep& b) { return a.flag == b.flag; }),
              d.end());
      it.d0 = (int32_t)P.deps.size();
      P.deps.insert(P.deps.end(), d.begin(), d.end());
      it.d1 = (int32_t)P.deps.size();
      it.flag = (int32_t)(done0 + i);
      P.items.push_back(it);
      for (int64_t b : colitems[i]) {
        const BlockLeaf& B = H.blocks[b];
        const Cluster& s = ct.cl[B.col];
        const LowRankBlock& Rb = H.lr[H.slot[b]];
        std::vector<LuDep> dc;
        add_deps(dc, B.col, done0);
        for (int j0 = 0; j0 < Rb.k; j0 += 4) {   // a few columns per item: long columns in parallel
          LuItem ci{};
          ci.kind = f == 0 ? LU_COL_L : LU_COL_U;
          ci.r0 = (int32_t)s.start;
          ci.nr = (int32_t)s.size();
          ci.c0 = (int32_t)P.cols.size();
          for (int j = j0; j < std::min(Rb.k, j0 + 4); ++j)
            put_col(csx[b], j, 0, s.size(), Rb.s[j] * csx[b].scale(j) * csw[b].scale(j), (int32_t)(cbase[b] + j), 0);
          ci.c1 = (int32_t)P.cols.size();
          ci.tri = -1;
          ci.d0 = (int32_t)P.deps.size();
          P.deps.insert(P.deps.end(), dc.begin(), dc.end());
          ci.d1 = (int32_t)P.deps.size();
          ci.flag = (int32_t)cnt[b];
          P.items.push_back(ci);
        }
      }
    }
  }
  P.nflags = 2 * nl + ncounter;
  P.pk.align(16);
  P.pk.pay.resize(P.pk.pay.size() + 256, 0);   // 8-code groups of a column's last rows read past its end
  if (P.pk.pay.size() >= (1ull << 40) || P.ncoef >= INT32_MAX || P.cols.size() >= (size_t)INT32_MAX) return false;
  return true;
}

}  // namespace hm
