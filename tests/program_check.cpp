// Host check of the launch program of a compressed matrix: the packed layout
// the product kernels stream, and the FP64 meaning of its launches.  Test code,
// built by tests/test_program_layout.py against the library's host objects; it
// runs no GPU code.
//
// For every launch shape of the program it checks
//  * copy descriptors: 16-byte aligned, inside the payload, at most one stage,
//    and of the size their inline header describes;
//  * every vector index a launch reads or writes (inputs and their 16-byte
//    padded copies, multipliers, outputs, partials, fix-up slots, fan-out
//    slots) inside the buffer the library allocates for it;
//  * warp ranges in order and covering their launch;
//  * within one launch, no vector entry both read as a multiplier or input and
//    written as an output (the launch's warps run concurrently);
//  * each launch's algorithmic byte count (the roofline numerator) equal to the
//    count from its units' headers by the per-unit definition;
//  * in the FP32 tier, every decoded value equal to the sum of the BF16 limbs
//    the multi-RHS path keeps for its piece (the `limbs` header field);
// then it replays the launches in program order in FP64 (Alg. 8: each code
// decoded, then Alg. 1 / 4-7 as the program orders them).  The replay must give
// the same y bit for bit on a second pass (no state left between products), and
// its distance from the FP64 product of the matrix as the host stores it (H
// blocks, or bases and couplings) is printed.  The runs of row-chunk launches
// the library fuses into one persistent launch are also replayed as dataflow:
// warps that step in random order, each piece waiting for the chunk versions
// of its dependencies.  No such order may stall with work left (a hang on the
// device) or change y by a single bit (a race).
//
// usage: program_check <points+x file> n format eps codec leaf nsm adm kernel [adjoint]
//   file: n*3 doubles (points, row-major) then n doubles (x, original order)
//   format 0 H, 1 UH, 2 H2, 3 UH with separate couplings; codec 0 none,
//   1 AFLP, 2 FPX; adm 0 standard, 1 HODLR, 2 BLR; kernel 0 Laplace, 1 Matern
//   adjoint 1: the program of the transposed matrix (transpose_host, as the
//   adjoint product runs it), compared with M^T x from the original's blocks
// prints one line per shape and "ok" or "FAILED <count>"; exit status 0 iff ok.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "program.h"

using namespace hm;

namespace {

int g_fails = 0;

#define CHECK(cond, ...)                                  \
  do {                                                    \
    if (!(cond)) {                                        \
      if (g_fails < 20) {                                 \
        std::printf("FAIL line %d: ", __LINE__);          \
        std::printf(__VA_ARGS__);                         \
        std::printf("\n");                                \
      }                                                   \
      ++g_fails;                                          \
    }                                                     \
  } while (0)

// Value of one code given the 16-bit format B | fmt << 4 | e << 6 | m << 10
// (fmt 0 FPX e8, 1 FPX e11, 2 AFLP as (s - 1) with s = 2^f (1 + mant 2^-m),
// its vmin applied by the scale the program attaches, 3 raw FP64).
double decode(uint64_t code, uint16_t f16) {
  const int B = f16 & 15, fmt = (f16 >> 4) & 3, e = (f16 >> 6) & 15, m = f16 >> 10;
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
  const double v = f ? std::ldexp(1.0 + std::ldexp((double)mant, -m), (int)f) - 1.0 : 0.0;
  return sign ? -v : v;
}

uint64_t load_code(const uint8_t* p, int B) {
  uint64_t c = 0;
  for (int b = 0; b < B; ++b) c |= (uint64_t)p[b] << (8 * b);
  return c;
}

uint16_t format16(int B, int fmt, uint16_t em) {
  return (uint16_t)(B | (fmt << 4) | ((em & 0xff) << 6) | ((em >> 8) << 10));
}

double ff(const F2& v) { return (double)v.hi + (double)v.lo; }

// Cut an FP32 value to BF16 (its top 16 bits), as its FP32 value.
float bf16_cut(float a) {
  uint32_t b;
  std::memcpy(&b, &a, 4);
  b &= 0xffff0000u;
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

// The multi-RHS kernels split each decoded value a (FP32) into BF16 limbs by
// truncation, a = l0 + l1 + l2 with l0 = cut(a), l1 = cut(a - l0),
// l2 = cut(a - l0 - l1) (the differences are exact), and multiply only the
// first `limbs` of them: true if those are exactly a.  Three limbs hold every
// FP32 value; a piece that keeps fewer must hold values of at most 8 * limbs
// significant bits, exact in FP32.
bool limbs_exact(double v, int limbs) {
  if (limbs >= 3) return true;
  const float a = (float)v;
  if ((double)a != v) return false;
  const float l0 = bf16_cut(a), r1 = a - l0, l1 = bf16_cut(r1), r2 = r1 - l1, l2 = bf16_cut(r2);
  const double sum = limbs == 1 ? (double)l0 : limbs == 2 ? (double)l0 + l1 : ((double)l0 + l1) + l2;
  return sum == v;
}

// Entries of a 16-byte aligned copy of `count` 8-byte entries starting at i.
int64_t padded_entries(int64_t i, int64_t count) { return ((i - (i & ~1LL) + count) * 8 + 15) / 16 * 2; }

struct Replay {
  const HostMatrix& H;
  const Program& P;
  int shape;
  double alpha;
  int64_t NV;                 // vector entries allocated (nvec + 16)
  int64_t nfix;               // fix-up slots of this shape
  int persistent_runs = 0;    // runs replayed as one persistent launch
  std::vector<double> v, part, fix, y;
  std::vector<int> cnt;

  Replay(const HostMatrix& h, const Program& p, int cf, double a)
      : H(h), P(p), shape(cf), alpha(a), NV(p.nvec + 16), nfix(cf == MR_SHAPE ? p.nfix_mr : p.nfix) {
    v.assign(P.nvec, NAN);
    part.assign(std::max<int64_t>(P.npartial, 1), NAN);
    fix.assign((size_t)std::max<int64_t>(nfix, 1) * CHUNK_ROWS, NAN);
    cnt.assign(P.splits.size(), 0);
  }

  void ranges(const Launch& L) {
    const int nw = L.nw[shape];
    if (nw == 0) return;
    CHECK(L.woff[shape] + nw < (int64_t)P.wbeg.size(), "range list past its end");
    const int32_t* wb = P.wbeg.data() + L.woff[shape];
    CHECK(wb[0] == L.off && wb[nw] == L.off + L.n, "ranges do not cover the launch");
    for (int w = 0; w < nw; ++w) CHECK(wb[w] <= wb[w + 1], "ranges out of order");
  }

  void column_dots(const Launch& L, std::vector<char>& read, std::vector<char>& written) {
    const auto& pay = P.pk.pay;
    for (int64_t it = L.off; it < L.off + L.n; ++it) {
      const ItemCopy& c = P.items[it];
      const uint64_t off = (uint64_t)c.off16 * 16;
      CHECK(off + ((c.bytes + 15) & ~15u) <= pay.size(), "item %ld outside the payload", (long)it);
      CHECK(c.bytes <= (uint32_t)STAGE_BYTES, "item %ld larger than a stage", (long)it);
      if (off + 16 > pay.size()) continue;
      CPieceHdr h;
      std::memcpy(&h, &pay[off], sizeof h);
      CHECK(h.vin == c.vin && h.nrows == c.nrows, "item %ld: descriptor and header differ", (long)it);
      CHECK(h.nrows >= 1 && h.nrows <= SEG_ROWS && h.ncols >= 1 && h.ncols <= CPIECE_MAX_COLS,
            "item %ld: header out of range", (long)it);
      const int64_t x0 = c.vin & ~1;
      CHECK(x0 >= 0 && x0 + padded_entries(c.vin, c.nrows) <= NV, "item %ld: input copy outside v", (long)it);
      CHECK(padded_entries(c.vin, c.nrows) * 8 <= SEG_ROWS * 8 + 16, "item %ld: input copy too long", (long)it);
      const bool final = h.flags & ITEM_FINAL;
      const int B = h.fb & 15, fmt = (h.fb >> 4) & 3;
      const size_t rows16 = (h.nrows + 15) & ~15, stride = rows16 * B;
      const size_t cb = off + 16 + (final ? 16 : 8) * (size_t)h.ncols;
      CHECK(cb + stride * h.ncols - off == c.bytes, "item %ld: %zu bytes described, %u copied", (long)it,
            cb + stride * h.ncols - off, c.bytes);
      if (cb + stride * h.ncols > pay.size()) continue;
      for (int64_t r = 0; r < h.nrows; ++r)
        if (h.vin + r >= 0 && h.vin + r < P.nvec) read[h.vin + r] = 1;
      const CColMeta* cm = reinterpret_cast<const CColMeta*>(&pay[off + 16]);
      const F2* sc = reinterpret_cast<const F2*>(&pay[off + 16 + 8 * (size_t)h.ncols]);
      for (int j = 0; j < h.ncols; ++j) {
        const uint16_t f16 = format16(B, fmt, cm[j].em);
        double s = 0;
        for (size_t r = 0; r < rows16; ++r) {
          const double d = decode(load_code(&pay[cb + j * stride + r * B], B), f16);
          if (r >= (size_t)h.nrows)
            CHECK(d == 0.0, "item %ld: padding row not zero", (long)it);
          else
            s += d * v[h.vin + r];
          if (P.tier == TIER_F32)
            CHECK(limbs_exact(d, h.limbs), "item %ld: a value needs more than %d BF16 limbs", (long)it, h.limbs);
        }
        if (final) {
          CHECK(cm[j].out >= 0 && cm[j].out < P.nvec, "item %ld: output outside v", (long)it);
          if (cm[j].out < 0 || cm[j].out >= P.nvec) continue;
          s *= ff(sc[j]);
          if (h.flags & ITEM_ALPHA) s *= alpha;
          v[cm[j].out] = s;
          written[cm[j].out] = 1;
        } else {
          CHECK(cm[j].out >= 0 && cm[j].out < P.npartial, "item %ld: partial outside its array", (long)it);
          if (cm[j].out >= 0 && cm[j].out < P.npartial) part[cm[j].out] = s;
        }
      }
    }
  }

  void segment_sums(const Launch& L) {
    for (int64_t i = L.off; i < L.off + L.n; ++i) {
      const GsumOut& o = P.gouts[i];
      double s = 0;
      for (int p = o.p0; p < o.p1; ++p) {
        CHECK(p >= 0 && p < P.npartial, "segment sum %ld: partial outside its array", (long)i);
        if (p < 0 || p >= P.npartial) continue;
        CHECK(!std::isnan(part[p]), "segment sum %ld: partial %d never written", (long)i, p);
        double w = 1.0;
        if (o.flags & 2) {
          const int64_t q = o.ps + (p - o.p0);
          CHECK(q >= 0 && q < (int64_t)P.pscale.size(), "segment sum %ld: weight outside its array", (long)i);
          if (q >= 0 && q < (int64_t)P.pscale.size()) w = ff(P.pscale[q]);
        }
        s += part[p] * w;
      }
      s *= ff(o.scale);
      if (o.flags & 1) s *= alpha;
      CHECK(o.out >= 0 && o.out < P.nvec, "segment sum %ld: output outside v", (long)i);
      if (o.out >= 0 && o.out < P.nvec) v[o.out] = s;
      if (L.scatter) {   // a folded fan-out: the output's own slots
        const int64_t a = o.pad, b = (int64_t)o.pad + (o.flags >> 8);
        CHECK(a >= 0 && b <= (int64_t)P.fan_dst.size(), "segment sum %ld: slot list outside", (long)i);
        for (int64_t q = a; q < b && q < (int64_t)P.fan_dst.size(); ++q) {
          const int32_t d = P.fan_dst[q];
          CHECK(d >= P.fan_base && d < P.nvec && P.fan_src[d - P.fan_base] == o.out, "segment sum %ld: slot %d",
                (long)i, d);
          if (d >= P.fan_base && d < P.nvec) v[d] = s;
        }
      }
    }
    if (L.scatter)   // and the copy entries of the one-segment column-dot outputs
      for (int64_t i = L.copy_off; i < L.copy_off + L.copy_n; ++i) {
        CHECK(i >= 0 && i < (int64_t)P.fan_copy_src.size(), "copy entry %ld outside its list", (long)i);
        if (i < 0 || i >= (int64_t)P.fan_copy_src.size()) break;
        const int32_t c = P.fan_copy_src[i], d = P.fan_copy_dst[i];
        CHECK(c >= 0 && c < P.fan_base && d >= P.fan_base && d < P.nvec && P.fan_src[d - P.fan_base] == c,
              "copy entry %ld: %d -> %d", (long)i, c, d);
        if (c >= 0 && c < P.fan_base && d >= P.fan_base && d < P.nvec) v[d] = v[c];
      }
    std::fill(part.begin(), part.end(), NAN);   // partials are consumed by the launch
  }

  void fan_out(const Launch& L) {
    CHECK(L.off >= 0 && L.off + L.n <= (int64_t)P.fan_src.size(), "fan-out range outside its list");
    for (int64_t i = L.off; i < L.off + L.n && i < (int64_t)P.fan_src.size(); ++i) {
      const int32_t s = P.fan_src[i];
      CHECK(s >= 0 && s < P.fan_base, "fan-out %ld reads outside the coefficients", (long)i);
      CHECK(P.fan_base + i < P.nvec, "fan-out slot %ld outside v", (long)i);
      if (s >= 0 && s < P.fan_base && P.fan_base + i < P.nvec) v[P.fan_base + i] = v[s];
    }
  }

  void row_chunks(const Launch& L, std::vector<char>& read, std::vector<char>& written) {
    CHECK((int64_t)P.pdesc[shape].size() == P.npieces, "descriptor list size");
    const int nw = L.nw[shape];
    const int32_t* wb = P.wbeg.data() + L.woff[shape];
    std::vector<double> acc(CHUNK_ROWS, 0.0);
    for (int w = 0; w < nw; ++w)
      for (int32_t pi = wb[w]; pi < wb[w + 1]; ++pi) piece(L, pi, acc, read, written);
  }

  // One row-chunk piece: its multipliers are read from v now (as a warp copies
  // them when the piece starts); its last piece of a part emits.  Returns true
  // if the piece emitted its chunk (a shared chunk: only its last part).
  bool piece(const Launch& L, int32_t pi, std::vector<double>& acc, std::vector<char>& read,
             std::vector<char>& written) {
    const auto& pay = P.pk.pay;
    const PieceCopy& c = P.pdesc[shape][pi];
    const uint64_t off = (uint64_t)c.off16 * 16;
    const uint32_t bytes = c.bytes_flags & 0xffff, rflags = (c.bytes_flags >> 16) & 0xff, ncols = c.bytes_flags >> 24;
    CHECK(off + ((bytes + 15) & ~15u) <= pay.size(), "piece %d outside the payload", pi);
    CHECK(bytes <= (uint32_t)STAGE_BYTES, "piece %d larger than a stage", pi);
    if (off + sizeof(PieceHdr) > pay.size()) return false;
    PieceHdr h;
    std::memcpy(&h, &pay[off], sizeof h);
    const int B = h.fb & 15, fmt = (h.fb >> 4) & 3;
    // (a piece without columns only emits its chunk: e.g. coefficients that
    // receive nothing at one level of the H2 down-sweep)
    CHECK(h.nrows >= 1 && h.nrows <= CHUNK_ROWS && h.ncols <= PIECE_MAX_COLS, "piece %d: header out of range", pi);
    CHECK(ncols == h.ncols, "piece %d: descriptor and header differ", pi);
    const bool tile = h.flags & PH_TILE;
    if (tile) CHECK(c.moff == h.vin0, "piece %d: tile multipliers differ", pi);
    CHECK(c.moff >= 0 && c.moff + h.ncols <= P.nvec, "piece %d: multipliers outside v", pi);
    CHECK((c.moff & ~1) + padded_entries(c.moff, h.ncols) <= NV, "piece %d: multiplier copy outside v", pi);
    CHECK(padded_entries(c.moff, h.ncols) * 8 <= PIECE_MAX_COLS * 8 + 16, "piece %d: multiplier copy too long", pi);
    const size_t stride = ((size_t)h.nrows * B + 7) & ~(size_t)7;
    const size_t cb = off + 40 + (tile ? 0 : ((2 * (size_t)h.ncols + 7) & ~(size_t)7));
    CHECK(cb + stride * h.ncols - off == bytes, "piece %d: %zu bytes described, %u copied", pi,
          cb + stride * h.ncols - off, bytes);
    if (cb + stride * h.ncols > pay.size() || c.moff < 0 || c.moff + h.ncols > P.nvec) return false;
    if (rflags & PD_FIRST) std::fill(acc.begin(), acc.end(), 0.0);
    const uint16_t* em = reinterpret_cast<const uint16_t*>(&pay[off + 40]);
    for (int j = 0; j < h.ncols; ++j) {
      const int32_t vi = c.moff + j;
      read[vi] = 1;
      const uint16_t f16 = format16(B, fmt, tile ? h.em : em[j]);
      double mult = v[vi];
      if (tile) {
        mult *= ff(h.scale);
        if (h.flags & PH_TALPHA) mult *= alpha;
      }
      for (int r = 0; r < h.nrows; ++r) {
        const double d = decode(load_code(&pay[cb + j * stride + (size_t)r * B], B), f16);
        if (P.tier == TIER_F32)
          CHECK(limbs_exact(d, h.limbs), "piece %d: a value needs more than %d BF16 limbs", pi, h.limbs);
        acc[r] += d * mult;
      }
    }
    return (rflags & PD_LAST) ? emit(L, h, c, acc, written, pi) : false;
  }

  bool emit(const Launch& L, const PieceHdr& h, const PieceCopy& c, const std::vector<double>& acc,
            std::vector<char>& written, int pi) {
    std::vector<double> out(acc.begin(), acc.begin() + h.nrows);
    if ((c.bytes_flags >> 16) & PD_SPLIT) {
      const int split = c.split_part >> 8, pidx = c.split_part & 0xff;
      CHECK(split >= 0 && split < (int)P.splits.size(), "piece %d: split outside its list", pi);
      if (split < 0 || split >= (int)P.splits.size()) return false;
      const Split& sp = P.splits[split];
      CHECK(sp.nparts >= 2 && sp.nparts <= 256 && pidx < sp.nparts, "piece %d: part outside its split", pi);
      CHECK(sp.slot0 >= 0 && sp.slot0 + sp.nparts <= nfix, "piece %d: fix-up slots outside their array", pi);
      if (pidx >= sp.nparts || sp.slot0 < 0 || sp.slot0 + sp.nparts > nfix) return false;
      for (int r = 0; r < h.nrows; ++r) fix[(size_t)(sp.slot0 + pidx) * CHUNK_ROWS + r] = acc[r];
      if (++cnt[split] != sp.nparts) return false;
      cnt[split] = 0;   // the last part resets the counter for the next product
      for (int r = 0; r < h.nrows; ++r) {
        double s = 0;
        for (int k = 0; k < sp.nparts; ++k) s += fix[(size_t)(sp.slot0 + k) * CHUNK_ROWS + r];
        out[r] = s;
      }
    }
    for (int r = 0; r < h.nrows; ++r) {
      const int64_t g = h.row0 + r;
      if (L.mode == MODE_Y) {
        CHECK(g >= 0 && g < H.n, "piece %d: row outside y", pi);
        if (g >= 0 && g < H.n) y[H.ct.perm[g]] = out[r];
        continue;
      }
      CHECK(g >= 0 && g < P.nvec, "piece %d: coefficient outside v", pi);
      if (g < 0 || g >= P.nvec) continue;
      double val = out[r];
      if (L.mode == MODE_VEC_ADD) val += v[g];
      if (L.use_rowscale) val *= P.rowscale[g];
      if (h.flags & PH_CALPHA) val *= alpha;
      v[g] = val;
      written[g] = 1;
    }
    return true;
  }

  // Row-chunk launches [first, last) as the phases of one persistent launch:
  // nwarps warps take the ranges of each phase in order (a warp without a range
  // claims the next one, moving to the next phase when a phase has none left)
  // and run them piece by piece.  A piece starts only when the chunk versions of
  // its SeqDep are reached; an emit of a chunk raises its version.  The warp that
  // steps next is drawn at random among those that can.  Work left with no warp
  // able to step would be a hang of the launch.
  void dataflow(size_t first, size_t last, const std::vector<SeqDep>& deps, int nchunks, int nwarps,
                std::mt19937& rng) {
    struct Warp {
      size_t phase = 0;
      int32_t next = 0, end = 0;
      bool done = false;
      std::vector<double> acc = std::vector<double>(CHUNK_ROWS, 0.0);
    };
    const size_t nph = last - first;
    std::vector<int> ver(nchunks, 0), claim(nph, 0);
    std::vector<Warp> warps(nwarps);
    std::vector<char> read(P.nvec, 0), written(P.nvec, 0);   // phases read what earlier phases wrote
    auto ready = [&](int32_t i) {
      const SeqDep& d = deps[i];
      return (d.c0 < 0 || ver[d.c0] >= d.v0) && (d.c1 < 0 || ver[d.c1] >= d.v1);
    };
    for (;;) {
      std::vector<int> can;
      bool left = false;
      for (int w = 0; w < nwarps; ++w) {
        Warp& a = warps[w];
        while (!a.done && a.next == a.end) {
          if (a.phase == nph) {
            a.done = true;
            break;
          }
          const Launch& L = P.launches[first + a.phase];
          const int r = claim[a.phase]++;
          if (r >= L.nw[shape]) {
            ++a.phase;
            continue;
          }
          const int32_t* wb = P.wbeg.data() + L.woff[shape];
          a.next = wb[r];
          a.end = wb[r + 1];
        }
        if (a.done) continue;
        left = true;
        if (ready(a.next)) can.push_back(w);
      }
      if (!left) break;
      CHECK(!can.empty(), "persistent run from launch %zu: work left and no warp can step", first);
      if (can.empty()) return;
      Warp& a = warps[can[rng() % can.size()]];
      const int32_t i = a.next++;
      if (piece(P.launches[first + a.phase], i, a.acc, read, written) && deps[i].c1 >= 0) ++ver[deps[i].c1];
    }
  }

  // Algorithmic bytes of a launch, counted from its units' inline headers by the
  // per-unit definition the benchmark's roofline uses: gather and fan-out 20 per
  // entry (index, value read, value write); a column-dot piece rows * B per column
  // + 16 (header) + 16 per column (metadata, output) + 8 per column (scale, one-
  // segment sets) + 8 * rows (input segment) + 16 (descriptor); a segment sum 8
  // per partial (16 with weights) + 40; a row-chunk piece rows * B per column + 40
  // (header) + 10 per column (8 for tiles: decode parameters, multiplier) + 16
  // (descriptor), and at a chunk's last piece per row 20 (y) or 8 / 16 (plain /
  // accumulated coefficients) + 8 with row scales.
  int64_t alg_bytes(const Launch& L) const {
    const auto& pay = P.pk.pay;
    int64_t b = 0;
    switch (L.kind) {
      case Launch::GATHER:
      case Launch::FANOUT:
        return L.n * 20;
      case Launch::GSUM:
        for (int64_t i = L.off; i < L.off + L.n; ++i) {
          const GsumOut& o = P.gouts[i];
          b += (int64_t)(o.p1 - o.p0) * ((o.flags & 2) ? 16 : 8) + 40;
          if (L.scatter) b += 12 * (int64_t)(o.flags >> 8);   // slot index, value written
        }
        if (L.scatter) b += 24 * L.copy_n;                      // indices, value read and written
        return b;
      case Launch::CDOT:
        for (int64_t it = L.off; it < L.off + L.n; ++it) {
          CPieceHdr h;
          std::memcpy(&h, &pay[(uint64_t)P.items[it].off16 * 16], sizeof h);
          const int64_t R = h.nrows, nc = h.ncols, B = h.fb & 15;
          b += R * B * nc + 16 + 16 * nc + ((h.flags & ITEM_FINAL) ? 8 * nc : 0) + 8 * R + 16;
        }
        return b;
      case Launch::RGEMV:
        for (int64_t i = L.off; i < L.off + L.n; ++i) {
          PieceHdr h, nx{};
          std::memcpy(&h, &pay[(uint64_t)P.pdesc[0][i].off16 * 16], sizeof h);
          if (i + 1 < L.off + L.n) std::memcpy(&nx, &pay[(uint64_t)P.pdesc[0][i + 1].off16 * 16], sizeof nx);
          const int64_t R = h.nrows, nc = h.ncols, B = h.fb & 15;
          b += R * B * nc + 40 + ((h.flags & PH_TILE) ? 8 : 10) * nc + 16;
          if (i + 1 == L.off + L.n || nx.row0 != h.row0)
            b += R * (L.mode == MODE_Y ? 20 : (L.mode == MODE_VEC_ADD ? 16 : 8) + (L.use_rowscale ? 8 : 0));
        }
        return b;
    }
    return -1;
  }

  // One product.  nwarps > 0: runs of row-chunk launches that the library fuses
  // into one persistent launch (SEQ_SHAPE) go through `dataflow`.
  void run(const std::vector<double>& x, int nwarps = 0, uint32_t seed = 1) {
    y.assign(H.n, NAN);
    std::mt19937 rng(seed);
    for (size_t li = 0; li < P.launches.size(); ++li) {
      const Launch& L = P.launches[li];
      if (nwarps > 0 && shape == SEQ_SHAPE && L.kind == Launch::RGEMV) {
        size_t j = li;
        while (j < P.launches.size() && P.launches[j].kind == Launch::RGEMV) ++j;
        std::vector<SeqDep> deps;
        int nchunks = 0;
        if (j - li >= 2 && seq_dependencies(P, li, j, deps, nchunks)) {
          for (size_t k = li; k < j; ++k) ranges(P.launches[k]);
          dataflow(li, j, deps, nchunks, nwarps, rng);
          ++persistent_runs;
          li = j - 1;
          continue;
        }
      }
      std::vector<char> read(P.nvec, 0), written(P.nvec, 0);
      switch (L.kind) {
        case Launch::GATHER:
          for (int64_t i = 0; i < H.n; ++i) v[i] = x[H.ct.perm[i]];
          break;
        case Launch::FANOUT:
          fan_out(L);
          break;
        case Launch::GSUM:
          segment_sums(L);
          break;
        case Launch::CDOT:
          ranges(L);
          column_dots(L, read, written);
          break;
        case Launch::RGEMV:
          ranges(L);
          row_chunks(L, read, written);
          break;
      }
      int64_t both = 0;
      for (int64_t i = 0; i < P.nvec; ++i) both += read[i] && written[i];
      CHECK(both == 0, "a launch reads and writes %ld vector entries", (long)both);
    }
    for (size_t s = 0; s < cnt.size(); ++s) CHECK(cnt[s] == 0, "split %zu: counter left at %d", s, cnt[s]);
  }
};

// Explicit basis of cluster c (n_c x k_c, column-major): stored for UH and for
// H2 leaves; an inner H2 cluster stacks its sons' bases times their transfer
// matrices (rows of son s: W_s E_s, E_s of size k_s x k_c).
std::vector<double> explicit_basis(const HostMatrix& H, const Bases& b, int c) {
  const Cluster& cl = H.ct.cl[c];
  if (H.prm.format != HM_FMT_H2 || cl.leaf()) return b.B[c];
  const int64_t nc = cl.end - cl.start;
  const int kc = b.k[c];
  std::vector<double> w((size_t)nc * kc, 0.0);
  for (int q = 0; q < cl.nsons; ++q) {
    const int s = cl.son[q];
    const Cluster& sc = H.ct.cl[s];
    const int64_t ns = sc.end - sc.start, r0 = sc.start - cl.start;
    const int ks = b.k[s];
    const std::vector<double> ws = explicit_basis(H, b, s);
    for (int j = 0; j < kc; ++j)
      for (int l = 0; l < ks; ++l) {
        const double e = b.E[s][l + (size_t)j * ks];
        for (int64_t i = 0; i < ns; ++i) w[(r0 + i) + (size_t)j * nc] += ws[i + (size_t)l * ns] * e;
      }
  }
  return w;
}

// alpha * M x (transpose: alpha * M^T x) in FP64, original order, for the matrix
// as the host stores it in its format: H blocks W diag(s) X^T; UH and H2 blocks
// W_t S X_s^T with the coupling S (separate couplings: S = Sr Sc^T); dense
// blocks D.  Each block maps its input cluster to its output cluster.
std::vector<double> host_product(const HostMatrix& H, const std::vector<double>& x, double alpha, bool transpose) {
  const int format = H.prm.format;
  std::vector<std::vector<double>> wb(H.ct.cl.size()), xb(H.ct.cl.size());
  if (format != HM_FMT_H)
    for (size_t c = 0; c < H.ct.cl.size(); ++c) {
      wb[c] = explicit_basis(H, H.rowb, (int)c);
      xb[c] = explicit_basis(H, H.colb, (int)c);
    }
  // column-major a (m x k) times v: a v, or a^T v
  auto apply = [](const std::vector<double>& a, int64_t m, int64_t k, const std::vector<double>& in, bool tr) {
    std::vector<double> out(tr ? k : m, 0.0);
    for (int64_t j = 0; j < k; ++j)
      for (int64_t i = 0; i < m; ++i) {
        if (tr)
          out[j] += a[i + (size_t)j * m] * in[i];
        else
          out[i] += a[i + (size_t)j * m] * in[j];
      }
    return out;
  };
  std::vector<double> y(H.n, 0.0);
  for (size_t b = 0; b < H.blocks.size(); ++b) {
    const BlockLeaf& bl = H.blocks[b];
    const Cluster& t = H.ct.cl[bl.row];
    const Cluster& s = H.ct.cl[bl.col];
    const int64_t nt = t.end - t.start, ns = s.end - s.start;
    const Cluster& in = transpose ? t : s;
    const Cluster& out = transpose ? s : t;
    std::vector<double> xi(in.end - in.start), yo;
    for (int64_t j = 0; j < (int64_t)xi.size(); ++j) xi[j] = x[H.ct.perm[in.start + j]];
    if (!bl.adm) {
      yo = apply(H.dn[H.slot[b]].D, nt, ns, xi, transpose);
    } else if (format == HM_FMT_H) {
      const LowRankBlock& L = H.lr[H.slot[b]];
      // W diag(s) X^T x, or X diag(s) W^T x
      std::vector<double> c = transpose ? apply(L.W, nt, L.k, xi, true) : apply(L.X, ns, L.k, xi, true);
      for (int k = 0; k < L.k; ++k) c[k] *= L.s[k];
      yo = transpose ? apply(L.X, ns, L.k, c, false) : apply(L.W, nt, L.k, c, false);
    } else {
      const int kt = H.rowb.k[bl.row], ks = H.colb.k[bl.col];
      std::vector<double> c = transpose ? apply(wb[bl.row], nt, kt, xi, true) : apply(xb[bl.col], ns, ks, xi, true);
      if (format == HM_FMT_UH_SEP) {   // S = R C with R (kt x kb), C (kb x ks)
        const auto& R = H.coupling_r[H.slot[b]];
        const auto& C = H.coupling_ct[H.slot[b]];
        const int kb = H.lr[H.slot[b]].k;
        c = transpose ? apply(C, kb, ks, apply(R, kt, kb, c, true), true)
                      : apply(R, kt, kb, apply(C, kb, ks, c, false), false);
      } else {
        c = apply(H.coupling[H.slot[b]], kt, ks, c, transpose);
      }
      yo = transpose ? apply(xb[bl.col], ns, ks, c, false) : apply(wb[bl.row], nt, kt, c, false);
    }
    for (int64_t i = 0; i < (int64_t)yo.size(); ++i) y[H.ct.perm[out.start + i]] += alpha * yo[i];
  }
  return y;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 10 && argc != 11) {
    std::fprintf(stderr, "usage: %s file n format eps codec leaf nsm adm kernel [adjoint]\n", argv[0]);
    return 2;
  }
  const bool adjoint = argc == 11 && std::atoi(argv[10]) != 0;
  const int64_t n = std::atoll(argv[2]);
  const int format = std::atoi(argv[3]), codec = std::atoi(argv[5]), leaf = std::atoi(argv[6]),
            nsm = std::atoi(argv[7]), adm = std::atoi(argv[8]), kernel = std::atoi(argv[9]);
  const double eps = std::atof(argv[4]);
  std::vector<double> pts(3 * n), x(n);
  FILE* f = std::fopen(argv[1], "rb");
  if (!f || std::fread(pts.data(), 8, 3 * n, f) != (size_t)(3 * n) || std::fread(x.data(), 8, n, f) != (size_t)n) {
    std::fprintf(stderr, "cannot read %s\n", argv[1]);
    return 2;
  }
  std::fclose(f);

  HostMatrix H;
  H.prm.kernel = (hm_kernel)kernel;
  H.prm.leaf_size = leaf;
  H.prm.eta = 2.0;
  H.prm.format = (hm_format)format;
  H.prm.eps_build = eps;
  H.prm.adm = (hm_adm)adm;
  H.n = n;
  H.kparam = kernel == HM_KERNEL_LAPLACE ? std::sqrt(4.0 * M_PI / (double)n) : 0.1;
  H.pts = pts;
  build_cluster_tree(H.pts.data(), n, leaf, H.ct);
  build_block_tree(H.ct, 2.0, H.blocks, adm);
  build_lowrank_blocks(H, 8);
  if (format == HM_FMT_UH || format == HM_FMT_UH_SEP) build_uniform_bases(H, 8);
  if (format == HM_FMT_H2) build_nested_bases(H, 8);
  HostMatrix T;   // adjoint: the program of the transposed matrix, as hm_matvec_adjoint runs it
  if (adjoint) transpose_host(H, T);
  const HostMatrix& M = adjoint ? T : H;
  Program P;
  if (!build_program(M, codec, eps, 1, nsm, P)) {
    std::printf("build_program failed\n");
    return 1;
  }
  const double alpha = 0.75;
  const std::vector<double> yref = host_product(H, x, alpha, adjoint);
  double den = 0;
  for (double t : yref) den += t * t;
  for (int cf = 0; cf < NSHAPES; ++cf) {
    Replay R(M, P, cf, alpha);
    if (cf == 0) {   // the launches' algorithmic byte counts (shape independent)
      int64_t tot = 0;
      for (size_t li = 0; li < P.launches.size(); ++li) {
        const int64_t a = R.alg_bytes(P.launches[li]);
        CHECK(a == P.launches[li].bytes, "launch %zu: %ld algorithmic bytes counted, %ld recorded", li, (long)a,
              (long)P.launches[li].bytes);
        static const char* kinds[] = {"gather", "cdot", "gsum", "rgemv", "fanout"};
        std::printf("launch %zu %s units %ld algorithmic bytes %ld\n", li, kinds[P.launches[li].kind],
                    (long)P.launches[li].n, (long)a);
        tot += a;
      }
      std::printf("algorithmic bytes %ld\n", (long)tot);
    }
    R.run(x);
    const std::vector<double> first = R.y;
    R.run(x);
    double num = 0;
    int64_t differ = 0;
    for (int64_t i = 0; i < n; ++i) {
      differ += !(R.y[i] == first[i]);
      num += (R.y[i] - yref[i]) * (R.y[i] - yref[i]);
    }
    CHECK(differ == 0, "shape %d: second product differs in %ld entries", cf, (long)differ);
    std::printf("shape %d rel_err %.6e\n", cf, std::sqrt(num / den));
    if (cf != SEQ_SHAPE) continue;
    // the persistent launch: any order its waits allow must give the same y
    const int warp_counts[] = {1, 2, 7, 64, 1000};
    for (int nwarps : warp_counts)
      for (uint32_t seed = 1; seed <= 3; ++seed) {
        Replay D(M, P, cf, alpha);
        D.run(x, nwarps, seed);
        int64_t d = 0;
        for (int64_t i = 0; i < n; ++i) d += !(D.y[i] == first[i]);
        CHECK(d == 0, "persistent launch, %d warps, seed %u: %ld entries differ", nwarps, seed, (long)d);
        if (nwarps == 1 && seed == 1) std::printf("persistent runs %d\n", D.persistent_runs);
      }
  }
  if (g_fails) {
    std::printf("FAILED %d\n", g_fails);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
