// Packed layout and launch program of one compressed matrix (host side).
#pragma once

#include <cstdint>
#include <vector>

#include "dev_types.h"
#include "hm_internal.h"

namespace hm {

inline F2 split_ff(double v) {
  const float h = (float)v;
  return F2{h, (float)(v - (double)h)};
}

struct Packer {
  std::vector<uint8_t> pay;       // packed stream: items and pieces, each 16-byte aligned
  int64_t value_bytes = 0;        // sum of n * B over all packed columns (no padding)
  int64_t meta_bytes = 0;         // inline headers, format lists, scales, column metadata

  uint64_t align(int a) {
    while (pay.size() & (uint64_t)(a - 1)) pay.push_back(0);
    return pay.size();
  }
  // append n codes of B bytes (little-endian) at the next 8-byte boundary; returns the offset
  uint64_t put(const uint64_t* codes, int64_t n, int B) {
    uint64_t off = align(8);
    pay.resize(off + (uint64_t)(n * B));
    uint8_t* dst = pay.data() + off;
    for (int64_t i = 0; i < n; ++i) {
      const uint64_t c = codes[i];
      for (int b = 0; b < B; ++b) dst[i * B + b] = (uint8_t)(c >> (8 * b));
    }
    value_bytes += n * B;
    align(8);
    return off;
  }
  // append R codes of B bytes plus R8 - R zero codes (rows padded to R8)
  uint64_t put_rows(const uint64_t* codes, int64_t R, int64_t R8, int B) {
    uint64_t off = align(8);
    pay.resize(off + (uint64_t)(R8 * B), 0);
    uint8_t* dst = pay.data() + off;
    for (int64_t i = 0; i < R; ++i) {
      const uint64_t c = codes[i];
      for (int b = 0; b < B; ++b) dst[i * B + b] = (uint8_t)(c >> (8 * b));
    }
    value_bytes += R * B;
    align(8);
    return off;
  }
  // append raw bytes (metadata) at the next 8-byte boundary
  uint64_t raw(const void* p, size_t n) {
    uint64_t off = align(8);
    const uint8_t* s = static_cast<const uint8_t*>(p);
    pay.insert(pay.end(), s, s + n);
    meta_bytes += (int64_t)n;
    return off;
  }
};

struct Launch {
  enum Kind { GATHER = 0, CDOT = 1, GSUM = 2, RGEMV = 3, FANOUT = 4 } kind = GATHER;
  int mode = 0;                   // RGEMV output mode
  int64_t off = 0, n = 0;         // range of items / outputs / pieces / fan-out slots
  bool use_rowscale = false;
  int64_t bytes = 0;              // algorithmic bytes moved by the launch
  int64_t woff[NSHAPES] = {};     // CDOT / RGEMV, per launch shape: ranges wbeg[woff .. woff + nw]
  int nw[NSHAPES] = {};           // ranges (warps; blocks for the multi-RHS shape) per launch shape
  int cfg = 0;                    // launch shape in use (autotuner choice)
  int maxrows = 0;                // RGEMV: rows of its widest chunk
  bool scatter = false;           // GSUM: also fills the slots of the folded fan-out after it
  int64_t copy_off = 0, copy_n = 0;  // GSUM with scatter: its copy entries fan_copy_{src,dst}[copy_off ..)
  int64_t xbytes = 0;             // bytes of that scatter (slot lists read, slots written)
};

struct Program {
  int tier = TIER_F32;
  std::vector<Launch> launches;
  std::vector<ItemCopy> items;    // column-dot items (copy descriptors)
  std::vector<int64_t> item_alg;  // algorithmic bytes of each item
  std::vector<GsumOut> gouts;
  std::vector<F2> pscale;         // per-partial weights of the outputs that use them
  std::vector<PieceCopy> pdesc[NSHAPES];  // row-chunk piece descriptors, one list per launch shape
  int64_t npieces = 0;
  std::vector<int64_t> piece_alg; // algorithmic bytes of each piece
  std::vector<int32_t> wbeg;      // per launch and shape: nw + 1 range starts (item / piece indices)
  std::vector<Split> splits;      // chunks shared by several warps (all launch shapes)
  int64_t nfix = 0;               // fix-up slots (CHUNK_ROWS float-float rows each), largest warp shape
  int64_t nfix_seq = 0;           // fix-up slots of shape SEQ_SHAPE, distinct across all launches
  bool too_large = false;         // build_program failed on an addressing limit (payload, vector)
  int64_t nfix_mr = 0;            // fix-up slots of the multi-RHS shape (CHUNK_ROWS x RP each)
  int64_t nchunks = 0;
  std::vector<int32_t> fan_src;   // fan-out: slot s takes v[fan_src[s]]; slot s is v[fan_base + s]
  int64_t fan_base = 0;
  // Folded fan-outs (a fan-out launch right after a segment-sum launch whose
  // slots all take coefficients of that launch or of the column dots before it):
  // a segment-sum output writes its slots fan_dst[pad .. pad + (flags >> 8)) of
  // its GsumOut; the slot fan_copy_dst[i] of a one-segment column-dot output
  // takes v[fan_copy_src[i]] in the same launch (vector indices throughout).
  std::vector<int32_t> fan_dst, fan_copy_src, fan_copy_dst;
  std::vector<double> rowscale;   // per vector entry (1 where unused)
  int64_t nvec = 0;               // float2 vector workspace entries (x first)
  int64_t npartial = 0;           // partials of the largest column-dot launch
  Packer pk;
  int64_t fp64_lowrank = 0, fp64_dense = 0;
};

constexpr int64_t MIN_WARP_BYTES = 4096;    // smallest share of a launch worth a warp
// Work-split weights: a warp's time grows with its bytes, with its pieces
// (header, input segment, reduction, outputs: column-dot pieces cost several
// times more than row-chunk pieces) and with the chunks it finishes.  The
// constants are in byte equivalents; measured per-warp timelines of the
// headline H product are flat (within noise) from half to twice these values.
constexpr int64_t PIECE_COST = 2048;    // row-chunk pieces
constexpr int64_t CPIECE_COST = 8192;   // column-dot pieces
constexpr int64_t EMIT_COST = 8192;     // finished row chunks

// Pack a built matrix with `codec` at accuracy eps (VALR if valr) and build its
// launch program for a GPU with nsm multiprocessors.  Returns false if a value
// range is outside what the kernels decode.
bool build_program(const HostMatrix& H, int codec, double eps, int valr, int nsm, Program& P);

// Dependencies (SeqDep per piece of shape SEQ_SHAPE) of the row-chunk launches
// [first, last) of P run as the phases of one persistent launch; nchunks is the
// number of coefficient chunks they version.  Returns false if the launches
// cannot run that way (they then run one launch each).
bool seq_dependencies(const Program& P, size_t first, size_t last, std::vector<SeqDep>& deps, int& nchunks);

// Packed factors and work list of the H-LU triangular solves x = U^-1 L^-1 b
// (Sec. 5, Conclusion).  L and U hold the factor blocks on the block tree of A
// (L: blocks after the diagonal and the unit lower diagonal triangles; U:
// blocks before it and the upper diagonal triangles).
struct LuProgram {
  int tier = TIER_FF;
  Packer pk;
  std::vector<LuCol> cols;
  std::vector<LuItem> items;
  std::vector<LuDep> deps;
  int64_t nflags = 0;       // done flags (2 per leaf) and coefficient counters
  int64_t ncoef = 0;        // coefficients of the low-rank blocks of both factors
  int64_t nleaves = 0;
  int64_t bytes_fp64 = 0;   // FP64 bytes of the same factors
};
bool build_lu_program(const HostMatrix& L, const HostMatrix& U, int codec, double eps, int valr, LuProgram& P);

// Dense unpivoted A = L U of the kernel matrix of prm on pts (cluster order),
// cut along A's block tree into the factor blocks of L and U (lu_factor.cpp).
// False if a pivot vanishes.  The dense array bounds n (LU_MAX_DENSE).
constexpr int64_t LU_MAX_DENSE = 8192;
bool lu_factor_host(const hm_build_params& prm, const double* pts, int64_t n, HostMatrix& L, HostMatrix& U);

}  // namespace hm
