// Device-side work descriptors shared by the kernels (kernels.cu) and the host
// layout builder (matrix.cpp).  Plain structs, identical layout on both sides.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define HM_HD __host__ __device__
#else
#define HM_HD
#endif

namespace hm {

// Packed value format word: B | fmt << 8 | e << 16 | m << 24.
//   fmt 0: FPX e8 (B 2..4)   1: FPX e11 (B 5..8)   2: AFLP (B 1..7)   3: raw FP64 (B 8)
// Every packed column starts 4-byte aligned and occupies pad4(rows * B) bytes.
HM_HD inline uint32_t fmt_word(int B, int fmt, int e, int m) {
  return (uint32_t)B | ((uint32_t)fmt << 8) | ((uint32_t)e << 16) | ((uint32_t)m << 24);
}

// Float-float pair (hi + lo): scales and partial sums, so that no FP64
// arithmetic runs per column (FP64 is 1/60 of the FP32 rate on GB300).
struct F2 {
  float hi, lo;
};

// Rows per lane in the product kernels: every lane decodes 8 consecutive
// values of a column (two groups of 4 codes = 2B 32-bit words, one 8-byte
// aligned run), so columns are padded to 8 bytes.
constexpr int RPL = 8;

// Column dots (phase A): sum_j = sum_{r < nrows} M[r, j] * v[vin + r] over the
// ncols columns of one item (one segment of a column set); column j has format
// word fmts[fmt + j] and output scale cscale[fmt + j] (float-float); columns are contiguous
// from `off`, each pad8(nrows * B_j) bytes.  A set with a single segment
// writes its coefficients directly (ITEM_FINAL): vout[out + j] =
// cscale[fmt + j] * (alpha if ITEM_ALPHA) * sum_j; otherwise partial[out + j] = sum_j.
constexpr int32_t ITEM_FINAL = 1;
constexpr int32_t ITEM_ALPHA = 2;
struct Item {
  uint64_t off;
  int32_t fmt;
  int32_t ncols;
  int32_t nrows;    // 1..128
  int32_t vin;      // vector index of row 0
  int32_t out;      // partial index, or vector index with ITEM_FINAL, of column 0
  int32_t flags;
};

// Uniform tile of a row chunk: ncols columns of the chunk's rows, one format
// word for all of them (direct compression), input v[vin + j] times `scale`.
struct Tile {
  uint64_t off;     // payload byte offset of column 0 (8-byte aligned)
  int32_t ncols;
  uint32_t fw;      // format word
  int32_t vin;
  int32_t flags;    // bit 0: multiply by alpha
  F2 scale;         // AFLP vmin of the direct-compressed matrix (float-float), else 1
};

// Column of a row chunk's merged VALR columns (W factors, row bases): its
// format word and the vector index of its multiplier; the columns follow each
// other from Chunk::coff, each pad8(nrows * B) bytes, sorted by format.
struct ColMeta {
  uint32_t fw;
  int32_t vin;
};

// A run of output rows owned by one thread block: uniform tiles [t0, t1) and
// merged columns [c0, c1) starting at payload offset coff.
struct Chunk {
  uint64_t coff;
  int32_t row0;     // output index of row 0
  int32_t nrows;    // 1..128
  int32_t t0, t1;
  int32_t c0, c1;
  int32_t flags;    // bit 0: multiply the result by alpha
  int32_t pad;
};

// out_vec[out] = scale * (alpha if flags&1) * sum_{p in [p0,p1)} pscale[p] * partial[plist[p]]
// (float-float arithmetic)
struct GsumOut {
  int32_t out;
  int32_t p0, p1;
  int32_t flags;
  F2 scale;
};

enum { MODE_Y = 0, MODE_VEC = 1, MODE_VEC_ADD = 2 };
enum { TIER_F32 = 0, TIER_FF = 1 };

}  // namespace hm
