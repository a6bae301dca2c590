// Device-side work descriptors shared by the kernels (kernels.cu) and the host
// layout builder (matrix.cpp).  Plain structs, identical layout on both sides.
#pragma once
#include <cstdint>

namespace hm {

// Packed value format word: B | fmt << 8 | e << 16 | m << 24.
//   fmt 0: FPX e8 (B 2..4)   1: FPX e11 (B 5..8)   2: AFLP (B 1..7)   3: raw FP64 (B 8)
// Every packed column starts 4-byte aligned and occupies pad4(rows * B) bytes.
__host__ __device__ inline uint32_t fmt_word(int B, int fmt, int e, int m) {
  return (uint32_t)B | ((uint32_t)fmt << 8) | ((uint32_t)e << 16) | ((uint32_t)m << 24);
}

// Column dot products (phase A): partial[pout + j] = sum_{r in segment} M[r, j] * v[vin + r]
// over the columns j < ncols of a packed matrix with nrows rows per column.
struct CdotItem {
  uint64_t off;     // payload byte offset of column 0
  int32_t fmt;      // >= 0: fmt index of column 0 (one word per column); < 0: ~index of one word
  int32_t ncols;
  int32_t nrows;    // rows of every column (column byte length pad4(nrows * B))
  int32_t row0;     // first row of the segment, a multiple of 4
  int32_t seg;      // rows in the segment, 1..512
  int32_t vin;      // vector index of row 0 of the column
  int32_t pout;     // partial index of column 0
  int32_t pad;
};

// One packed column-major tile (rows = the chunk's rows) multiplied by a vector segment.
struct Tile {
  uint64_t off;     // payload byte offset of column 0
  int32_t fmt;      // as CdotItem::fmt
  int32_t ncols;
  int32_t vin;      // vector index of column 0's input value
  int32_t flags;    // bit 0: multiply by alpha
  double scale;     // AFLP vmin of a direct-compressed matrix, else 1
};

// A run of output rows owned by one thread block; its tiles are [t0, t1).
struct Chunk {
  int32_t row0;     // output index of row 0
  int32_t nrows;    // 1..128
  int32_t t0, t1;
  int32_t flags;    // bit 0: multiply the result by alpha
  int32_t pad;
};

// out_vec[out] = scale * (alpha if flags&1) * sum_{p in [p0,p1)} pscale[p] * partial[plist[p]]
struct GsumOut {
  int32_t out;
  int32_t p0, p1;
  int32_t flags;
  double scale;
};

enum { MODE_Y = 0, MODE_VEC = 1, MODE_VEC_ADD = 2 };
enum { TIER_F32 = 0, TIER_FF = 1 };

}  // namespace hm
