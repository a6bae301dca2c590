// Device-side work descriptors shared by the kernels (kernels.cu) and the host
// layout builder (program.cpp).  Plain structs, identical layout on both sides.
//
// The packed payload is self-describing: every unit of work a warp streams
// into shared memory with one bulk copy (a column-dot item, a row-chunk piece)
// starts with an inline header that holds everything the warp needs to decode
// it, so the only descriptors read from global memory are the compact copy
// descriptors (offset, size) the warp prefetches 32 at a time.
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
HM_HD inline uint32_t fmt_word(int B, int fmt, int e, int m) {
  return (uint32_t)B | ((uint32_t)fmt << 8) | ((uint32_t)e << 16) | ((uint32_t)m << 24);
}

// 16-bit form of a format word used inside the streams: B (4 bits) | fmt << 4
// (2 bits) | e << 6 (4 bits) | m << 10 (6 bits).
HM_HD inline uint16_t fmt16(uint32_t fw) {
  const uint32_t B = fw & 0xff, f = (fw >> 8) & 0xff, e = (fw >> 16) & 0xff, m = fw >> 24;
  return (uint16_t)(B | (f << 4) | (e << 6) | (m << 10));
}

// Float-float pair (hi + lo): scales and partial sums, so that no FP64
// arithmetic runs per column (FP64 is 1/60 of the FP32 rate on GB300).
struct F2 {
  float hi, lo;
};

// Rows per lane in the product kernels: a lane decodes 8 (float-float tier)
// or 16 (FP32 tier) consecutive values of a column, i.e. groups of 4 codes,
// 8*B bytes per 8 rows, from an 8-byte aligned address; every packed column
// is padded to 8 bytes.
constexpr int RPL = 8;      // rows per group of two 4-code words
constexpr int RPL_MAX = 16;

// Shared-memory staging of the streaming kernels (per warp: NS stages).
// Launch shapes (warps per block, stages per warp) the autotuner chooses from;
// one block per SM.  Column dots also stage an input segment per stage.
constexpr int NCFG = 3;
constexpr int CS_CFG_WARPS[NCFG] = {16, 10, 7};
constexpr int CS_CFG_STAGES[NCFG] = {2, 3, 4};
constexpr int RS_CFG_WARPS[NCFG] = {16, 11, 8};
constexpr int RS_CFG_STAGES[NCFG] = {2, 3, 4};
// Multi-RHS products run in panels of RP right-hand sides on a separate split
// of every launch (launch shape index MR_SHAPE): row-chunk launches into
// MP_PAIRS ranges per SM (one per warp pair of the FP32-pipe kernel; the
// tensor-core kernel takes MP_PAIRS consecutive ranges per CTA), column-dot
// launches into MR_CDOT_RANGES ranges per SM.  Chunks of at most MP_ROWS rows
// may run on the FP32-pipe kernel; wider ones run on the tensor-core kernel.
constexpr int RP = 32;
constexpr int MP_PAIRS = 4;
constexpr int MP_ROWS = 64;
constexpr int MR_CDOT_RANGES = 16;
constexpr int MR_SHAPE = NCFG;
constexpr int NSHAPES = NCFG + 1;
constexpr int SEQ_SHAPE = 0;               // row-chunk shape of the persistent (multi-phase) launch

// One phase of a persistent launch: a row-chunk launch's warp ranges of shape
// SEQ_SHAPE.
struct SeqPhase {
  int32_t mode;      // output mode
  int32_t woff;      // range starts wbeg[woff .. woff + nw]
  int32_t nw;
  int32_t rowscale;  // 1: scale the rows by the row-scale vector
};

// One phase of the whole-product persistent launch (hm_persistent mode 2):
// the launches of one product run as the phases of ONE cooperative launch,
// phases separated by grid barriers, runs of row-chunk launches as dataflow.
enum { PP_GATHER = 0, PP_CDOT = 1, PP_GSUM = 2, PP_FANOUT = 3, PP_RGEMV = 4, PP_RUN = 5 };
struct ProgPhase {
  int32_t kind;
  int32_t off, n;     // GATHER: n entries; CDOT / RGEMV: ranges wbeg[off .. off + n]; GSUM / FANOUT:
                      // outputs / slots [off, off + n); RUN: SeqPhase entries [off, off + n)
  int32_t mode;       // RGEMV: output mode; RUN: the run's index
  int32_t rowscale;   // RGEMV: rows scaled by the row-scale vector
  int32_t aux;        // FANOUT: vector index of slot 0; RUN: offset of its state (versions, abort, claims)
  int32_t nchunks;    // RUN: versioned coefficient chunks
  int32_t pad;
};

// Dependencies of one piece of a persistent launch, as versions of coefficient
// chunks (a version counts the emits of the chunk so far in the launch): the
// piece's multipliers are final once ver[c0] >= v0 (c0 < 0: written before the
// launch), and its own chunk (c1, whose emit increments ver[c1]) holds the
// value it adds to once ver[c1] >= v1.
struct SeqDep {
  int32_t c0, v0, c1, v1;
};
constexpr int STAGE_BYTES = 6144;          // payload bytes of one stage (item / piece incl. header)
constexpr int SEG_ROWS = 64;               // rows of a column-dot segment
constexpr int CHUNK_ROWS = 128;            // rows of a row chunk
constexpr int PIECE_MAX_COLS = 64;         // columns of one row-chunk piece (2 multipliers per lane)

// ---------------------------------------------------------------- column dots (phase A)
// A column-dot piece holds <= 32 columns of one decode class over the same
// <= SEG_ROWS rows (one segment of a column cluster: the columns of every
// column set that multiplies the same part of the input vector), laid out as
//   CPieceHdr | CColMeta[ncols] | F2 scale[ncols] (ITEM_FINAL only) | columns
// where every column holds pad16(nrows) codes (rows past nrows are zero codes),
// i.e. pad16(nrows) * B bytes.  sum_j = sum_{r < nrows} M[r, j] * v[vin + r];
// ITEM_FINAL (the set fits one segment): v[out_j] = scale_j * (alpha if
// ITEM_ALPHA) * sum_j; otherwise partial[out_j] = sum_j.
constexpr int32_t ITEM_FINAL = 1;
constexpr int32_t ITEM_ALPHA = 2;
constexpr int CPIECE_MAX_COLS = 64;
struct CPieceHdr {
  int32_t vin;       // vector index of row 0
  uint16_t nrows;    // 1..SEG_ROWS
  uint16_t ncols;    // 1..CPIECE_MAX_COLS
  uint16_t fb;       // decode class: fmt << 4 | B
  uint16_t flags;    // ITEM_FINAL | ITEM_ALPHA
  int32_t limbs;     // BF16 limbs (1..3) that hold every decoded value exactly (multi-RHS path)
};
static_assert(sizeof(CPieceHdr) == 16, "CPieceHdr layout");

// Per column-dot column: e | m << 8 of its codes and its output index.
struct CColMeta {
  uint16_t em;
  uint16_t pad;
  int32_t out;
};

// Copy descriptor of a column-dot piece (pieces start 16-byte aligned):
// payload offset / 16, total bytes (header included), vector index of row 0,
// rows.  The input segment is copied only when it differs from the previous
// piece's of the same warp.
struct ItemCopy {
  uint32_t off16;
  uint32_t bytes;
  int32_t vin;
  int32_t nrows;
};

// ---------------------------------------------------------------- row chunks (phase C)
// A row chunk (a leaf cluster's rows of y, or <= 128 coefficients) is the sum
// of many columns restricted to its rows: the uniform tiles of directly
// compressed matrices (dense leaves, couplings, transfers) and the merged
// VALR columns (W factors of all low-rank blocks of its ancestors' block rows,
// or row bases).  They are cut into pieces of <= PIECE_MAX_COLS columns of one
// decode class (fmt, B) and <= STAGE_BYTES bytes, laid out as
//   PieceHdr | uint16 em[ncols] (merged pieces, padded to 8) | columns
// with column j at offset j * pad8(nrows * B) after the metadata.  A piece's
// multipliers are ncols consecutive vector entries v[moff ..] (a tile's input
// segment, or a run of multiplier slots that a fan-out launch fills from the
// scattered coefficients before the chunks run), copied into shared memory
// with the piece.
// Piece header flags (properties of the data).
constexpr uint16_t PH_TILE = 4;     // uniform tile piece (multipliers v[vin0 + j] * scale)
constexpr uint16_t PH_TALPHA = 8;   // tile piece multiplied by alpha
constexpr uint16_t PH_CALPHA = 32;  // chunk result multiplied by alpha (coefficient modes)
struct PieceHdr {
  int32_t row0;      // output index of the chunk's row 0
  uint16_t nrows;    // rows of the chunk (1..128)
  uint16_t flags;
  uint16_t fb;       // decode class: fmt << 4 | B
  uint16_t em;       // tile pieces: e | m << 8
  int32_t vin0;      // tile pieces: multiplier index of the piece's column 0
  uint16_t ncols;
  uint16_t limbs;    // BF16 limbs (1..3) that hold every decoded value exactly (multi-RHS path)
  int32_t pad1;
  F2 scale;          // tile pieces: AFLP vmin of the matrix (float-float), else 1
  int32_t pad[2];
};
static_assert(sizeof(PieceHdr) == 40, "PieceHdr layout");

// Copy descriptor of a piece for one split of the launch into warp ranges:
// payload offset / 16 (pieces start 16-byte aligned); bytes (header included) |
// range flags << 16 | ncols << 24;
// first multiplier index; for a chunk shared by several warps, its split index
// << 8 | this part's index (else -1).
constexpr uint32_t PD_FIRST = 1;    // first piece of this warp's part of the chunk: clear sums
constexpr uint32_t PD_LAST = 2;     // last piece of the part: emit
constexpr uint32_t PD_SPLIT = 4;    // the chunk is shared by several warps: emit through the fix-up
struct PieceCopy {
  uint32_t off16;
  uint32_t bytes_flags;
  int32_t moff;
  int32_t split_part;
};

// A chunk whose pieces are spread over several warps: the parts write their
// row sums to fix[(slot0 + pidx) * CHUNK_ROWS + r]; the last part to finish
// (counter) adds them in part order and emits.
struct Split {
  int32_t slot0;
  int32_t nparts;
};

// out_vec[out] = scale * (alpha if flags & 1) * sum_{p in [p0, p1)} w_p * partial[p], with
// w_p = pscale[ps + p - p0] if flags & 2, else 1 (float-float arithmetic).
// Each coefficient's partials (one per segment) are contiguous.
struct GsumOut {
  int32_t out;
  int32_t p0, p1;
  int32_t flags;
  F2 scale;
  int32_t ps;
  int32_t pad;
};

// Decoder check (hm_decompress_debug): 8 consecutive codes of one packed
// column at payload byte offset `off` (8-byte aligned), decode class
// fb = fmt << 4 | B and em = e | m << 8 packed as fb | em << 16; values
// out .. out + nr - 1 of the result take the first nr of them.
struct DbgTask {
  uint64_t off;
  uint32_t fbem;
  int32_t out;
  int32_t nr;
  int32_t pad;
};

// ---------------------------------------------------------------- H-LU triangular solves
// One packed column of a factor, restricted to the rows an item reads: a
// column of a dense leaf block or of a diagonal triangle (direct compression,
// one format per block), a column of W_b restricted to a leaf's rows, or a
// whole column of X_b (VALR, one format per column).
constexpr int32_t LC_COEF = 1;   // the multiplier is a coefficient t_b[j] (else the solved vector)
struct LuCol {
  uint64_t off;     // payload byte offset of the first row's code (8-byte aligned)
  double scale;     // value scale: AFLP vmin of a direct block, or the coefficient scale (column items)
  int32_t rows;
  int32_t mult;     // multiplier index (row items) / coefficient index (column items)
  uint16_t fb, em;  // decode class fmt << 4 | B; e | m << 8
  int32_t flags;
};
static_assert(sizeof(LuCol) == 32, "LuCol layout");

// Work items of the solve, in an order in which every item depends only on
// earlier ones.  Row items solve one leaf cluster's rows: forward (L, unit
// lower triangle) or backward (U, upper triangle); column items form the
// coefficients t_b = X_b^T z_sigma of the low-rank factor blocks once z_sigma
// is final.
enum { LU_ROW_L = 0, LU_COL_L = 1, LU_ROW_U = 2, LU_COL_U = 3 };
struct LuItem {
  int32_t kind;
  int32_t r0, nr;   // row items: the leaf's rows [r0, r0 + nr); column items: sigma's first row, rows
  int32_t c0, c1;   // column table range: contributions (row items) / X_b columns (column items)
  int32_t tri;      // row items: the first of nr columns of the diagonal triangle
  int32_t d0, d1;   // dependency range
  int32_t flag;     // row items: the done flag it sets; column items: the counter it adds to
  int32_t pad[3];
};
static_assert(sizeof(LuItem) == 48, "LuItem layout");

// A dependency: flags[flag] must reach target (done flags 1, coefficient counters k_b).
struct LuDep {
  int32_t flag, target;
};

enum { MODE_Y = 0, MODE_VEC = 1, MODE_VEC_ADD = 2 };
enum { TIER_F32 = 0, TIER_FF = 1 };

}  // namespace hm
