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
  std::vector<uint8_t> pay;       // packed codes, every column 8-byte aligned
  std::vector<uint32_t> fmts;     // format words
  std::vector<F2> cscale;         // output scale of column-dot columns (parallel to fmts)
  int64_t value_bytes = 0;        // sum of n * B over all packed columns (no padding)

  uint64_t align8() {
    while (pay.size() & 7) pay.push_back(0);
    return pay.size();
  }
  // append n codes of B bytes (little-endian); returns the 8-byte aligned offset
  uint64_t put(const uint64_t* codes, int64_t n, int B) {
    uint64_t off = align8();
    pay.resize(off + (uint64_t)(n * B));
    uint8_t* dst = pay.data() + off;
    for (int64_t i = 0; i < n; ++i) {
      const uint64_t c = codes[i];
      for (int b = 0; b < B; ++b) dst[i * B + b] = (uint8_t)(c >> (8 * b));
    }
    value_bytes += n * B;
    align8();
    return off;
  }
};

struct Launch {
  enum Kind { GATHER = 0, CDOT = 1, GSUM = 2, RGEMV = 3 } kind = GATHER;
  int mode = 0;                   // RGEMV output mode
  int64_t off = 0, n = 0;         // range of items / outputs
  bool use_rowscale = false;
  int64_t bytes = 0;              // algorithmic bytes moved by the launch
};

struct Program {
  int tier = TIER_F32;
  std::vector<Launch> launches;
  std::vector<Item> items;        // column-dot items
  std::vector<GsumOut> gouts;
  std::vector<int32_t> plist;
  std::vector<F2> pscale;
  std::vector<Tile> tiles;        // uniform row-chunk tiles
  std::vector<ColMeta> cols;      // merged row-chunk columns
  std::vector<Chunk> chunks;
  std::vector<double> rowscale;   // per vector entry (1 where unused)
  int64_t nvec = 0;               // float2 vector workspace entries (x first)
  int64_t npartial = 0;           // partials of the largest column-dot launch
  Packer pk;
  int64_t fp64_lowrank = 0, fp64_dense = 0;
};

// Pack a built matrix with `codec` at accuracy eps (VALR if valr) and build its
// launch program for a GPU with nsm multiprocessors.  Returns false if a value
// range is outside what the kernels decode.
bool build_program(const HostMatrix& H, int codec, double eps, int valr, int nsm, Program& P);

}  // namespace hm
