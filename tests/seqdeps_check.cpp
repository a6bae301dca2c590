// Host check of seq_dependencies (the dependency analysis of the persistent
// launch) on small hand-built programs: which chunk a multiplier run reads, the
// versions it waits for, and the cases that must keep the launches separate (a
// run straddling a chunk boundary; a chunk written after a phase read it).
// Test code, built by tests/test_program_layout.py; prints "ok" or the failures.
#include <cstdio>
#include <cstring>
#include <vector>

#include "program.h"

using namespace hm;

namespace {

int g_fails = 0;

void expect(bool cond, const char* what) {
  if (!cond) {
    std::printf("FAIL: %s\n", what);
    ++g_fails;
  }
}

// A program of row-chunk launches, one piece each: piece p writes rows
// [row0, row0 + nrows) in mode `mode` and reads ncols multipliers from moff.
struct Piece {
  int mode, row0, nrows, moff, ncols;
};

Program make(const std::vector<Piece>& ps) {
  Program P;
  for (size_t i = 0; i < ps.size(); ++i) {
    const Piece& q = ps[i];
    const uint64_t off = P.pk.align(16);
    PieceHdr h{};
    h.row0 = q.row0;
    h.nrows = (uint16_t)q.nrows;
    h.ncols = (uint16_t)q.ncols;
    P.pk.raw(&h, sizeof h);
    P.pk.align(16);
    P.pdesc[SEQ_SHAPE].push_back(PieceCopy{(uint32_t)(off >> 4), (uint32_t)sizeof h | (uint32_t)q.ncols << 24,
                                           q.moff, -1});
    Launch L;
    L.kind = Launch::RGEMV;
    L.mode = q.mode;
    L.off = (int64_t)i;
    L.n = 1;
    P.launches.push_back(L);
  }
  P.npieces = (int64_t)ps.size();
  return P;
}

bool deps_of(const std::vector<Piece>& ps, std::vector<SeqDep>& d) {
  const Program P = make(ps);
  int nchunks = 0;
  d.clear();
  return seq_dependencies(P, 0, ps.size(), d, nchunks);
}

}  // namespace

int main() {
  std::vector<SeqDep> d;
  // phase 0 writes chunk A = [100, 108); phase 1 writes B = [200, 208) reading [m0, m0 + nc)
  auto two = [&](int m0, int nc) {
    return deps_of({{MODE_VEC, 100, 8, 0, 0}, {MODE_VEC, 200, 8, m0, nc}}, d);
  };
  expect(two(100, 8) && d[1].c0 == 0 && d[1].v0 == 1, "a run inside chunk A waits for A's first emit");
  expect(two(102, 4) && d[1].c0 == 0 && d[1].v0 == 1, "a run strictly inside A waits for A");
  expect(two(108, 4) && d[1].c0 == -1, "a run starting at A's end reads no chunk");
  expect(two(92, 8) && d[1].c0 == -1, "a run ending at A's start reads no chunk");
  expect(!two(104, 8), "a run crossing A's end keeps the launches separate");
  expect(!two(96, 8), "a run crossing A's start keeps the launches separate");
  expect(!two(96, 16), "a run covering A keeps the launches separate");
  expect(two(100, 8) && d[1].c1 == 1 && d[1].v1 == 0 && d[0].c1 == 0 && d[0].v1 == 0,
         "each piece's own chunk at its current version");
  // read-modify-write of one chunk by consecutive phases: ordered by versions
  expect(deps_of({{MODE_VEC, 100, 8, 0, 0}, {MODE_VEC_ADD, 100, 8, 0, 0}}, d) && d[1].c1 == 0 && d[1].v1 == 1,
         "a second write of A waits for the first");
  // a chunk written after a phase read it: a reader could see the later value
  expect(!deps_of({{MODE_VEC, 100, 8, 0, 0}, {MODE_VEC, 200, 8, 100, 8}, {MODE_VEC_ADD, 100, 8, 0, 0}}, d),
         "writing A after a phase read it keeps the launches separate");
  // the first phase of the run reads A, a later one writes it
  expect(!deps_of({{MODE_VEC, 200, 8, 100, 8}, {MODE_VEC, 100, 8, 0, 0}}, d),
         "writing A after the first phase read it keeps the launches separate");
  // a final MODE_Y phase reads coefficients but owns no chunk
  expect(deps_of({{MODE_VEC, 100, 8, 0, 0}, {MODE_Y, 0, 8, 100, 8}}, d) && d[1].c0 == 0 && d[1].v0 == 1 &&
             d[1].c1 == -1,
         "a MODE_Y phase waits for its coefficients and versions nothing");
  if (g_fails) {
    std::printf("FAILED %d\n", g_fails);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
