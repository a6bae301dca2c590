// hm_save / hm_load: the built matrix (Sec. 2: cluster tree, block tree,
// dense leaves, low-rank factors, cluster bases, couplings and transfer
// matrices, in FP64) and its compression settings, in one binary file.
//
// The packed form is not stored: it depends on the GPU it was laid out for
// (the warp ranges follow the number of SMs), and it is rebuilt from the
// stored matrix by hm_compress, deterministically, so that a loaded matrix
// gives the saved matrix's product bit for bit on the same GPU.  What the file
// saves is the expensive part, the host construction.
//
// Layout: little-endian, "HMAT" magic, a format version, then the fields in the
// order of write_matrix below; every array is a uint64 count followed by its
// elements.  The reader checks every count against the bytes left in the file.
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "hm_internal.h"

namespace hm {
// The matrix object and the compression entry point live in matrix.cpp.
HostMatrix& host_of(hm_matrix* m);
bool compressed_state(const hm_matrix* m, double& eps, int& codec, int& valr);
hm_matrix* new_matrix();
}  // namespace hm

using namespace hm;

namespace {

constexpr char kMagic[4] = {'H', 'M', 'A', 'T'};
constexpr uint32_t kVersion = 1;

struct Writer {
  FILE* f;
  bool ok = true;
  void raw(const void* p, size_t n) {
    if (ok && n && std::fwrite(p, 1, n, f) != n) ok = false;
  }
  template <typename T>
  void pod(const T& v) {
    raw(&v, sizeof v);
  }
  template <typename T>
  void vec(const std::vector<T>& v) {
    pod<uint64_t>(v.size());
    raw(v.data(), v.size() * sizeof(T));
  }
  template <typename T>
  void vecvec(const std::vector<std::vector<T>>& v) {
    pod<uint64_t>(v.size());
    for (const auto& x : v) vec(x);
  }
};

struct Reader {
  FILE* f;
  uint64_t left;
  bool ok = true;
  void raw(void* p, size_t n) {
    if (!ok) return;
    if (n > left || (n && std::fread(p, 1, n, f) != n)) {
      ok = false;
      return;
    }
    left -= n;
  }
  template <typename T>
  void pod(T& v) {
    raw(&v, sizeof v);
  }
  template <typename T>
  void vec(std::vector<T>& v) {
    uint64_t n = 0;
    pod(n);
    if (!ok || n > left / sizeof(T)) {
      ok = false;
      return;
    }
    v.resize(n);
    raw(v.data(), n * sizeof(T));
  }
  template <typename T>
  void vecvec(std::vector<std::vector<T>>& v) {
    uint64_t n = 0;
    pod(n);
    if (!ok || n > left / sizeof(uint64_t)) {
      ok = false;
      return;
    }
    v.resize(n);
    for (auto& x : v) vec(x);
  }
};

void write_bases(Writer& w, const Bases& b) {
  w.vecvec(b.B);
  w.vecvec(b.sig);
  w.vecvec(b.E);
  w.vec(b.k);
  w.pod(b.tau);
}

void read_bases(Reader& r, Bases& b) {
  r.vecvec(b.B);
  r.vecvec(b.sig);
  r.vecvec(b.E);
  r.vec(b.k);
  r.pod(b.tau);
}

void write_matrix(Writer& w, const HostMatrix& H) {
  w.pod(H.prm);
  w.pod(H.n);
  w.pod(H.kparam);
  w.vec(H.pts);
  w.vec(H.ct.cl);
  w.vec(H.ct.perm);
  w.pod(H.ct.depth);
  w.vec(H.blocks);
  w.vec(H.slot);
  w.pod<uint64_t>(H.lr.size());
  for (const LowRankBlock& L : H.lr) {
    w.pod(L.k);
    w.vec(L.W);
    w.vec(L.s);
    w.vec(L.X);
  }
  w.pod<uint64_t>(H.dn.size());
  for (const DenseBlock& D : H.dn) w.vec(D.D);
  write_bases(w, H.rowb);
  write_bases(w, H.colb);
  w.vecvec(H.coupling);
  w.vecvec(H.coupling_r);
  w.vecvec(H.coupling_ct);
}

bool read_matrix(Reader& r, HostMatrix& H) {
  r.pod(H.prm);
  r.pod(H.n);
  r.pod(H.kparam);
  r.vec(H.pts);
  r.vec(H.ct.cl);
  r.vec(H.ct.perm);
  r.pod(H.ct.depth);
  r.vec(H.blocks);
  r.vec(H.slot);
  uint64_t nl = 0;
  r.pod(nl);
  if (!r.ok || nl > r.left) return false;
  H.lr.resize(nl);
  for (LowRankBlock& L : H.lr) {
    r.pod(L.k);
    r.vec(L.W);
    r.vec(L.s);
    r.vec(L.X);
  }
  uint64_t nd = 0;
  r.pod(nd);
  if (!r.ok || nd > r.left) return false;
  H.dn.resize(nd);
  for (DenseBlock& D : H.dn) r.vec(D.D);
  read_bases(r, H.rowb);
  read_bases(r, H.colb);
  r.vecvec(H.coupling);
  r.vecvec(H.coupling_r);
  r.vecvec(H.coupling_ct);
  return r.ok;
}

// Structural consistency of a read matrix (a damaged file must not reach the
// packer with out-of-range indices).
bool consistent(const HostMatrix& H) {
  const int64_t n = H.n;
  if (n < 1 || (int64_t)H.pts.size() != 3 * n || (int64_t)H.ct.perm.size() != n || H.ct.cl.empty()) return false;
  const int nc = (int)H.ct.cl.size();
  for (const Cluster& c : H.ct.cl)
    if (c.start < 0 || c.end > n || c.start > c.end || c.parent >= nc || c.nsons < 0 || c.nsons > 2 ||
        c.son[0] >= nc || c.son[1] >= nc)
      return false;
  for (int64_t p : H.ct.perm)
    if (p < 0 || p >= n) return false;
  if (H.slot.size() != H.blocks.size()) return false;
  for (size_t b = 0; b < H.blocks.size(); ++b) {
    const BlockLeaf& B = H.blocks[b];
    if (B.row < 0 || B.row >= nc || B.col < 0 || B.col >= nc) return false;
    const int s = H.slot[b];
    const int64_t m = H.ct.cl[B.row].size(), k = H.ct.cl[B.col].size();
    if (B.adm) {
      if (s < 0 || s >= (int)H.lr.size()) return false;
      const LowRankBlock& L = H.lr[s];
      if (L.k < 0 || (int64_t)L.W.size() != m * L.k || (int64_t)L.X.size() != k * L.k || (int)L.s.size() != L.k)
        return false;
    } else {
      if (s < 0 || s >= (int)H.dn.size() || (int64_t)H.dn[s].D.size() != m * k) return false;
    }
  }
  return true;
}

}  // namespace

extern "C" {

hm_status hm_save(const hm_matrix* m, const char* path) {
  if (!m || !path) return HM_ERR_ARG;
  const HostMatrix& H = host_of(const_cast<hm_matrix*>(m));
  double eps = 0;
  int codec = 0, valr = 0;
  const int32_t comp = compressed_state(m, eps, codec, valr) ? 1 : 0;
  FILE* f = std::fopen(path, "wb");
  if (!f) return HM_ERR_IO;
  Writer w{f};
  w.raw(kMagic, 4);
  w.pod(kVersion);
  w.pod(comp);
  w.pod(eps);
  w.pod<int32_t>(codec);
  w.pod<int32_t>(valr);
  write_matrix(w, H);
  const bool ok = w.ok && std::fflush(f) == 0;
  if (std::fclose(f) != 0 || !ok) return HM_ERR_IO;
  return HM_OK;
}

hm_status hm_load(const char* path, hm_matrix** out) {
  if (!path || !out) return HM_ERR_ARG;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return HM_ERR_IO;
  std::fseek(f, 0, SEEK_END);
  const long sz = std::ftell(f);
  std::fseek(f, 0, SEEK_SET);
  if (sz < 0) {
    std::fclose(f);
    return HM_ERR_IO;
  }
  Reader r{f, (uint64_t)sz};
  char mg[4] = {};
  uint32_t ver = 0;
  int32_t comp = 0, codec = 0, valr = 0;
  double eps = 0;
  r.raw(mg, 4);
  r.pod(ver);
  r.pod(comp);
  r.pod(eps);
  r.pod(codec);
  r.pod(valr);
  std::unique_ptr<hm_matrix, hm_status (*)(hm_matrix*)> M(nullptr, hm_free);
  bool ok = r.ok && std::memcmp(mg, kMagic, 4) == 0 && ver == kVersion;
  try {
    if (ok) {
      M.reset(new_matrix());
      ok = read_matrix(r, host_of(M.get())) && r.left == 0 && consistent(host_of(M.get()));
    }
  } catch (const std::bad_alloc&) {
    std::fclose(f);
    return HM_ERR_OOM;
  }
  std::fclose(f);
  if (!ok) return HM_ERR_IO;
  if (comp) {
    const hm_status s = hm_compress(M.get(), eps, codec, valr);
    if (s != HM_OK) return s;
  }
  *out = M.release();
  return HM_OK;
}

}  // extern "C"
