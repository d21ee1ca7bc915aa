// Factor files: the checkpoint of the host construction.  The FP64 build of §2.3-2.4
// (entry evaluation and randomized SVDs of every block) runs once; its padded factor set
// is written to a file and later processes load it instead of rebuilding.
//
// Layout (version 1, the host's little-endian byte order, recorded by a tag):
//   header (64 bytes): magic "MBFFACT1", version, endian tag 0x01020304, dim, L, n_out,
//                      n_in, n_w, max_leaf_x, max_leaf_w, nnz
//   x_perm[n_out], x_off[c^L + 1], w_perm[n_w], w_off[c^L + 1]        int64
//   RU[L + 1], RV[L + 1]                                               int32
//   UL, VL, G[h..L-1], H[h..L-1]    complex128 (interleaved), shapes of mbf_factors_t
//   S                                                                   float64
//   checksum                        uint64, over every byte before it
// The file is written under a temporary name and renamed when complete, so a file with
// the final name is never a partial write.
//
// A file written by a build (build_or_load) has a kernel record beside it, `path`.kernel:
// magic "MBFKERN1", count, dim, then count entries K(x, xi) of the kernel it was built
// from (natural x index, natural xi index, Re, Im) and a checksum.  Loading the file for
// a build evaluates the build's entry function at the same points and rejects the file if
// they differ, so that factors of one kernel are never taken for another with the same
// grids and trees (a 2-D DFT and a 2-D FIO without polar transform, for instance).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mbf_internal.hpp"

namespace mbf {
namespace {

constexpr char kMagic[8] = {'M', 'B', 'F', 'F', 'A', 'C', 'T', '1'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kEndianTag = 0x01020304u;

struct FileHeader {
  char magic[8];
  uint32_t version, endian;
  int32_t dim, L;
  int64_t n_out, n_in, n_w;
  int32_t max_leaf_x, max_leaf_w;
  int64_t nnz;
};
static_assert(sizeof(FileHeader) == 64, "factor file header is 64 bytes");

// 64-bit FNV-1a taken over 8-byte words (then the tail bytes): a corruption check, not
// a cryptographic hash.
struct Checksum {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    constexpr uint64_t kPrime = 1099511628211ull;
    const unsigned char* b = static_cast<const unsigned char*>(p);
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
      uint64_t w;
      std::memcpy(&w, b + i, 8);
      h = (h ^ w) * kPrime;
    }
    for (; i < n; ++i) h = (h ^ b[i]) * kPrime;
  }
};

// a * b, failing on int64 overflow (sizes read from a file are not trusted).
int64_t mul(int64_t a, int64_t b) {
  int64_t r;
  if (a < 0 || b < 0 || __builtin_mul_overflow(a, b, &r)) fail(MBF_ERR_IO, "corrupt factor file (sizes overflow)");
  return r;
}

// Array sizes (elements) of a factor set with the given header and ranks.
struct Sizes {
  int c = 4, h = 1;
  int64_t nL = 0, ul = 0, vl = 0, s = 0;
  std::vector<int64_t> g, hh;
};
Sizes sizes_of(int dim, int L, int32_t max_leaf_x, int32_t max_leaf_w, const int32_t* RU, const int32_t* RV) {
  Sizes z;
  z.c = 1 << dim;
  z.h = L / 2;
  z.nL = Tree::ipow(z.c, L);
  z.ul = mul(mul(z.nL, max_leaf_x), RU[L]);
  z.vl = mul(mul(z.nL, max_leaf_w), RV[L]);
  for (int l = z.h; l < L; ++l) {
    z.g.push_back(mul(mul(mul(z.nL, z.c), RU[l + 1]), RU[l]));
    z.hh.push_back(mul(mul(mul(z.nL, z.c), RV[l + 1]), RV[l]));
  }
  z.s = mul(Tree::ipow(z.c, 2 * z.h), RU[z.h]);
  return z;
}

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

class Writer {
 public:
  Writer(FILE* f, const std::string& path) : f_(f), path_(path) {}
  void put(const void* p, size_t n) {
    if (n && std::fwrite(p, 1, n, f_) != n) fail(MBF_ERR_IO, "write failed: " + path_);
    sum_.add(p, n);
  }
  uint64_t sum() const { return sum_.h; }

 private:
  FILE* f_;
  std::string path_;
  Checksum sum_;
};

class Reader {
 public:
  Reader(FILE* f, const std::string& path) : f_(f), path_(path) {}
  void get(void* p, size_t n) {
    if (n && std::fread(p, 1, n, f_) != n) fail(MBF_ERR_IO, "truncated factor file: " + path_);
    sum_.add(p, n);
  }
  template <class T>
  std::vector<T> vec(int64_t count) {
    std::vector<T> v(static_cast<size_t>(count));
    get(v.data(), size_t(count) * sizeof(T));
    return v;
  }
  uint64_t sum() const { return sum_.h; }

 private:
  FILE* f_;
  std::string path_;
  Checksum sum_;
};

}  // namespace

void save_factors(const mbf_factors_t& f, const std::string& path) {
  validate(f);
  const Sizes z = sizes_of(f.dim, f.L, f.max_leaf_x, f.max_leaf_w, f.RU, f.RV);
  const std::string tmp = path + ".tmp";
  try {
    File file;
    file.f = std::fopen(tmp.c_str(), "wb");
    if (!file.f) fail(MBF_ERR_IO, "cannot create " + tmp);
    Writer w(file.f, tmp);
    FileHeader hd{};
    std::memcpy(hd.magic, kMagic, 8);
    hd.version = kVersion;
    hd.endian = kEndianTag;
    hd.dim = f.dim;
    hd.L = f.L;
    hd.n_out = f.n_out;
    hd.n_in = f.n_in;
    hd.n_w = f.n_w;
    hd.max_leaf_x = f.max_leaf_x;
    hd.max_leaf_w = f.max_leaf_w;
    hd.nnz = f.nnz;
    w.put(&hd, sizeof hd);
    w.put(f.x_perm, size_t(f.n_out) * 8);
    w.put(f.x_off, size_t(z.nL + 1) * 8);
    w.put(f.w_perm, size_t(f.n_w) * 8);
    w.put(f.w_off, size_t(z.nL + 1) * 8);
    w.put(f.RU, size_t(f.L + 1) * 4);
    w.put(f.RV, size_t(f.L + 1) * 4);
    w.put(f.UL, size_t(z.ul) * 16);
    w.put(f.VL, size_t(z.vl) * 16);
    for (size_t q = 0; q < z.g.size(); ++q) w.put(f.G[q], size_t(z.g[q]) * 16);
    for (size_t q = 0; q < z.hh.size(); ++q) w.put(f.H[q], size_t(z.hh[q]) * 16);
    w.put(f.S, size_t(z.s) * 8);
    const uint64_t sum = w.sum();
    if (std::fwrite(&sum, 1, 8, file.f) != 8) fail(MBF_ERR_IO, "write failed: " + tmp);
    const int rc = std::fclose(file.f);
    file.f = nullptr;
    if (rc != 0) fail(MBF_ERR_IO, "write failed: " + tmp);
  } catch (...) {   // no partial file is left behind
    std::remove(tmp.c_str());
    throw;
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    fail(MBF_ERR_IO, "cannot rename " + tmp + " to " + path);
  }
}

FactorSet load_factors(const std::string& path) {
  File file;
  file.f = std::fopen(path.c_str(), "rb");
  if (!file.f) fail(MBF_ERR_IO, "cannot open " + path);
  if (std::fseek(file.f, 0, SEEK_END) != 0) fail(MBF_ERR_IO, "cannot seek " + path);
  const long long file_bytes = std::ftell(file.f);
  std::rewind(file.f);
  Reader r(file.f, path);
  FileHeader hd{};
  if (file_bytes < static_cast<long long>(sizeof hd) + 8) fail(MBF_ERR_IO, "not a factor file (too short): " + path);
  r.get(&hd, sizeof hd);
  if (std::memcmp(hd.magic, kMagic, 8) != 0) fail(MBF_ERR_IO, "not a factor file: " + path);
  if (hd.version != kVersion) fail(MBF_ERR_IO, "unsupported factor file version " + std::to_string(hd.version));
  if (hd.endian != kEndianTag) fail(MBF_ERR_IO, "factor file written with another byte order: " + path);
  // bounds on the header before any allocation it sizes
  const int64_t kMaxN = int64_t(1) << 40;
  if ((hd.dim != 2 && hd.dim != 3) || hd.L < 2 || hd.L > 20 || hd.L % 2 || hd.n_out < 1 || hd.n_out > kMaxN ||
      hd.n_in < 1 || hd.n_in > kMaxN || hd.n_w < 0 || hd.n_w > hd.n_in || hd.max_leaf_x < 1 ||
      hd.max_leaf_w < 1 || hd.max_leaf_x > (1 << 24) || hd.max_leaf_w > (1 << 24))
    fail(MBF_ERR_IO, "corrupt factor file header: " + path);
  const int c = 1 << hd.dim;
  if (hd.L * hd.dim > 40) fail(MBF_ERR_IO, "corrupt factor file header (c^L too large): " + path);
  const int64_t nL = Tree::ipow(c, hd.L);
  int64_t need = int64_t(sizeof hd) + 8 * (hd.n_out + hd.n_w + 2 * (nL + 1)) + 8 * (hd.L + 1);
  if (need > file_bytes) fail(MBF_ERR_IO, "truncated factor file: " + path);
  FactorSet fs;
  fs.d = hd.dim;
  fs.L = hd.L;
  fs.n_out = hd.n_out;
  fs.n_in = hd.n_in;
  fs.n_w = hd.n_w;
  fs.max_leaf_x = hd.max_leaf_x;
  fs.max_leaf_w = hd.max_leaf_w;
  fs.nnz = hd.nnz;
  fs.x_perm = r.vec<int64_t>(hd.n_out);
  fs.x_off = r.vec<int64_t>(nL + 1);
  fs.w_perm = r.vec<int64_t>(hd.n_w);
  fs.w_off = r.vec<int64_t>(nL + 1);
  fs.RU = r.vec<int32_t>(hd.L + 1);
  fs.RV = r.vec<int32_t>(hd.L + 1);
  const int h = hd.L / 2;
  for (int l = h; l <= hd.L; ++l)
    if (fs.RU[size_t(l)] < 1 || fs.RV[size_t(l)] < 1 || fs.RU[size_t(l)] > 4096 || fs.RV[size_t(l)] > 4096)
      fail(MBF_ERR_IO, "corrupt factor file (ranks): " + path);
  const Sizes z = sizes_of(hd.dim, hd.L, hd.max_leaf_x, hd.max_leaf_w, fs.RU.data(), fs.RV.data());
  auto add = [&](int64_t bytes) {
    if (__builtin_add_overflow(need, bytes, &need)) fail(MBF_ERR_IO, "corrupt factor file (sizes overflow)");
  };
  add(mul(16, z.ul));
  add(mul(16, z.vl));
  add(mul(8, z.s));
  add(8);
  for (size_t q = 0; q < z.g.size(); ++q) {
    add(mul(16, z.g[q]));
    add(mul(16, z.hh[q]));
  }
  if (need != file_bytes)
    fail(MBF_ERR_IO, "factor file size " + std::to_string(file_bytes) + " does not match its header (" +
                         std::to_string(need) + " bytes): " + path);
  fs.UL = r.vec<cd>(z.ul);
  fs.VL = r.vec<cd>(z.vl);
  for (size_t q = 0; q < z.g.size(); ++q) fs.G.push_back(r.vec<cd>(z.g[q]));
  for (size_t q = 0; q < z.hh.size(); ++q) fs.H.push_back(r.vec<cd>(z.hh[q]));
  fs.S = r.vec<double>(z.s);
  const uint64_t expect = r.sum();
  uint64_t stored = 0;
  if (std::fread(&stored, 1, 8, file.f) != 8) fail(MBF_ERR_IO, "truncated factor file: " + path);
  if (stored != expect) fail(MBF_ERR_IO, "factor file checksum mismatch (corrupt file): " + path);
  validate(fs.view());
  return fs;
}

namespace {

constexpr char kKernMagic[8] = {'M', 'B', 'F', 'K', 'E', 'R', 'N', '1'};
constexpr int kKernEntries = 16;

struct KernelEntry {
  int64_t x, xi;
  double re, im;
};

// The sampled entries: fixed positions in tree order (spread by two primes), the
// kernel evaluated through the entry function at their grid coordinates (eqs. X, Omega).
std::vector<KernelEntry> kernel_entries(const mbf_problem_t& prob, const FactorSet& fs, mbf_entry_fn fn, void* ctx) {
  std::vector<KernelEntry> e;
  if (!fn || fs.n_out < 1 || fs.n_w < 1) return e;
  const int d = prob.dim, n = prob.n;
  for (int k = 0; k < kKernEntries; ++k) {
    KernelEntry q{};
    q.x = fs.x_perm[size_t((int64_t(k) * 7919) % fs.n_out)];
    q.xi = fs.w_perm[size_t((int64_t(k) * 104729 + 3) % fs.n_w)];
    double x[3], xi[3], out[2];
    if (prob.tree == MBF_TREE_POINTS) {
      for (int t = 0; t < d; ++t) {
        x[t] = prob.x_pts[q.x * d + t];
        xi[t] = prob.w_pts[q.xi * d + t];
      }
    } else {
      int64_t a = q.x, b = q.xi;
      for (int t = d - 1; t >= 0; --t) {
        x[t] = double(a % n) / n;
        xi[t] = double(b % n) - n / 2;
        a /= n;
        b /= n;
      }
    }
    fn(x, 1, xi, 1, d, out, ctx);
    q.re = out[0];
    q.im = out[1];
    e.push_back(q);
  }
  return e;
}

void save_kernel_record(const std::string& path, int dim, const std::vector<KernelEntry>& e) {
  const std::string tmp = path + ".tmp";
  {
    File file;
    file.f = std::fopen(tmp.c_str(), "wb");
    if (!file.f) fail(MBF_ERR_IO, "cannot create " + tmp);
    Writer w(file.f, tmp);
    const int32_t head[2] = {int32_t(e.size()), dim};
    w.put(kKernMagic, 8);
    w.put(head, sizeof head);
    w.put(e.data(), e.size() * sizeof(KernelEntry));
    const uint64_t sum = w.sum();
    if (std::fwrite(&sum, 1, 8, file.f) != 8) fail(MBF_ERR_IO, "write failed: " + tmp);
    const int rc = std::fclose(file.f);
    file.f = nullptr;
    if (rc != 0) {
      std::remove(tmp.c_str());
      fail(MBF_ERR_IO, "write failed: " + tmp);
    }
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    fail(MBF_ERR_IO, "cannot rename " + tmp + " to " + path);
  }
}

std::vector<KernelEntry> load_kernel_record(const std::string& path) {
  File file;
  file.f = std::fopen(path.c_str(), "rb");
  if (!file.f)
    fail(MBF_ERR_INVALID, "factor file has no kernel record (" + path +
                              "): it was not written by a build, so its kernel cannot be checked");
  Reader r(file.f, path);
  char magic[8];
  int32_t head[2];
  r.get(magic, 8);
  r.get(head, sizeof head);
  if (std::memcmp(magic, kKernMagic, 8) != 0 || head[0] < 0 || head[0] > 1024)
    fail(MBF_ERR_IO, "corrupt kernel record: " + path);
  std::vector<KernelEntry> e = r.vec<KernelEntry>(head[0]);
  const uint64_t expect = r.sum();
  uint64_t stored = 0;
  if (std::fread(&stored, 1, 8, file.f) != 8 || stored != expect) fail(MBF_ERR_IO, "corrupt kernel record: " + path);
  return e;
}

}  // namespace

FactorSet build_or_load(const mbf_problem_t& prob, mbf_entry_fn fn, void* ctx, const mbf_build_opts_t& opts) {
  const char* path = opts.factor_file;
  if (!path || !*path) return build_factors(prob, fn, ctx, opts);
  if (FILE* probe = std::fopen(path, "rb")) {
    std::fclose(probe);
    FactorSet fs = load_factors(path);
    // the file must describe this problem: its dimension, depth, trees (point sets and
    // orders, which fix n and the tree kind) and ranks within r
    Tree xt, wt;
    problem_trees(prob, xt, wt);
    const std::string who = std::string("factor file ") + path + " was built for another problem: ";
    if (fs.d != prob.dim || fs.L != prob.L) fail(MBF_ERR_INVALID, who + "dim or L");
    const int64_t n_in = prob.tree == MBF_TREE_POINTS ? prob.n_w_pts : Tree::ipow(prob.n, prob.dim);
    if (fs.x_perm != xt.perm || fs.x_off != xt.off || fs.n_in != n_in)
      fail(MBF_ERR_INVALID, who + "X tree or grid size");
    if (fs.w_perm != wt.perm || fs.w_off != wt.off) fail(MBF_ERR_INVALID, who + "Omega tree or point set");
    for (int l = fs.L / 2; l <= fs.L; ++l)
      if (fs.RU[size_t(l)] > prob.r || fs.RV[size_t(l)] > prob.r) fail(MBF_ERR_INVALID, who + "ranks above r");
    // and the kernel: the recorded entries against the entry function of the problem being built
    const std::vector<KernelEntry> rec = load_kernel_record(std::string(path) + ".kernel");
    const std::vector<KernelEntry> now = kernel_entries(prob, fs, fn, ctx);
    bool same = rec.size() == now.size();
    for (size_t k = 0; same && k < rec.size(); ++k)
      same = rec[k].x == now[k].x && rec[k].xi == now[k].xi &&
             std::abs(rec[k].re - now[k].re) + std::abs(rec[k].im - now[k].im) <= 1e-9;
    if (!same) fail(MBF_ERR_INVALID, who + "kernel entries differ from the kernel record");
    return fs;
  }
  FactorSet fs = build_factors(prob, fn, ctx, opts);
  save_kernel_record(std::string(path) + ".kernel", prob.dim, kernel_entries(prob, fs, fn, ctx));
  save_factors(fs.view(), path);
  return fs;
}

}  // namespace mbf
