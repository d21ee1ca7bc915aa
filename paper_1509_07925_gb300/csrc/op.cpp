// Packer, resident operator and the C ABI of libmbf.
//
// The packer turns a padded FP64 factor set into the stage/item/chunk layout of
// layout.hpp: complex64 tiles with split real/imaginary planes, 128-byte aligned,
// the tree permutations kept as int32 index tables that the kernels fold into
// their leaf loads and stores, and M^h folded into the columns of the first G
// block (G^h_{c i + t, jp} diag(S^h_{i, c jp + tp}), §2.3 and eq. RSh2).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "apply.hpp"
#include "mbf_internal.hpp"

#include "op_internal.hpp"

namespace mbf {

namespace {
thread_local std::string g_last_error;

void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(MBF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Failure-detection test hook (mbf_debug_fail_alloc): while >= 0, the number of device
// allocations of this file still allowed to succeed; the next one fails as if the
// device were out of memory.
std::atomic<int64_t> g_alloc_budget{-1};

template <class T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  int64_t k = g_alloc_budget.load();
  while (k >= 0) {
    if (g_alloc_budget.compare_exchange_weak(k, k - 1)) {
      if (k == 0) {
        *p = nullptr;
        g_alloc_budget.store(-1);
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}

template <class T>
T* dev_upload(const std::vector<T>& v, const char* what) {
  T* p = nullptr;
  const size_t bytes = std::max<size_t>(sizeof(T), v.size() * sizeof(T));
  cudaError_t e = dev_alloc(&p, bytes);
  if (e != cudaSuccess) fail(MBF_ERR_OOM, std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e));
  if (!v.empty()) cuda_check(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), what);
  return p;
}

int64_t ipow(int64_t b, int e) { return Tree::ipow(b, e); }

struct Packer {
  const mbf_factors_t& f;
  int d, c, L, h;
  std::vector<uint8_t> arena;
  std::vector<Item> items;

  explicit Packer(const mbf_factors_t& fa) : f(fa) {}

  int64_t stage_nnz = 0, leaf_x_nnz = 0;   // nonzero entries packed (this stage; U^L items)

  // Append one item: `nlines` lines of `len` entries, value(line, e) -> complex.
  template <class F>
  Item add_item(int nlines, int len, uint8_t kind, uint8_t t, F value) {
    Item it{};
    size_t off = (arena.size() + 127) & ~size_t(127);
    if (off / 128 > UINT32_MAX) fail(MBF_ERR_INVALID, "factor arena larger than 512 GB");
    arena.resize(off, 0);
    it.off128 = uint32_t(off / 128);
    it.nlines = uint16_t(nlines);
    it.len = uint16_t(len);
    it.lpc = uint16_t(lines_per_chunk(len));
    it.kind = kind;
    it.t = t;
    const int64_t bytes = item_bytes(nlines, len, it.lpc);
    arena.resize(off + size_t(bytes), 0);
    uint8_t* p = arena.data() + off;
    for (int l0 = 0; l0 < nlines; l0 += it.lpc) {
      const int nl = std::min<int>(it.lpc, nlines - l0);
      float* re = reinterpret_cast<float*>(p);
      float* im = re + pad4(int64_t(nl) * len);
      for (int l = 0; l < nl; ++l)
        for (int e = 0; e < len; ++e) {
          const cd v = value(l0 + l, e);
          re[l * len + e] = float(v.real());
          im[l * len + e] = float(v.imag());
          if (v != cd(0.0, 0.0)) {
            ++stage_nnz;
            if (kind == ITEM_LEAF_X) ++leaf_x_nnz;
          }
        }
      p += chunk_bytes(nl, len);
    }
    return it;
  }

  // Main item of a group: c Rin lines (input entry (t, k) is line t Rin + k) of c Rout
  // entries.  In a compact stage only the first r_t lines of each input segment t are
  // stored, r_t = 1 + its last line holding a nonzero entry (0: none), with the c = 4
  // counts in the item's base, one byte each.
  template <class F>
  Item add_main(const Stage& st, int Rin, int Rout, F value) {
    if (!st.compact) return add_item(c * Rin, c * Rout, ITEM_MAIN, 0, value);
    std::vector<int> lines;
    uint32_t counts = 0;
    for (int t = 0; t < c; ++t) {
      int r = 0;
      for (int k = Rin - 1; k >= 0 && r == 0; --k)
        for (int e = 0; e < c * Rout; ++e)
          if (value(t * Rin + k, e) != cd(0.0, 0.0)) {
            r = k + 1;
            break;
          }
      for (int k = 0; k < r; ++k) lines.push_back(t * Rin + k);
      counts |= uint32_t(r) << (8 * t);
    }
    Item it = add_item(int(lines.size()), c * Rout, ITEM_MAIN, 0,
                       [&](int line, int e) { return value(lines[size_t(line)], e); });
    it.base = int32_t(counts);
    return it;
  }

  void run(mbf_op_s& op) {
    d = f.dim;
    L = f.L;
    c = 1 << d;
    h = L / 2;
    const int64_t nL = ipow(c, L);
    const int32_t* RU = f.RU;
    const int32_t* RV = f.RV;
    auto cplx = [](const double* a, int64_t i) { return cd(a[2 * i], a[2 * i + 1]); };
    Plan& plan = op.plan;
    plan = Plan{};
    plan.c = c;
    plan.d = d;
    plan.L = L;
    int ns = 0;
    auto begin_stage = [&](int level, int side) -> Stage& {
      Stage& st = plan.st[ns++];
      st.level = level;
      st.side = side;
      st.n_groups = int32_t(ipow(c, L - 1));
      st.B = int32_t(ipow(c, L - level - 1));
      st.ch = int32_t(ipow(c, h));
      st.item_base = int64_t(items.size());
      st.compact = c == 4 ? 1 : 0;   // r_t <= 64 fits a byte; four bytes fit the base
      return st;
    };
    // ---- leaf stage: (V^L_j)^* for the c leaves of each group, written to the
    // coefficient vector of level L (leaf j at position j * RV[L])
    {
      Stage& st = begin_stage(L, 1);
      st.B = 1;
      st.R_in = RV[L];
      st.R_out = RV[L];
      st.in_pat = PAT_LEAF;
      st.out_pat = PAT_CONTIG;
      st.n_items = 1;
      st.main_idx = -1;
      st.leaf_only = 1;
      st.compact = 0;
      const size_t a0 = arena.size();
      for (int64_t g = 0; g < st.n_groups; ++g) {
        // all points of the group's c leaves in one item: line = a point (tree order),
        // entry k = column k of its leaf's V^L
        const int64_t p0 = f.w_off[c * g], p1 = f.w_off[c * g + c];
        items.push_back(add_item(int(p1 - p0), RV[L], ITEM_LEAF_W, 0, [&](int b, int k) {
          int64_t leaf = c * g;
          while (f.w_off[leaf + 1] <= p0 + b) ++leaf;
          const int64_t row = p0 + b - f.w_off[leaf];
          return std::conj(cplx(f.VL, (leaf * f.max_leaf_w + row) * RV[L] + k));
        }));
        items.back().base = int32_t(p0);
      }
      st.bytes = int64_t(arena.size() - a0);
      op.nnz_stage.push_back(stage_nnz);
      stage_nnz = 0;
    }
    // ---- H-stages l = L-1 .. h: (H^l)^*
    for (int l = L - 1; l >= h; --l) {
      Stage& st = begin_stage(l, 1);
      const int R2 = RV[l + 1], R1 = RV[l];
      st.R_in = R2;
      st.R_out = R1;
      st.in_pat = PAT_SPLIT;
      st.out_pat = PAT_CONTIG;
      st.n_items = 1;
      st.main_idx = 0;
      const double* Hl = f.H[l - h];
      const size_t a0 = arena.size();
      for (int64_t g = 0; g < st.n_groups; ++g) {
        // T[(tp,k)][(t,k2)] = conj(H^l_{c j + t, ip}[k2][(tp,k)]), lines = (t,k2)
        items.push_back(add_main(st, R2, R1, [&](int line, int e) {
          const int t = line / R2, k2 = line % R2, tp = e / R1, k = e % R1;
          return std::conj(cplx(Hl, ((((g * c + t) * R2 + k2) * c + tp) * R1) + k));
        }));
      }
      st.bytes = int64_t(arena.size() - a0);
      op.nnz_stage.push_back(stage_nnz);
      stage_nnz = 0;
    }
    // ---- G-stages l = h .. L-1: G^l, the first with M^h folded in, the last fused with U^L
    for (int l = h; l < L; ++l) {
      Stage& st = begin_stage(l, 0);
      const int R1 = RU[l], R2 = RU[l + 1];
      st.R_in = R1;
      st.R_out = R2;
      st.in_pat = l == h ? PAT_CORNER : PAT_CONTIG;
      st.out_pat = l == L - 1 ? PAT_LEAF : PAT_SPLIT;
      const bool leaves = l == L - 1;
      st.n_items = leaves ? 2 : 1;
      st.main_idx = 0;
      const double* Gl = f.G[l - h];
      const int64_t B = st.B, ch = st.ch;
      const size_t a0 = arena.size();
      for (int64_t g = 0; g < st.n_groups; ++g) {
        const int64_t i = g / B, jp = g % B;
        items.push_back(add_main(st, R1, R2, [&](int line, int e) {
          const int tp = line / R1, k = line % R1, t = e / R2, k2 = e % R2;
          cd v = cplx(Gl, ((((g * c + t) * R2 + k2) * c + tp) * R1) + k);
          if (l == h) v *= f.S[(i * ch + (c * jp + tp)) * R1 + k];
          return v;
        }));
        if (leaves) {
          // U^L_i for the c leaves i = c g + t in one item, stored by columns: line = a
          // column k (an input of the leaf products), entry a = a point of the group
          const int64_t p0 = f.x_off[c * g], p1 = f.x_off[c * g + c];
          const int np = int(p1 - p0);
          items.push_back(add_item(np > 0 ? RU[L] : 0, std::max(np, 1), ITEM_LEAF_X, 0, [&](int k, int a) {
            int64_t leaf = c * g;
            while (f.x_off[leaf + 1] <= p0 + a) ++leaf;
            const int64_t row = p0 + a - f.x_off[leaf];
            return cplx(f.UL, (leaf * f.max_leaf_x + row) * RU[L] + k);
          }));
          items.back().base = int32_t(p0);
        }
      }
      st.bytes = int64_t(arena.size() - a0);
      op.nnz_stage.push_back(stage_nnz);
      stage_nnz = 0;
    }
    plan.n_stages = ns;
    (void)nL;
  }
};

// ---------------------------------------------------------------- tensor-core packing
uint16_t bf16_rn(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  return uint16_t((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}
float bf16_to_float(uint16_t h) {
  const uint32_t u = uint32_t(h) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Split-bf16 tiles of every G^l / (H^l)^* group product (the main stages of the SIMT
// plan; the last G stage writes the level-L coefficient vector instead of applying U^L).
// Ranks are rounded up to R8 (a multiple of 8) with zero rows and columns, so that every
// tree-node pair owns a whole number of 8-row core matrices.  Tile element (m, k) of a
// group = output entry m = (t, k2), input entry k = (tp, kk), with m = t R8_out + k2 and
// k = tp R8_in + kk; value x (FP64) is stored as hi = bf16(x), lo = bf16(x - hi) for the
// real and imaginary parts, each plane K-major in 8 x 8 core matrices.
void pack_tc(const mbf_factors_t& f, const Plan& sp, TCPlan& tp, std::vector<uint8_t>& arena, int& mt_max,
             int& kpad_max) {
  const int c = 1 << f.dim, L = f.L, h = L / 2;
  auto cplx = [](const double* a, int64_t i) { return cd(a[2 * i], a[2 * i + 1]); };
  auto r8 = [](int r) { return (r + 7) & ~7; };
  tp = TCPlan{};
  tp.c = c;
  tp.d = f.dim;
  tp.L = L;
  mt_max = 16;
  kpad_max = 16;
  int n = 0;
  for (int e = 1; e < sp.n_stages; ++e) {
    const Stage& st = sp.st[e];
    TCStage& ts = tp.st[n++];
    ts.n_groups = st.n_groups;
    ts.R_in = st.R_in;
    ts.R_out = st.R_out;
    ts.R8_in = r8(st.R_in);
    ts.R8_out = r8(st.R_out);
    ts.M_t = c * ts.R8_out;
    ts.K_t = c * ts.R8_in;
    if (ts.M_t > kTcMaxRows || ts.K_t > kTcMaxK) fail(MBF_ERR_INVALID, "tile too large for the tensor path");
    ts.K_pad = (ts.K_t + 15) & ~15;
    ts.in_pat = st.in_pat;
    ts.last = e == sp.n_stages - 1;
    ts.out_pat = st.out_pat == PAT_LEAF ? PAT_SPLIT : st.out_pat;   // B = 1: writes block c g + t
    ts.B = st.B;
    ts.ch = st.ch;
    ts.plane_bytes = ts.M_t * 32;
    ts.tile_bytes = int64_t(ts.K_pad / 16) * 4 * ts.plane_bytes;
    size_t base = (arena.size() + 127) & ~size_t(127);
    ts.base = int64_t(base);
    arena.resize(base + size_t(ts.tile_bytes) * size_t(ts.n_groups), 0);
    mt_max = std::max(mt_max, ts.M_t);
    kpad_max = std::max(kpad_max, ts.K_pad);
    const int l = st.level, R1 = st.side == 1 ? f.RV[l] : f.RU[l], R2 = st.side == 1 ? f.RV[l + 1] : f.RU[l + 1];
    const double* M = st.side == 1 ? f.H[l - h] : f.G[l - h];
    for (int64_t g = 0; g < ts.n_groups; ++g) {
      uint8_t* tile = arena.data() + base + size_t(g) * size_t(ts.tile_bytes);
      const int64_t i = g / st.B, jp = g % st.B;
      for (int m = 0; m < ts.M_t; ++m)
        for (int k = 0; k < ts.K_t; ++k) {
          const int mo = m / ts.R8_out, mi = m % ts.R8_out, ko = k / ts.R8_in, ki = k % ts.R8_in;
          if (mi >= ts.R_out || ki >= ts.R_in) continue;   // zero padding
          cd v;
          if (st.side == 1) {   // T[(tp,k)][(t,k2)] = conj(H^l_{c j + t, ip}[k2][(tp,k)])
            const int tp_ = mo, kk = mi, t = ko, k2 = ki;
            v = std::conj(cplx(M, ((((g * c + t) * R2 + k2) * c + tp_) * R1) + kk));
          } else {              // T[(t,k2)][(tp,k)] = G^l_{c i + t, jp}[k2][(tp,k)] (x S^h at l = h)
            const int t = mo, k2 = mi, tp_ = ko, kk = ki;
            v = cplx(M, ((((g * c + t) * R2 + k2) * c + tp_) * R1) + kk);
            if (l == h) v *= f.S[(i * st.ch + (c * jp + tp_)) * R1 + kk];
          }
          const float re = float(v.real()), im = float(v.imag());
          const uint16_t rh = bf16_rn(re), ih = bf16_rn(im);
          const uint16_t rl = bf16_rn(float(v.real() - double(bf16_to_float(rh))));
          const uint16_t il = bf16_rn(float(v.imag() - double(bf16_to_float(ih))));
          const uint16_t vals[4] = {rh, ih, rl, il};   // planes: Re hi, Im hi, Re lo, Im lo
          const int kk16 = k / 16, kc = k % 16;
          const size_t in_plane = size_t(((m / 8) * 2 + kc / 8) * 128 + (m % 8) * 16 + (kc % 8) * 2);
          for (int pl = 0; pl < 4; ++pl)
            std::memcpy(tile + size_t(kk16 * 4 + pl) * size_t(ts.plane_bytes) + in_plane, &vals[pl], 2);
        }
    }
  }
  tp.n_stages = n;
}

// The tensor adjoint's plan: stage e of it is forward stage S - 1 - e with its tile
// conjugate-transposed (M_t <-> K_t), reading where the forward stage writes and writing
// where it reads (same pattern parameters).  Throws where a forward tile's shape has no
// adjoint tile of the same bytes (K_pad != K_t).
void adjoint_tile_plan(const TCPlan& fp, TCPlan& ap) {
  ap = fp;
  for (int e = 0; e < fp.n_stages; ++e) {
    const TCStage& fs = fp.st[fp.n_stages - 1 - e];
    TCStage& as = ap.st[e];
    as = fs;
    as.M_t = fs.K_t;
    as.K_t = fs.M_t;
    as.K_pad = fs.M_t;
    as.in_pat = fs.out_pat;
    as.out_pat = fs.in_pat;
    as.R_in = fs.R_out;
    as.R_out = fs.R_in;
    as.R8_in = fs.R8_out;
    as.R8_out = fs.R8_in;
    as.plane_bytes = as.M_t * 32;
    as.last = e == fp.n_stages - 1;
    if (fs.K_pad != fs.K_t || as.M_t > kTcMaxRows || as.K_pad % 16 != 0 ||
        int64_t(as.K_pad / 16) * 4 * as.plane_bytes != fs.tile_bytes)
      fail(MBF_ERR_INVALID, "tile shape not supported by the tensor adjoint");
  }
}

void validate_factors(const mbf_factors_t& f) {
  if (f.dim != 2 && f.dim != 3) fail(MBF_ERR_INVALID, "dim must be 2 or 3");
  if (f.L < 2 || f.L % 2 || f.L > 20) fail(MBF_ERR_INVALID, "L must be even, 2..20");
  const int c = 1 << f.dim, h = f.L / 2;
  if (2 * (f.L - h) + 1 > kMaxStages) fail(MBF_ERR_INVALID, "too many stages");
  if (!f.x_perm || !f.x_off || !f.w_perm || !f.w_off || !f.RU || !f.RV || !f.UL || !f.VL || !f.G ||
      !f.H || !f.S)
    fail(MBF_ERR_INVALID, "factor set has a NULL array");
  if (f.RU[h] != f.RV[h]) fail(MBF_ERR_INVALID, "RU[h] must equal RV[h]");
  for (int l = h; l <= f.L; ++l) {
    if (f.RU[l] < 1 || f.RV[l] < 1) fail(MBF_ERR_INVALID, "ranks must be >= 1");
    if (int64_t(c) * f.RU[l] > kMaxLen || int64_t(c) * f.RV[l] > kMaxLen)
      fail(MBF_ERR_INVALID, "c * rank exceeds " + std::to_string(kMaxLen));
  }
  if (int64_t(c) * f.max_leaf_x > 65535 || int64_t(c) * f.max_leaf_w > 65535)
    fail(MBF_ERR_INVALID, "the leaves of a group hold more than 65535 points");
  const int64_t nL = Tree::ipow(c, f.L);
  if (f.x_off[0] != 0 || f.x_off[nL] != f.n_out) fail(MBF_ERR_INVALID, "x_off must span n_out");
  if (f.w_off[0] != 0 || f.w_off[nL] != f.n_w) fail(MBF_ERR_INVALID, "w_off must span n_w");
  for (int64_t q = 0; q < nL; ++q) {
    if (f.x_off[q + 1] - f.x_off[q] > f.max_leaf_x || f.x_off[q + 1] < f.x_off[q])
      fail(MBF_ERR_INVALID, "x_off inconsistent with max_leaf_x");
    if (f.w_off[q + 1] - f.w_off[q] > f.max_leaf_w || f.w_off[q + 1] < f.w_off[q])
      fail(MBF_ERR_INVALID, "w_off inconsistent with max_leaf_w");
  }
  std::vector<char> seen(size_t(f.n_out), 0);
  for (int64_t q = 0; q < f.n_out; ++q) {
    const int64_t v = f.x_perm[q];
    if (v < 0 || v >= f.n_out || seen[size_t(v)]) fail(MBF_ERR_INVALID, "x_perm is not a permutation");
    seen[size_t(v)] = 1;
  }
  std::vector<char> seenw(size_t(f.n_in), 0);
  for (int64_t q = 0; q < f.n_w; ++q) {
    const int64_t v = f.w_perm[q];
    if (v < 0 || v >= f.n_in || seenw[size_t(v)]) fail(MBF_ERR_INVALID, "w_perm: index out of range or repeated");
    seenw[size_t(v)] = 1;
  }
  if (f.n_out > INT32_MAX || f.n_in > INT32_MAX) fail(MBF_ERR_INVALID, "too many points");
}

// Host check of the packed plan, run before any device work: every gather and
// scatter the kernels will do stays inside the coefficient workspace, the positions
// each stage writes are exactly those the next stage reads (so forward and adjoint
// never read an unwritten entry), and every item lies inside the arena with the
// shape its stage expects.
int64_t host_pat_off(int pat, int64_t g, int t, const Stage& s, int64_t R, int c) {
  const int64_t a = g / s.B, b = g % s.B;
  if (pat == PAT_SPLIT) return ((c * a + t) * s.B + b) * R;
  if (pat == PAT_CONTIG) return (int64_t(c) * g + t) * R;
  return ((c * b + t) * int64_t(s.ch) + a) * R;
}
// group of stage s whose input pattern reads segment P (the kernel's consumer map)
int64_t host_pat_group(int pat, int64_t P, const Stage& s, int c) {
  if (pat == PAT_CONTIG) return P / c;
  if (pat == PAT_SPLIT) return (P / s.B / c) * s.B + P % s.B;
  return (P % s.ch) * s.B + (P / s.ch) / c;
}

// The kernel replaces grid barriers by counting: each group adds 1 to the counter of
// the consumer of each of its c output segments and a consumer starts at c.  Check,
// forward and adjoint, that every consumer is told exactly c times and that the
// group named for a segment is the one whose gather reads it.
void check_dependencies(const Plan& plan) {
  const int c = plan.c, S = plan.n_stages;
  for (int adj = 0; adj < 2; ++adj) {
    for (int e = 0; e + 1 < S; ++e) {
      const Stage& st = plan.st[adj ? S - 1 - e : e];
      const Stage& nx = plan.st[adj ? S - 2 - e : e + 1];
      const int out_pat = adj ? st.in_pat : st.out_pat, in_pat = adj ? nx.out_pat : nx.in_pat;
      const int64_t Rout = adj ? st.R_in : st.R_out, Rin = adj ? nx.R_out : nx.R_in;
      if (in_pat == PAT_LEAF || out_pat == PAT_LEAF) fail(MBF_ERR_INVALID, "plan: leaf pattern between stages");
      if (Rout != Rin) fail(MBF_ERR_INVALID, "plan: segment lengths differ between stages");
      std::vector<int> cnt(size_t(nx.n_groups), 0);
      for (int64_t g = 0; g < st.n_groups; ++g)
        for (int t = 0; t < c; ++t) {
          const int64_t P = host_pat_off(out_pat, g, t, st, Rout, c) / Rout;
          const int64_t h = host_pat_group(in_pat, P, nx, c);
          if (h < 0 || h >= nx.n_groups) fail(MBF_ERR_INVALID, "plan: consumer group out of range");
          bool reads = false;
          for (int tt = 0; tt < c; ++tt) reads |= host_pat_off(in_pat, h, tt, nx, Rin, c) == P * Rin;
          if (!reads) fail(MBF_ERR_INVALID, "plan: consumer map names a group that does not read the segment");
          ++cnt[size_t(h)];
        }
      for (int v : cnt)
        if (v != c) fail(MBF_ERR_INVALID, "plan: a consumer group is not fed by exactly c segments");
    }
  }
}

// Limits that only the SIMT kernel has (its leaf gathers and pipeline slots) are
// returned in *simt_reason instead of failing: such an operator applies on the tensor
// cores only.
void check_plan(const Plan& plan, const std::vector<Item>& items, size_t arena_bytes, int64_t positions,
                const mbf_factors_t& f, std::string* simt_reason) {
  const int c = plan.c;
  if (f.max_leaf_x > kMaxLeaf || f.max_leaf_w > kMaxLeaf)
    *simt_reason = "a leaf holds more than " + std::to_string(kMaxLeaf) + " points";
  check_dependencies(plan);
  std::vector<char> wrote, read;
  for (int e = 0; e < plan.n_stages; ++e) {
    const Stage& st = plan.st[e];
    std::vector<char> rd(size_t(positions), 0), wr(size_t(positions), 0);
    auto mark = [&](int pat, int R, std::vector<char>& bm) {
      if (pat == PAT_LEAF) return;
      for (int64_t g = 0; g < st.n_groups; ++g)
        for (int t = 0; t < c; ++t) {
          const int64_t a = g / st.B, b = g % st.B;
          int64_t off;
          if (pat == PAT_SPLIT) off = ((c * a + t) * st.B + b) * R;
          else if (pat == PAT_CONTIG) off = (int64_t(c) * g + t) * R;
          else off = ((c * b + t) * int64_t(st.ch) + a) * R;
          if (off < 0 || off + R > positions) fail(MBF_ERR_INVALID, "plan: vector offset out of range");
          for (int k = 0; k < R; ++k) {
            if (bm[size_t(off + k)]) fail(MBF_ERR_INVALID, "plan: position touched twice in one stage");
            bm[size_t(off + k)] = 1;
          }
        }
    };
    mark(st.in_pat, st.R_in, rd);
    mark(st.out_pat, st.R_out, wr);
    if (e > 0 && st.in_pat != PAT_LEAF && rd != wrote)
      fail(MBF_ERR_INVALID, "plan: stage reads differ from the previous stage's writes");
    wrote = wr;
    const int64_t nL = Tree::ipow(c, plan.L);
    if (st.n_items > 32) fail(MBF_ERR_INVALID, "plan: more than 32 items in a group");
    if (st.in_pat == PAT_LEAF || st.out_pat == PAT_LEAF) {
      const int64_t* off = st.in_pat == PAT_LEAF ? f.w_off : f.x_off;
      for (int64_t g = 0; g < st.n_groups; ++g)
        if (off[c * g + c] - off[c * g] > kMaxGroupPoints)
          *simt_reason = "the leaves of one group hold more than " + std::to_string(kMaxGroupPoints) + " points";
    }
    for (int64_t g = 0; g < st.n_groups; ++g)
      for (int m = 0; m < st.n_items; ++m) {
        const Item& it = items[size_t(st.item_base + g * st.n_items + m)];
        if (size_t(it.off128) * 128 + size_t(item_bytes(it.nlines, it.len, it.lpc)) > arena_bytes)
          fail(MBF_ERR_INVALID, "plan: item outside the arena");
        if (chunk_bytes(std::min<int64_t>(it.lpc, std::max<int64_t>(it.nlines, 1)), it.len) > kSlotBytes ||
            it.len > kMaxLen || (it.kind != ITEM_MAIN && it.nlines > kMaxLeaf))
          *simt_reason = "an item line or chunk exceeds the SIMT kernel's pipeline slot";
        const int64_t leaf = c * g;
        if (it.kind == ITEM_MAIN) {
          int64_t lines = int64_t(c) * st.R_in;
          if (st.compact) {
            if (c != 4) fail(MBF_ERR_INVALID, "plan: compact stage with c != 4");
            lines = 0;
            for (int t = 0; t < c; ++t) {
              if (seg_lines(it.base, t) > st.R_in) fail(MBF_ERR_INVALID, "plan: segment line count above the rank");
              lines += seg_lines(it.base, t);
            }
          }
          if (it.nlines != lines || it.len != c * st.R_out) fail(MBF_ERR_INVALID, "plan: main block shape");
        } else if (it.kind == ITEM_LEAF_W) {
          if (st.in_pat != PAT_LEAF || leaf + c > nL || it.len != st.R_in ||
              it.nlines != f.w_off[leaf + c] - f.w_off[leaf] || it.base != f.w_off[leaf])
            fail(MBF_ERR_INVALID, "plan: Omega leaf item");
        } else if (it.kind == ITEM_LEAF_X) {
          const int64_t np = f.x_off[leaf + c] - f.x_off[leaf];
          if (st.out_pat != PAT_LEAF || leaf + c > nL || it.len != std::max<int64_t>(np, 1) ||
              it.nlines != (np > 0 ? st.R_out : 0) || it.base != f.x_off[leaf])
            fail(MBF_ERR_INVALID, "plan: X leaf item");
        } else {
          fail(MBF_ERR_INVALID, "plan: unknown item kind");
        }
      }
  }
}

void op_free(mbf_op_s* op) {
  if (!op) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(op->device);
  for (Workspace* w : op->ws_pool) {
    ws_free(*w);
    delete w;
  }
  cudaFree(op->d_arena);
  cudaFree(op->d_items);
  cudaFree(op->d_x_perm);
  cudaFree(op->d_x_off);
  cudaFree(op->d_w_perm);
  cudaFree(op->d_w_off);
  cudaFree(op->d_x_nat);
  cudaFree(op->d_w_nat);
  ws_free(op->ws);
  cudaFree(op->d_stage_in);
  cudaFree(op->d_stage_out);
  for (int b = 0; b < 2; ++b) {
    cudaFree(op->d_pipe_in[b]);
    cudaFree(op->d_pipe_out[b]);
    if (op->pipe_st[b]) cudaStreamDestroy(op->pipe_st[b]);
    for (auto& ev : op->pipe_ev)
      if (ev[b]) cudaEventDestroy(ev[b]);
  }
  cudaFree(op->d_tc_arena);
  cudaFree(op->d_tc_arena_tf32);
  cudaFree(op->d_tc_arena_adj);
  cudaFree(op->d_x_inv);
  for (auto& r : op->prof_pending) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  cudaFree(op->d_w_inv);
  cudaSetDevice(prev);
  delete op;
}

std::atomic<uint64_t> g_op_serial{0};

mbf_op_s* op_create(const mbf_factors_t& f) {
  validate_factors(f);
  auto* op = new mbf_op_s();
  op->serial = ++g_op_serial;
  try {
    op->d = f.dim;
    op->c = 1 << f.dim;
    op->L = f.L;
    op->h = f.L / 2;
    op->n_out = f.n_out;
    op->n_in = f.n_in;
    op->n_w = f.n_w;
    op->RU.assign(f.RU, f.RU + f.L + 1);
    op->RV.assign(f.RV, f.RV + f.L + 1);
    op->nnz = f.nnz;
    Packer pk(f);
    pk.run(*op);
    op->nnz_leaf_x = pk.leaf_x_nnz;
    op->bytes_packed = int64_t(pk.arena.size());
    if (op->nnz <= 0)   // not given with the factors: the nonzero entries packed
      for (int64_t v : op->nnz_stage) op->nnz += v;
    int64_t rmax = 1;
    for (int l = op->h; l <= op->L; ++l) rmax = std::max<int64_t>({rmax, op->RU[size_t(l)], op->RV[size_t(l)]});
    op->positions = Tree::ipow(op->c, op->L) * rmax;
    check_plan(op->plan, pk.items, pk.arena.size(), op->positions, f, &op->simt_unavailable);
    // ---- device side
    cuda_check(cudaGetDevice(&op->device), "cudaGetDevice");
    op->d_arena = dev_upload(pk.arena, "factor arena");
    op->d_items = dev_upload(pk.items, "item table");
    auto to32 = [](const int64_t* p, int64_t n) {
      std::vector<int32_t> v(static_cast<size_t>(n));
      for (int64_t q = 0; q < n; ++q) v[size_t(q)] = int32_t(p[q]);
      return v;
    };
    const int64_t nL = Tree::ipow(op->c, op->L);
    for (int64_t q = 0; q < nL; ++q) {
      op->leaf_pts_x = std::max(op->leaf_pts_x, f.x_off[q + 1] - f.x_off[q]);
      op->leaf_pts_w = std::max(op->leaf_pts_w, f.w_off[q + 1] - f.w_off[q]);
    }
    // a tree whose largest group of c leaves holds more than twice the mean of the
    // non-empty groups gets one CTA per leaf in the leaf kernels of its U^L side
    auto ragged = [&](const int64_t* off) {
      int64_t mx = 0, tot = 0, ne = 0;
      for (int64_t gq = 0; gq < nL / op->c; ++gq) {
        const int64_t np = off[(gq + 1) * op->c] - off[gq * op->c];
        mx = std::max(mx, np);
        tot += np;
        ne += np > 0;
      }
      return ne > 0 && mx * ne > 2 * tot;
    };
    op->split_x = ragged(f.x_off) ? 1 : 0;
    op->split_w = ragged(f.w_off) ? 1 : 0;
    op->d_x_perm = dev_upload(to32(f.x_perm, f.n_out), "x_perm");
    op->d_x_off = dev_upload(to32(f.x_off, nL + 1), "x_off");
    op->d_w_perm = dev_upload(to32(f.w_perm, std::max<int64_t>(f.n_w, 1)), "w_perm");
    op->d_w_off = dev_upload(to32(f.w_off, nL + 1), "w_off");
    auto nat_table = [&](const int64_t* perm, const int64_t* off, int64_t max_pts, int32_t* stride) {
      *stride = int32_t(std::max<int64_t>(8, (max_pts + 7) & ~int64_t(7)));
      std::vector<int32_t> t(size_t(nL) * size_t(*stride), 0);
      for (int64_t q = 0; q < nL; ++q)
        for (int64_t b = off[q]; b < off[q + 1]; ++b) t[size_t(q) * size_t(*stride) + size_t(b - off[q])] = int32_t(perm[b]);
      return t;
    };
    op->d_x_nat = dev_upload(nat_table(f.x_perm, f.x_off, op->leaf_pts_x, &op->x_nat_stride), "X leaf index table");
    op->d_w_nat = dev_upload(nat_table(f.w_perm, f.w_off, op->leaf_pts_w, &op->w_nat_stride), "Omega leaf index table");
    ws_init(op, op->ws);
    for (int nrb : {1, 2, 4}) cuda_check(simt_config(nrb, &op->grid, &op->ns[nrb], &op->smem[nrb]), "simt_config");
    cuda_check(cudaDeviceGetAttribute(&op->sms, cudaDevAttrMultiProcessorCount, op->device), "attr");
    // tensor-core tiles (the multi-RHS path); an operator whose tiles do not fit keeps
    // the SIMT path only and says why
    try {
      std::vector<uint8_t> tc_arena;
      pack_tc(f, op->plan, op->tcplan, tc_arena, op->tc_mt_max, op->tc_kpad_max);
      const Stage& first = op->plan.st[0];
      const Stage& last = op->plan.st[op->plan.n_stages - 1];
      if (op->plan.n_stages < 2 || first.n_items != 1 || last.n_items != 2 || last.B != 1 ||
          op->tcplan.st[0].in_pat != PAT_SPLIT || op->tcplan.st[0].B != 1)
        fail(MBF_ERR_INVALID, "plan shape not supported by the tensor path");
      int optin = 0;
      cuda_check(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, op->device), "attr");
      if (!leaf_fits(op->tcplan.st[0].R8_in, op->c) || leaf_smem_bytes(op->RU[size_t(op->L)], op->c, true) > size_t(optin) ||
          leaf_smem_bytes(op->RV[size_t(op->L)], op->c, false) > size_t(optin))
        fail(MBF_ERR_INVALID, "leaf rank too large for the tensor path");
      // accumulator sets (2 M_t TMEM columns each), panel buffers, A ring slots; more
      // than half the SM's shared memory, so one CTA per SM and each CTA's 512-column
      // TMEM allocation never waits on another CTA of the same launch
      auto config = [&](int mt, int kp, int& nsets, int& nxb, int& nsa, size_t& sm) {
        nsets = 4 * mt <= 512 ? 2 : 1;
        nxb = 2;
        auto smem = [&](int n) { return tc_smem_bytes(n, nxb, nsets, mt, kp); };
        if (smem(2) > size_t(optin)) nxb = 1;
        if (smem(2) > size_t(optin)) fail(MBF_ERR_INVALID, "tiles too large for the tensor path");
        nsa = 2;   // a multiple of the tile stream's producer lanes (2)
        while (nsa + 2 <= 16 && smem(nsa + 2) <= size_t(optin)) nsa += 2;
        sm = std::max(smem(nsa), size_t(optin) / 2 + 1024);
      };
      config(op->tc_mt_max, op->tc_kpad_max, op->tc_nsets, op->tc_nxb, op->tc_nsa, op->tc_smem);
      // the tensor adjoint: its plan (adjoint_tile_plan) and launch configuration
      try {
        const TCPlan& ap = op->tcplan_adj;
        adjoint_tile_plan(op->tcplan, op->tcplan_adj);
        op->tca_mt_max = op->tc_kpad_max;
        op->tca_kpad_max = op->tc_mt_max;
        if (!leaf_fits(ap.st[0].R8_in, op->c) || leaf_smem_bytes(op->RV[size_t(op->L)], op->c, true) > size_t(optin) ||
            leaf_smem_bytes(op->RU[size_t(op->L)], op->c, false) > size_t(optin))
          fail(MBF_ERR_INVALID, "leaf rank too large for the tensor adjoint");
        config(op->tca_mt_max, op->tca_kpad_max, op->tca_nsets, op->tca_nxb, op->tca_nsa, op->tca_smem);
        std::vector<int32_t> xinv(size_t(std::max<int64_t>(f.n_out, 1)), -1);
        for (int64_t p = 0; p < f.n_out; ++p) xinv[size_t(f.x_perm[p])] = int32_t(p);
        op->d_x_inv = dev_upload(xinv, "inverse X permutation");
      } catch (const Error& err) {
        op->tc_adj_unavailable = err.what();
      }
      std::vector<int32_t> winv(size_t(std::max<int64_t>(f.n_in, 1)), -1);
      for (int64_t p = 0; p < f.n_w; ++p) winv[size_t(f.w_perm[p])] = int32_t(p);
      op->d_w_inv = dev_upload(winv, "inverse Omega permutation");
      op->tc_bytes = int64_t(tc_arena.size());
      op->d_tc_arena = dev_upload(tc_arena, "tensor-core arena");
    } catch (const Error& err) {
      op->tc_unavailable = err.what();
    }
    if (!op->simt_unavailable.empty() && !op->tc_unavailable.empty())
      fail(MBF_ERR_INVALID, "no apply path: SIMT (" + op->simt_unavailable + "), tensor cores (" + op->tc_unavailable + ")");
  } catch (...) {
    op_free(op);
    throw;
  }
  return op;
}

// ---------------------------------------------------------------- kernel timing
enum ProfKind { PK_SIMT = 0, PK_PERMUTE, PK_LEAF_V, PK_TC, PK_LEAF_U, PK_COUNT };
const char* const kProfNames[PK_COUNT] = {"bf_apply_simt", "permute_in", "leaf_v", "bf_apply_tc", "leaf_u"};

// Records an event before a launch when profiling is on (nullptr otherwise).
cudaEvent_t prof_begin(mbf_op_s* op, cudaStream_t st) {
  if (!op->prof_on) return nullptr;
  cudaEvent_t e = nullptr;
  cuda_check(cudaEventCreate(&e), "cudaEventCreate");
  cuda_check(cudaEventRecord(e, st), "cudaEventRecord");
  return e;
}
void prof_end(mbf_op_s* op, int kind, cudaEvent_t e0, cudaStream_t st) {
  if (!e0) return;
  cudaEvent_t e1 = nullptr;
  cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
  cuda_check(cudaEventRecord(e1, st), "cudaEventRecord");
  op->prof_pending.push_back({kind, e0, e1});
}
void prof_collect(mbf_op_s* op) {
  for (auto& r : op->prof_pending) {
    float ms = 0.f;
    const cudaError_t err = cudaEventSynchronize(r.e1);
    if (err == cudaSuccess && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
      op->prof_ms[r.kind] += ms;
      op->prof_launches[r.kind] += 1;
    }
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  op->prof_pending.clear();
}

// Tensor-core apply, per panel of 64 RHS: permute the panel into Omega-tree order, the
// (V^L)^* leaf kernel, the persistent tcgen05 kernel over the G / H levels, the U^L leaf
// kernel (which scatters u to natural order).
void apply_tc(mbf_op_s* op, Workspace& w, const float2* g, float2* u, int64_t nrhs, cudaStream_t st, int grid, bool accumulate,
              bool host_io, bool tf32, const RowTable* rows = nullptr) {
  if (!op->tc_unavailable.empty()) fail(MBF_ERR_INVALID, "tensor path unavailable: " + op->tc_unavailable);
  const TCPlan& tp = op->tcplan;
  const int S = tp.n_stages;
  const int64_t vec_bytes = tc_vec_bytes(op);
  ws_prepare_tc(op, w);
  if (tf32 && !op->d_tc_arena_tf32) {   // first TF32 apply: convert the tiles (kept, like the split ones)
    if (dev_alloc(&op->d_tc_arena_tf32, size_t(op->tc_bytes)) != cudaSuccess) {
      op->d_tc_arena_tf32 = nullptr;
      fail(MBF_ERR_OOM, "cudaMalloc TF32 tiles");
    }
    for (int e = 0; e < S; ++e) {
      const TCStage& ts = tp.st[e];
      cuda_check(launch_tf32_tiles(op->d_tc_arena + ts.base, op->d_tc_arena_tf32 + ts.base,
                                   int64_t(ts.n_groups) * (ts.K_pad / 16), ts.M_t, st),
                 "TF32 tile conversion");
    }
  }
  int sms = op->sms;
  if (grid > 0) sms = std::min(sms, grid);
  const Stage& leaf_st = op->plan.st[0];
  const Stage& last_st = op->plan.st[op->plan.n_stages - 1];
  uint8_t* yl = w.tc_bufs;                       // level-L input of the main stages
  uint8_t* bufs = yl + vec_bytes;                    // main stage e < S - 1 writes bufs + e * vec_bytes
  float* ylast = reinterpret_cast<float*>(yl + int64_t(S) * vec_bytes);   // last main stage
  for (int64_t r0 = 0; r0 < nrhs; r0 += kTcNR) {
    // the tensor kernel's dependency counters (cleared per panel)
    cuda_check(cudaMemsetAsync(w.tc_counters, 0, tc_counter_bytes(tp), st), "counter clear");
    // page-locked host input: g -> panel in tree order first (rows read across the
    // host link as 16-byte runs); device input: gathered by the leaf kernel itself
    cudaEvent_t e0 = nullptr;
    if (host_io) {
      LeafArgs pa{};
      pa.perm = op->d_w_inv;
      pa.vec = g;
      pa.outp = w.tc_gt;
      pa.len_vec = op->n_in;
      pa.nrhs = int32_t(nrhs);
      pa.rhs0 = int32_t(r0);
      e0 = prof_begin(op, st);
      cuda_check(launch_permute_in(pa, st), "panel permute launch");
      prof_end(op, PK_PERMUTE, e0, st);
    }
    // (V^L)^*: panel (or g) -> yl
    LeafArgs la{};
    la.arena = op->d_arena;
    la.items = op->d_items;
    la.item_base = leaf_st.item_base;
    la.item_stride = leaf_st.n_items;
    la.off = op->d_w_off;
    la.vec = host_io ? w.tc_gt : g;
    if (rows) {   // one panel (nrhs <= kRowTab): the rows are addressed by RHS index
      la.use_rows = 1;
      la.rows = *rows;
    }
    la.gather = host_io ? 0 : 1;
    la.perm = op->d_w_perm;
    la.nat = op->d_w_nat;
    la.nat_stride = op->w_nat_stride;
    la.len_vec = op->n_in;
    la.nrhs = int32_t(nrhs);
    la.rhs0 = int32_t(r0);
    la.outs = yl;
    la.c = op->c;
    la.R = op->RV[size_t(op->L)];
    la.R8 = tp.st[0].R8_in;
    la.pts_cap = leaf_pts_cap(op->leaf_pts_w);
    e0 = prof_begin(op, st);
    cuda_check(launch_leaf(la, false, leaf_st.n_groups, st, tf32), "leaf (V^L)^* launch");
    prof_end(op, PK_LEAF_V, e0, st);
    // G / H levels on tensor cores
    TCArgs ta{};
    ta.arena = tf32 ? op->d_tc_arena_tf32 : op->d_tc_arena;
    ta.x_in = yl;
    ta.bufs = bufs;
    ta.y_out = ylast;
    ta.buf_stride = vec_bytes;
    ta.counters = w.tc_counters;
    ta.status = w.status;
    ta.nsa = op->tc_nsa;
    ta.nxb = op->tc_nxb;
    ta.nsets = op->tc_nsets;
    ta.mt_max = op->tc_mt_max;
    ta.kpad_max = op->tc_kpad_max;
    ta.plan = tp;
    e0 = prof_begin(op, st);
    cuda_check(launch_apply_tc(ta, sms, op->tc_smem, st, tf32), "tensor-core launch");
    prof_end(op, PK_TC, e0, st);
    // U^L: last main stage output -> u
    LeafArgs lu{};
    lu.arena = op->d_arena;
    lu.items = op->d_items;
    lu.item_base = last_st.item_base + 1;   // item 1 (the U^L item) of each group of the last stage
    lu.item_stride = last_st.n_items;
    lu.perm = op->d_x_perm;
    lu.off = op->d_x_off;
    lu.wl = ylast;
    lu.outp = u;
    if (rows) {
      lu.use_rows = 1;
      lu.rows = *rows;
    }
    lu.len_out = op->n_out;
    lu.nrhs = int32_t(nrhs);
    lu.rhs0 = int32_t(r0);
    lu.c = op->c;
    lu.R = op->RU[size_t(op->L)];
    lu.accumulate = accumulate ? 1 : 0;
    lu.leaf_split = op->split_x;
    e0 = prof_begin(op, st);
    cuda_check(launch_leaf(lu, true, last_st.n_groups, st), "leaf U^L launch");
    prof_end(op, PK_LEAF_U, e0, st);
  }
}

// Tensor-core adjoint g = K^* u, per panel of 64 RHS: permute the panel into X-tree
// order, the U^* leaf products (from the U^L items), the persistent tcgen05 kernel over
// the reversed levels with conjugate-transposed tiles, the V^L leaf products (from the
// (V^L)^* items) scattered to natural Omega order.
void apply_tc_adj(mbf_op_s* op, Workspace& w, const float2* u, float2* g, int64_t nrhs, cudaStream_t st, int grid,
                  bool accumulate, bool host_io) {
  if (!op->tc_unavailable.empty()) fail(MBF_ERR_INVALID, "tensor path unavailable: " + op->tc_unavailable);
  if (!op->tc_adj_unavailable.empty()) fail(MBF_ERR_INVALID, "tensor adjoint unavailable: " + op->tc_adj_unavailable);
  const TCPlan& fp = op->tcplan;
  const TCPlan& ap = op->tcplan_adj;
  const int S = ap.n_stages;
  const int64_t vec_bytes = tc_vec_bytes(op);
  ws_prepare_tc(op, w);
  if (!op->d_tc_arena_adj) {   // first adjoint apply: conjugate-transpose the tiles (kept)
    if (dev_alloc(&op->d_tc_arena_adj, size_t(op->tc_bytes)) != cudaSuccess) {
      op->d_tc_arena_adj = nullptr;
      fail(MBF_ERR_OOM, "cudaMalloc adjoint tiles");
    }
    for (int e = 0; e < fp.n_stages; ++e) {
      const TCStage& fs = fp.st[e];
      cuda_check(launch_adjoint_tiles(op->d_tc_arena + fs.base, op->d_tc_arena_adj + fs.base, fs.n_groups, fs.M_t,
                                      fs.K_t, st),
                 "adjoint tile conversion");
    }
  }
  if (op->n_w < op->n_in && !accumulate)   // Omega points outside the tree: zero
    cuda_check(cudaMemsetAsync(g, 0, size_t(nrhs) * size_t(op->n_in) * sizeof(float2), st), "cudaMemsetAsync");
  int sms = op->sms;
  if (grid > 0) sms = std::min(sms, grid);
  const Stage& leaf_st = op->plan.st[0];                        // (V^L)^* items
  const Stage& last_st = op->plan.st[op->plan.n_stages - 1];    // U^L items (item 1)
  uint8_t* yl = w.tc_bufs;
  uint8_t* bufs = yl + vec_bytes;
  float* ylast = reinterpret_cast<float*>(yl + int64_t(S) * vec_bytes);
  for (int64_t r0 = 0; r0 < nrhs; r0 += kTcNR) {
    // the tensor kernel's dependency counters (cleared per panel)
    cuda_check(cudaMemsetAsync(w.tc_counters, 0, tc_counter_bytes(ap), st), "counter clear");
    // u -> panel in X-tree order (page-locked host input), or gathered by the leaf kernel
    cudaEvent_t e0 = nullptr;
    if (host_io) {
      LeafArgs pa{};
      pa.perm = op->d_x_inv;
      pa.vec = u;
      pa.outp = w.tc_gt;
      pa.len_vec = op->n_out;
      pa.nrhs = int32_t(nrhs);
      pa.rhs0 = int32_t(r0);
      e0 = prof_begin(op, st);
      cuda_check(launch_permute_in(pa, st), "panel permute launch");
      prof_end(op, PK_PERMUTE, e0, st);
    }
    // (U^L)^*: panel (or u) -> yl (X-leaf blocks)
    LeafArgs la{};
    la.arena = op->d_arena;
    la.items = op->d_items;
    la.item_base = last_st.item_base + 1;
    la.item_stride = last_st.n_items;
    la.off = op->d_x_off;
    la.vec = host_io ? w.tc_gt : u;
    la.gather = host_io ? 0 : 1;
    la.perm = op->d_x_perm;
    la.nat = op->d_x_nat;
    la.nat_stride = op->x_nat_stride;
    la.len_vec = op->n_out;
    la.nrhs = int32_t(nrhs);
    la.rhs0 = int32_t(r0);
    la.outs = yl;
    la.c = op->c;
    la.R = op->RU[size_t(op->L)];
    la.R8 = ap.st[0].R8_in;
    la.pts_cap = leaf_pts_cap(op->leaf_pts_x);
    e0 = prof_begin(op, st);
    cuda_check(launch_leaf(la, false, last_st.n_groups, st, false, true), "leaf (U^L)^* launch");
    prof_end(op, PK_LEAF_V, e0, st);
    // (G^l)^*, l = L-1 .. h, (M^h)^*, H^l, l = h .. L-1 on tensor cores
    TCArgs ta{};
    ta.arena = op->d_tc_arena_adj;
    ta.x_in = yl;
    ta.bufs = bufs;
    ta.y_out = ylast;
    ta.buf_stride = vec_bytes;
    ta.counters = w.tc_counters;
    ta.status = w.status;
    ta.nsa = op->tca_nsa;
    ta.nxb = op->tca_nxb;
    ta.nsets = op->tca_nsets;
    ta.mt_max = op->tca_mt_max;
    ta.kpad_max = op->tca_kpad_max;
    ta.plan = ap;
    e0 = prof_begin(op, st);
    cuda_check(launch_apply_tc(ta, sms, op->tca_smem, st, false), "tensor-core launch");
    prof_end(op, PK_TC, e0, st);
    // V^L: last stage output -> g (natural Omega order)
    LeafArgs lv{};
    lv.arena = op->d_arena;
    lv.items = op->d_items;
    lv.item_base = leaf_st.item_base;
    lv.item_stride = leaf_st.n_items;
    lv.perm = op->d_w_perm;
    lv.off = op->d_w_off;
    lv.wl = ylast;
    lv.outp = g;
    lv.len_out = op->n_in;
    lv.nrhs = int32_t(nrhs);
    lv.rhs0 = int32_t(r0);
    lv.c = op->c;
    lv.R = op->RV[size_t(op->L)];
    lv.accumulate = accumulate ? 1 : 0;
    lv.leaf_split = op->split_w;
    e0 = prof_begin(op, st);
    cuda_check(launch_leaf(lv, true, leaf_st.n_groups, st, false, true), "leaf V^L launch");
    prof_end(op, PK_LEAF_U, e0, st);
  }
}

void apply_impl(mbf_op_s* op, const void* in, void* out, int64_t nrhs, int32_t precision, void* stream,
                bool adj, int grid = 0, bool accumulate = false, Workspace* ws = nullptr, bool host_io = false,
                const RowTable* rows = nullptr) {
  if (!op) fail(MBF_ERR_INVALID, "operator is NULL");
  Workspace& w = ws ? *ws : op->ws;
  if (nrhs < 0) fail(MBF_ERR_INVALID, "nrhs < 0");
  if (nrhs == 0) return;
  if (rows && (adj || host_io || nrhs > kRowTab)) fail(MBF_ERR_INVALID, "row tables: forward device applies of <= 64 RHS");
  if (!rows && (!in || !out)) fail(MBF_ERR_INVALID, "NULL vector");
  if (precision != MBF_PREC_AUTO && precision != MBF_PREC_FP32_SIMT && precision != MBF_PREC_BF16X3 &&
      precision != MBF_PREC_TF32)
    fail(MBF_ERR_INVALID, "precision not available");
  if (nrhs > (int64_t(1) << 24)) fail(MBF_ERR_INVALID, "nrhs too large");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (uses_tensor(op, nrhs, precision, adj)) {
    if (adj) {
      if (precision == MBF_PREC_TF32) fail(MBF_ERR_INVALID, "TF32 operands apply the forward operator only");
      apply_tc_adj(op, w, static_cast<const float2*>(in), static_cast<float2*>(out), nrhs, st, grid, accumulate,
                   host_io);
      return;
    }
    apply_tc(op, w, static_cast<const float2*>(in), static_cast<float2*>(out), nrhs, st, grid, accumulate, host_io,
             precision == MBF_PREC_TF32, rows);
    return;
  }
  if (!op->simt_unavailable.empty()) fail(MBF_ERR_INVALID, "FP32 SIMT path unavailable: " + op->simt_unavailable);
  const int nrb = nrhs >= 4 ? 4 : (nrhs >= 2 ? 2 : 1);
  ApplyArgs a{};
  a.arena = op->d_arena;
  a.items = op->d_items;
  a.x_perm = op->d_x_perm;
  a.x_off = op->d_x_off;
  a.w_perm = op->d_w_perm;
  a.w_off = op->d_w_off;
  a.in = static_cast<const float2*>(in);
  a.out = static_cast<float2*>(out);
  a.in_len = adj ? op->n_out : op->n_in;
  a.out_len = adj ? op->n_in : op->n_out;
  a.bufs = w.bufs;
  a.buf_stride = op->positions * nrb;
  a.barrier = w.barrier;
  a.counters = w.barrier + 64;
  a.status = w.status;
  a.nrhs = int32_t(nrhs);
  a.n_pass = int32_t((nrhs + nrb - 1) / nrb);
  a.n_slots = op->ns[nrb];
  a.plan = op->plan;
  a.accumulate = accumulate ? 1 : 0;
  a.wait_ns = op->dbg_wait_ns;
  a.stall_stage1 = op->dbg_stall_stage1;
  if (rows) {
    a.use_rows = 1;
    a.rows = *rows;
  }
  if (adj && op->n_w < op->n_in && !accumulate)
    cuda_check(cudaMemsetAsync(out, 0, size_t(nrhs) * size_t(op->n_in) * sizeof(float2), st), "cudaMemsetAsync");
  cudaEvent_t e0 = prof_begin(op, st);
  const int g = grid > 0 ? std::min(grid, op->grid) : op->grid;
  cuda_check(launch_apply_simt(a, nrb, adj, g, op->smem[nrb], st), "apply launch");
  prof_end(op, PK_SIMT, e0, st);
}

}  // namespace

void validate(const mbf_factors_t& f) { validate_factors(f); }

void set_last_error(const std::string& m) { g_last_error = m; }

// Which path an apply takes: split-BF16x3 or TF32 on request; AUTO uses the split-BF16x3
// tensor cores from tc_min_rhs right-hand sides (8, or what the tuner measured), for the
// adjoint too where its conjugate-transposed tiles fit.
bool uses_tensor(const mbf_op_s* op, int64_t nrhs, int32_t precision, bool adj) {
  if (precision == MBF_PREC_AUTO && !op->simt_unavailable.empty() && op->tc_unavailable.empty() &&
      (!adj || op->tc_adj_unavailable.empty()))
    return true;   // an operator the SIMT kernel cannot take: tensor cores for any RHS count
  return precision == MBF_PREC_BF16X3 || precision == MBF_PREC_TF32 ||
         (precision == MBF_PREC_AUTO && nrhs >= op->tc_min_rhs && op->tc_unavailable.empty() &&
          (!adj || op->tc_adj_unavailable.empty()));
}

// Bytes of one tensor-path vector: every block of a level at the largest R8, split or
// complex64 (8 bytes an entry, 64 RHS).
int64_t tc_vec_bytes(const mbf_op_s* op) {
  int r8max = 8;
  for (int e = 0; e < op->tcplan.n_stages; ++e)
    r8max = std::max({r8max, op->tcplan.st[e].R8_in, op->tcplan.st[e].R8_out});
  return Tree::ipow(op->c, op->L) * split_block_bytes(r8max);
}

// Workspaces.  The SIMT parts at operator creation; the tensor path's on its first use
// (or through tc_prepare / the server before a capture), so later applies allocate
// nothing.
void ws_init(const mbf_op_s* op, Workspace& w) {
  const size_t vbytes = size_t(op->plan.n_stages) * size_t(op->positions) * 4 * sizeof(float2);
  if (dev_alloc(&w.bufs, vbytes) != cudaSuccess) fail(MBF_ERR_OOM, "cudaMalloc workspace");
  if (dev_alloc(&w.barrier, 256 + counter_bytes(op->plan)) != cudaSuccess || dev_alloc(&w.status, 256) != cudaSuccess)
    fail(MBF_ERR_OOM, "cudaMalloc barrier");
  cuda_check(cudaMemset(w.status, 0, 256), "cudaMemset status");
}

void ws_prepare_tc(const mbf_op_s* op, Workspace& w) {
  if (w.tc_bufs || !op->tc_unavailable.empty()) return;
  const int S = op->tcplan.n_stages;
  const int64_t vec_bytes = tc_vec_bytes(op);
  if (dev_alloc(&w.tc_bufs, size_t(S + 1) * size_t(vec_bytes)) != cudaSuccess)
    fail(MBF_ERR_OOM, "cudaMalloc tensor-path workspace");
  if (dev_alloc(&w.tc_counters, tc_counter_bytes(op->tcplan)) != cudaSuccess)
    fail(MBF_ERR_OOM, "cudaMalloc tensor-path counters");
  if (dev_alloc(&w.tc_gt, size_t(std::max<int64_t>({op->n_w, op->n_out, 1})) * kTcNR * sizeof(float2)) != cudaSuccess)
    fail(MBF_ERR_OOM, "cudaMalloc tensor-path input panel");
}

void ws_free(Workspace& w) {
  cudaFree(w.bufs);
  cudaFree(w.barrier);
  cudaFree(w.status);
  cudaFree(w.tc_bufs);
  cudaFree(w.tc_counters);
  cudaFree(w.tc_gt);
  w = Workspace{};
}

void tc_prepare(mbf_op_s* op) { ws_prepare_tc(op, op->ws); }

void pack_host(const mbf_factors_t& f, PackedHost& out) {
  validate_factors(f);
  mbf_op_s tmp;   // receives the plan and the per-stage counts; no device state
  Packer pk(f);
  pk.run(tmp);
  int64_t rmax = 1;
  for (int l = f.L / 2; l <= f.L; ++l) rmax = std::max<int64_t>({rmax, f.RU[l], f.RV[l]});
  const int64_t positions = Tree::ipow(int64_t(1) << f.dim, f.L) * rmax;
  out = PackedHost{};
  check_plan(tmp.plan, pk.items, pk.arena.size(), positions, f, &out.simt_unavailable);
  out.plan = tmp.plan;
  out.items = std::move(pk.items);
  out.arena = std::move(pk.arena);
  try {
    int mt = 0, kp = 0;
    pack_tc(f, out.plan, out.tcplan, out.tc_arena, mt, kp);
    const Stage& first = out.plan.st[0];
    const Stage& last = out.plan.st[out.plan.n_stages - 1];
    if (out.plan.n_stages < 2 || first.n_items != 1 || last.n_items != 2 || last.B != 1 ||
        out.tcplan.st[0].in_pat != PAT_SPLIT || out.tcplan.st[0].B != 1)
      fail(MBF_ERR_INVALID, "plan shape not supported by the tensor path");
  } catch (const Error& err) {
    out.tc_unavailable = err.what();
    out.tc_arena.clear();
    return;
  }
  try {
    adjoint_tile_plan(out.tcplan, out.tcplan_adj);
  } catch (const Error& err) {
    out.tc_adj_unavailable = err.what();
  }
}

Workspace* ws_acquire(mbf_op_s* op, bool tensor) {
  std::lock_guard<std::mutex> lk(op->ws_mu);
  Workspace* w = nullptr;
  if (!op->ws_own_lent) {
    op->ws_own_lent = true;
    w = &op->ws;
  } else {
    for (size_t k = 0; k < op->ws_pool.size() && !w; ++k)
      if (!op->ws_pool_lent[k]) {
        op->ws_pool_lent[k] = true;
        w = op->ws_pool[k];
      }
    if (!w) {
      auto* nw = new Workspace();
      try {
        ws_init(op, *nw);
      } catch (...) {
        ws_free(*nw);
        delete nw;
        throw;
      }
      op->ws_pool.push_back(nw);
      op->ws_pool_lent.push_back(true);
      w = nw;
    }
  }
  try {
    if (tensor) ws_prepare_tc(op, *w);
  } catch (...) {
    if (w == &op->ws) op->ws_own_lent = false;
    for (size_t k = 0; k < op->ws_pool.size(); ++k)
      if (op->ws_pool[k] == w) op->ws_pool_lent[k] = false;
    throw;
  }
  return w;
}

void ws_release(mbf_op_s* op, Workspace* w) {
  std::lock_guard<std::mutex> lk(op->ws_mu);
  if (w == &op->ws) {
    op->ws_own_lent = false;
    return;
  }
  for (size_t k = 0; k < op->ws_pool.size(); ++k)
    if (op->ws_pool[k] == w) op->ws_pool_lent[k] = false;
}

void apply_dev(mbf_op_s* op, const void* in, void* out, int64_t nrhs, int32_t precision, cudaStream_t st,
               bool adj, int grid, bool accumulate, Workspace* ws, const RowTable* rows) {
  apply_impl(op, in, out, nrhs, precision, st, adj, grid, accumulate, ws, false, rows);
}

}  // namespace mbf

using namespace mbf;

extern "C" {

const char* mbf_last_error(void) { return g_last_error.c_str(); }
const char* mbf_version(void) { return "mbf-gb300 0.1 (sm_103a)"; }

mbf_status mbf_build_factors(const mbf_problem_t* prob, mbf_entry_fn fn, void* ctx,
                             const mbf_build_opts_t* opts, mbf_factors_h* out) {
  return abi_guard([&] {
    if (!prob || !out) fail(MBF_ERR_INVALID, "NULL argument");
    mbf_build_opts_t o{};
    if (opts) o = *opts;
    auto* h = new mbf_factors_s();
    try {
      h->fs = build_or_load(*prob, fn, ctx, o);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

mbf_status mbf_build_from_applies(const mbf_problem_t* prob, mbf_apply_fn fn, void* ctx,
                                  const mbf_build_opts_t* opts, mbf_factors_h* out) {
  return abi_guard([&] {
    if (!prob || !out) fail(MBF_ERR_INVALID, "NULL argument");
    mbf_build_opts_t o{};
    if (opts) o = *opts;
    auto* h = new mbf_factors_s();
    try {
      h->fs = build_factors_from_applies(*prob, fn, ctx, o);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

mbf_status mbf_factors_view(mbf_factors_h f, mbf_factors_t* view) {
  return abi_guard([&] {
    if (!f || !view) fail(MBF_ERR_INVALID, "NULL argument");
    *view = f->fs.view();
  });
}

mbf_status mbf_factors_destroy(mbf_factors_h f) {
  return abi_guard([&] { delete f; });
}

mbf_status mbf_factors_save(const mbf_factors_t* f, const char* path) {
  return abi_guard([&] {
    if (!f || !path) fail(MBF_ERR_INVALID, "NULL argument");
    save_factors(*f, path);
  });
}

mbf_status mbf_factors_load(const char* path, mbf_factors_h* out) {
  return abi_guard([&] {
    if (!path || !out) fail(MBF_ERR_INVALID, "NULL argument");
    auto* h = new mbf_factors_s();
    try {
      h->fs = load_factors(path);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

mbf_status mbf_op_create(const mbf_factors_t* f, mbf_op_t* out) {
  return abi_guard([&] {
    if (!f || !out) fail(MBF_ERR_INVALID, "NULL argument");
    *out = op_create(*f);
  });
}

mbf_status mbf_build_from_entries(const mbf_problem_t* prob, mbf_entry_fn fn, void* ctx,
                                  const mbf_build_opts_t* opts, mbf_op_t* out) {
  return abi_guard([&] {
    if (!prob || !out) fail(MBF_ERR_INVALID, "NULL argument");
    mbf_build_opts_t o{};
    if (opts) o = *opts;
    FactorSet fs = build_or_load(*prob, fn, ctx, o);
    mbf_factors_t v = fs.view();
    mbf_op_s* op = op_create(v);
    fs = FactorSet{};
    try {
      // the §3.3 estimator on 256 sampled outputs, kept for mbf_op_info (grid problems)
      if (prob->tree != MBF_TREE_POINTS) estimate_error(op, fn, ctx, 256, o.seed ^ 0x6570735f65737469ull, nullptr);
    } catch (...) {
      op_free(op);
      throw;
    }
    *out = op;
  });
}

mbf_status mbf_op_estimate_error(mbf_op_t op, mbf_entry_fn fn, void* ctx, int32_t n_samples, uint64_t seed,
                                 void* stream, double* eps) {
  return abi_guard([&] {
    if (!op) fail(MBF_ERR_INVALID, "NULL operator");
    const double e = estimate_error(op, fn, ctx, n_samples, seed, static_cast<cudaStream_t>(stream));
    if (eps) *eps = e;
  });
}

mbf_status mbf_op_destroy(mbf_op_t op) {
  return abi_guard([&] { op_free(op); });
}

mbf_status mbf_op_info(mbf_op_t op, mbf_op_info_t* info) {
  return abi_guard([&] {
    if (!op || !info) fail(MBF_ERR_INVALID, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->dim = op->d;
    info->L = op->L;
    info->c = op->c;
    info->n_stages = op->plan.n_stages;
    info->n_out = op->n_out;
    info->n_in = op->n_in;
    for (int l = 0; l <= op->L && l < 32; ++l) {
      info->RU[l] = op->RU[size_t(l)];
      info->RV[l] = op->RV[size_t(l)];
    }
    info->nnz_algorithmic = op->nnz;
    info->bytes_algorithmic = 8 * op->nnz;
    info->bytes_packed = op->bytes_packed;
    for (int s = 0; s < op->plan.n_stages && s < 32; ++s) info->bytes_stage[s] = op->plan.st[s].bytes;
    info->grid = op->grid;
    info->threads = simt_threads(1);
    info->smem = int(op->smem[1]);
    for (size_t e = 0; e < op->nnz_stage.size() && e < 32; ++e) info->nnz_stage[e] = op->nnz_stage[e];
    info->nnz_leaf_u = op->nnz_leaf_x;
    info->tensor_ok = op->tc_unavailable.empty() ? 1 : 0;
    info->tensor_stages = op->tcplan.n_stages;
    info->bytes_tensor = op->tc_bytes;
    info->tensor_smem = int(op->tc_smem);
    info->tensor_slots = op->tc_nsa;
    std::snprintf(info->tensor_unavailable, sizeof(info->tensor_unavailable), "%s", op->tc_unavailable.c_str());
    info->eps = op->eps;
    info->eps_samples = op->eps_samples;
  });
}

mbf_status mbf_op_set_profiling(mbf_op_t op, int32_t enable) {
  return abi_guard([&] {
    if (!op) fail(MBF_ERR_INVALID, "NULL operator");
    prof_collect(op);
    op->prof_on = enable != 0;
    for (int k = 0; k < 8; ++k) {
      op->prof_launches[k] = 0;
      op->prof_ms[k] = 0.0;
    }
  });
}

mbf_status mbf_op_profile(mbf_op_t op, mbf_profile_t* out) {
  return abi_guard([&] {
    if (!op || !out) fail(MBF_ERR_INVALID, "NULL argument");
    prof_collect(op);
    std::memset(out, 0, sizeof(*out));
    out->n_kinds = PK_COUNT;
    for (int k = 0; k < PK_COUNT; ++k) {
      std::snprintf(out->name[k], sizeof(out->name[k]), "%s", kProfNames[k]);
      out->launches[k] = op->prof_launches[k];
      out->ms[k] = op->prof_ms[k];
      op->prof_launches[k] = 0;
      op->prof_ms[k] = 0.0;
    }
  });
}

mbf_status mbf_apply(mbf_op_t op, const void* g, void* u, int64_t nrhs, int32_t precision, void* stream) {
  return abi_guard([&] { apply_impl(op, g, u, nrhs, precision, stream, false); });
}

mbf_status mbf_apply_adjoint(mbf_op_t op, const void* u, void* g, int64_t nrhs, int32_t precision,
                             void* stream) {
  return abi_guard([&] { apply_impl(op, u, g, nrhs, precision, stream, true); });
}

mbf_status mbf_apply_host(mbf_op_t op, const void* g_host, void* u_host, int64_t nrhs, int32_t precision,
                          void* stream) {
  return abi_guard([&] {
    if (!op || !g_host || !u_host) fail(MBF_ERR_INVALID, "NULL argument");
    if (nrhs <= 0) return;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t in_b = size_t(nrhs) * size_t(op->n_in) * sizeof(float2);
    const size_t out_b = size_t(nrhs) * size_t(op->n_out) * sizeof(float2);
    // Page-locked host buffers that the device can address (the usual case for
    // cudaHostAlloc / cudaHostRegister memory): the tensor path's permute kernel reads g
    // and its U^L kernel writes u across the host link directly, each element once, so
    // the transfers overlap the apply instead of preceding and following it.
    if (uses_tensor(op, nrhs, precision, false)) {
      cudaPointerAttributes ag{}, au{};
      if (cudaPointerGetAttributes(&ag, g_host) == cudaSuccess && cudaPointerGetAttributes(&au, u_host) == cudaSuccess &&
          ag.type == cudaMemoryTypeHost && au.type == cudaMemoryTypeHost && ag.devicePointer && au.devicePointer) {
        apply_impl(op, ag.devicePointer, au.devicePointer, nrhs, precision, stream, false, 0, false, nullptr, true);
        cuda_check(cudaStreamSynchronize(st), "sync");
        return;
      }
      cudaGetLastError();   // clear a failed query (not page-locked): copy below
    }
    if (in_b > op->stage_in_bytes) {
      cuda_check(cudaStreamSynchronize(st), "sync");
      cudaFree(op->d_stage_in);
      op->d_stage_in = nullptr;
      if (dev_alloc(&op->d_stage_in, in_b) != cudaSuccess) fail(MBF_ERR_OOM, "cudaMalloc staging");
      op->stage_in_bytes = in_b;
    }
    if (out_b > op->stage_out_bytes) {
      cuda_check(cudaStreamSynchronize(st), "sync");
      cudaFree(op->d_stage_out);
      op->d_stage_out = nullptr;
      if (dev_alloc(&op->d_stage_out, out_b) != cudaSuccess) fail(MBF_ERR_OOM, "cudaMalloc staging");
      op->stage_out_bytes = out_b;
    }
    cuda_check(cudaMemcpyAsync(op->d_stage_in, g_host, in_b, cudaMemcpyHostToDevice, st), "H2D");
    apply_impl(op, op->d_stage_in, op->d_stage_out, nrhs, precision, stream, false);
    cuda_check(cudaMemcpyAsync(u_host, op->d_stage_out, out_b, cudaMemcpyDeviceToHost, st), "D2H");
    cuda_check(cudaStreamSynchronize(st), "sync");
  });
}

mbf_status mbf_apply_host_batch(mbf_op_t op, const void* g_host, void* u_host, int64_t nbatch, int64_t nrhs,
                                int32_t precision, void* stream) {
  return abi_guard([&] {
    if (!op) fail(MBF_ERR_INVALID, "operator is NULL");
    if (nbatch < 0 || nrhs < 0) fail(MBF_ERR_INVALID, "negative count");
    if (nbatch == 0 || nrhs == 0) return;
    if (!g_host || !u_host) fail(MBF_ERR_INVALID, "NULL argument");
    if (nrhs > (int64_t(1) << 24)) fail(MBF_ERR_INVALID, "nrhs too large");
    const size_t in_b = size_t(nrhs) * size_t(op->n_in) * sizeof(float2);
    const size_t out_b = size_t(nrhs) * size_t(op->n_out) * sizeof(float2);
    if (size_t(nbatch) > SIZE_MAX / std::max<size_t>(std::max(in_b, out_b), 1))
      fail(MBF_ERR_INVALID, "nbatch x panel bytes overflows");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // staging pairs (re)allocated when a larger panel comes; the previous call has
    // synchronized, so none is in use
    if (in_b > op->pipe_in_bytes || out_b > op->pipe_out_bytes) {
      op->pipe_in_bytes = op->pipe_out_bytes = 0;
      for (int b = 0; b < 2; ++b) {
        cudaFree(op->d_pipe_in[b]);
        cudaFree(op->d_pipe_out[b]);
        op->d_pipe_in[b] = op->d_pipe_out[b] = nullptr;
      }
      for (int b = 0; b < 2; ++b)
        if (dev_alloc(&op->d_pipe_in[b], in_b) != cudaSuccess || dev_alloc(&op->d_pipe_out[b], out_b) != cudaSuccess)
          fail(MBF_ERR_OOM, "cudaMalloc pipeline staging");
      op->pipe_in_bytes = in_b;
      op->pipe_out_bytes = out_b;
    }
    for (int b = 0; b < 2; ++b) {
      if (!op->pipe_st[b]) cuda_check(cudaStreamCreateWithFlags(&op->pipe_st[b], cudaStreamNonBlocking), "stream");
      for (auto& ev : op->pipe_ev)
        if (!ev[b]) cuda_check(cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming), "event");
    }
    cudaStream_t c_in = op->pipe_st[0], c_out = op->pipe_st[1];
    cudaEvent_t* copied_in = op->pipe_ev[0];
    cudaEvent_t* applied = op->pipe_ev[1];
    cudaEvent_t* copied_out = op->pipe_ev[2];
    const char* gi = static_cast<const char*>(g_host);
    char* uo = static_cast<char*>(u_host);
    try {
      // panel i uses pair b = i mod 2: its input copy waits until apply i-2 has read the
      // pair's input, its apply until the output of panel i-2 has left the pair
      for (int64_t i = 0; i < nbatch; ++i) {
        const int b = int(i & 1);
        if (i >= 2) cuda_check(cudaStreamWaitEvent(c_in, applied[b], 0), "wait");
        cuda_check(cudaMemcpyAsync(op->d_pipe_in[b], gi + size_t(i) * in_b, in_b, cudaMemcpyHostToDevice, c_in),
                   "H2D");
        cuda_check(cudaEventRecord(copied_in[b], c_in), "record");
        cuda_check(cudaStreamWaitEvent(st, copied_in[b], 0), "wait");
        if (i >= 2) cuda_check(cudaStreamWaitEvent(st, copied_out[b], 0), "wait");
        apply_impl(op, op->d_pipe_in[b], op->d_pipe_out[b], nrhs, precision, stream, false);
        cuda_check(cudaEventRecord(applied[b], st), "record");
        cuda_check(cudaStreamWaitEvent(c_out, applied[b], 0), "wait");
        cuda_check(cudaMemcpyAsync(uo + size_t(i) * out_b, op->d_pipe_out[b], out_b, cudaMemcpyDeviceToHost, c_out),
                   "D2H");
        cuda_check(cudaEventRecord(copied_out[b], c_out), "record");
      }
    } catch (...) {
      // nothing of this call may still be in flight when it returns
      cudaStreamSynchronize(c_in);
      cudaStreamSynchronize(st);
      cudaStreamSynchronize(c_out);
      throw;
    }
    cuda_check(cudaStreamSynchronize(c_out), "sync");
    cuda_check(cudaStreamSynchronize(st), "sync");
  });
}

mbf_status mbf_debug_fail_alloc(int64_t after) {
  return abi_guard([&] { g_alloc_budget.store(after < 0 ? -1 : after); });
}

mbf_status mbf_op_debug_stall(mbf_op_t op, int32_t stage, int64_t wait_ns) {
  return abi_guard([&] {
    if (!op) fail(MBF_ERR_INVALID, "NULL operator");
    if (stage >= op->plan.n_stages) fail(MBF_ERR_INVALID, "stall stage beyond the plan");
    if (wait_ns < 0) fail(MBF_ERR_INVALID, "negative wait limit");
    op->dbg_stall_stage1 = stage >= 0 ? stage + 1 : 0;
    op->dbg_wait_ns = uint64_t(wait_ns);
  });
}

mbf_status mbf_op_check(mbf_op_t op, void* stream) {
  return abi_guard([&] {
    if (!op) fail(MBF_ERR_INVALID, "NULL operator");
    cuda_check(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "cudaStreamSynchronize");
    int st = 0;
    cuda_check(cudaMemcpy(&st, op->ws.status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    if (st != ST_OK) {
      cuda_check(cudaMemset(op->ws.status, 0, sizeof(int)), "clear status");
      static const char* names[] = {"ok", "grid barrier", "full mbarrier", "empty mbarrier", "bad item",
                                    "dependency counter"};
      fail(MBF_ERR_TIMEOUT, std::string("device wait gave up: ") + (st >= 0 && st <= 5 ? names[st] : "unknown"));
    }
  });
}

}  // extern "C"
