// Host interpreter of the packed device layouts (mbf_debug_layout_apply): the factor
// set is packed on the host by the packers mbf_op_create uses (pack_host), and the
// packed arena is then applied in FP64 by reading it the way the layout's definitions
// in layout.hpp and the tile packer state it.  A test facility: it lets the packers,
// the stage plan and the tile contents be checked against the oracle without a device.
//
// The apply is the product of eq. (gbf), §2.3: (V^L)^* leaf products, the (H^l)^* and
// G^l group products of the stages, M^h folded into the G^h gather and tiles, and the
// U^L leaf products scattered to the natural X order.
#include <algorithm>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "layout.hpp"
#include "mbf_internal.hpp"
#include "op_internal.hpp"

namespace {

using mbf::cd;
using mbf::Error;
using mbf::fail;
using mbf::Item;
using mbf::Stage;
using mbf::TCStage;

// Entry e of line `line` of an item: chunks of lpc lines, each a real plane then an
// imaginary plane of nl * len floats (the plane padded to a multiple of 4 floats).
cd item_at(const std::vector<uint8_t>& arena, const Item& it, int line, int e) {
  const int lpc = it.lpc, ci = line / lpc, li = line - ci * lpc;
  const int nl = std::min(lpc, int(it.nlines) - ci * lpc);
  const size_t chunk = size_t(it.off128) * 128 + size_t(ci) * size_t(mbf::chunk_bytes(lpc, it.len));
  const size_t q = size_t(li) * it.len + size_t(e);
  const size_t im = size_t(mbf::pad4(int64_t(nl) * it.len));
  if (chunk + 4 * (im + q) + 4 > arena.size()) fail(MBF_ERR_INVALID, "layout: item entry beyond the arena");
  float re_v, im_v;
  std::memcpy(&re_v, arena.data() + chunk + 4 * q, 4);
  std::memcpy(&im_v, arena.data() + chunk + 4 * (im + q), 4);
  return cd(re_v, im_v);
}

// Offset of segment t of group g in a coefficient vector of segments of R entries:
// PAT_SPLIT ((c a + t) B + b) R, PAT_CONTIG (c g + t) R, PAT_CORNER ((c b + t) c^h + a) R,
// with a = g / B, b = g mod B.
int64_t seg(int pat, int64_t g, int t, int64_t B, int64_t ch, int64_t R, int c) {
  const int64_t a = g / B, b = g % B;
  if (pat == mbf::PAT_SPLIT) return ((c * a + t) * B + b) * R;
  if (pat == mbf::PAT_CONTIG) return (c * g + t) * R;
  if (pat == mbf::PAT_CORNER) return ((c * b + t) * ch + a) * R;
  fail(MBF_ERR_INVALID, "layout: leaf pattern between stages");
}

// Child t (0..c-1) of group g whose leaf holds tree-order point p.
int leaf_child(const int64_t* off, int64_t g, int c, int64_t p) {
  for (int t = 0; t < c; ++t)
    if (off[c * g + t] <= p && p < off[c * g + t + 1]) return t;
  fail(MBF_ERR_INVALID, "layout: a leaf item's point lies outside its group");
}

float bf16_value(const uint8_t* p) {
  uint16_t h;
  std::memcpy(&h, p, 2);
  const uint32_t u = uint32_t(h) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Tile element (m, k) of one group: chunk k / 16 holds planes Re hi, Im hi, Re lo, Im lo
// of plane_bytes each; inside a plane, 8 x 8 core matrices of 128 bytes, the two of a
// row group adjacent: byte ((m / 8) 2 + kc / 8) 128 + (m mod 8) 16 + (kc mod 8) 2.
cd tile_at(const uint8_t* tile, const TCStage& ts, int m, int k) {
  const int kc = k % 16;
  const size_t in_plane = size_t(((m / 8) * 2 + kc / 8) * 128 + (m % 8) * 16 + (kc % 8) * 2);
  const uint8_t* chunk = tile + size_t(k / 16) * 4 * size_t(ts.plane_bytes) + in_plane;
  const double re = double(bf16_value(chunk)) + double(bf16_value(chunk + 2 * size_t(ts.plane_bytes)));
  const double im = double(bf16_value(chunk + ts.plane_bytes)) + double(bf16_value(chunk + 3 * size_t(ts.plane_bytes)));
  return cd(re, im);
}

struct Interp {
  const mbf_factors_t& f;
  const mbf::PackedHost& ph;
  int c = 4;
  int64_t nL = 0, rmax = 1;

  Interp(const mbf_factors_t& fa, const mbf::PackedHost& p) : f(fa), ph(p) {
    c = ph.plan.c;
    nL = mbf::Tree::ipow(c, f.L);
    for (int l = f.L / 2; l <= f.L; ++l) rmax = std::max<int64_t>({rmax, f.RU[l], f.RV[l]});
  }
  const Item& item(const Stage& st, int64_t g, int k) const {
    const int64_t i = st.item_base + g * st.n_items + k;
    if (i < 0 || i >= int64_t(ph.items.size())) fail(MBF_ERR_INVALID, "layout: item index out of range");
    return ph.items[size_t(i)];
  }

  // Input entry (t, k), as line t Rin + k of the full block, of each stored line of a
  // main item: all c Rin lines, or in a compact stage the first r_t of each segment t
  // (r_t from byte t of the item's base).
  std::vector<int> main_lines(const Stage& st, const Item& m) const {
    std::vector<int> lines;
    for (int t = 0; t < c; ++t) {
      const int r = st.compact ? mbf::seg_lines(m.base, t) : st.R_in;
      if (r > st.R_in) fail(MBF_ERR_INVALID, "layout: segment line count above the rank");
      for (int k = 0; k < r; ++k) lines.push_back(t * st.R_in + k);
    }
    if (int(lines.size()) != m.nlines || m.len != c * st.R_out) fail(MBF_ERR_INVALID, "layout: main item shape");
    return lines;
  }

  // (V^L)^*: the level-L coefficient vector from g (natural Omega order)
  void leaf_forward(const cd* g, std::vector<cd>& out) const {
    const Stage& s0 = ph.plan.st[0];
    for (int64_t grp = 0; grp < s0.n_groups; ++grp) {
      const Item& it = item(s0, grp, 0);
      for (int b = 0; b < it.nlines; ++b) {
        const int64_t p = it.base + b;
        const int t = leaf_child(f.w_off, grp, c, p);
        const cd x = g[f.w_perm[p]];
        const int64_t o = seg(s0.out_pat, grp, t, s0.B, s0.ch, s0.R_out, c);
        for (int k = 0; k < it.len; ++k) out[size_t(o + k)] += item_at(ph.arena, it, b, k) * x;
      }
    }
  }
  // U^L of group grp: u[x_perm(p)] += sum_k U^L[p][k] y[t(p) Rs + k] for its points p
  void leaf_u_forward(const Stage& st, int64_t grp, const std::vector<cd>& y, int Rs, cd* u) const {
    const Item& lx = item(st, grp, 1);
    if (lx.nlines == 0) return;
    for (int a = 0; a < lx.len; ++a) {
      const int64_t p = lx.base + a;
      const int t = leaf_child(f.x_off, grp, c, p);
      cd s = 0;
      for (int k = 0; k < lx.nlines; ++k) s += item_at(ph.arena, lx, k, a) * y[size_t(t * Rs + k)];
      u[f.x_perm[p]] += s;
    }
  }

  void simt_forward(const cd* g, cd* u) const {
    std::vector<cd> cur(size_t(nL * rmax), 0.0), nxt(cur.size());
    leaf_forward(g, cur);
    for (int e = 1; e < ph.plan.n_stages; ++e) {
      const Stage& st = ph.plan.st[e];
      std::fill(nxt.begin(), nxt.end(), cd(0.0));
      std::vector<cd> y(size_t(c * st.R_out));
      for (int64_t grp = 0; grp < st.n_groups; ++grp) {
        const Item& m = item(st, grp, st.main_idx);
        const std::vector<int> full = main_lines(st, m);
        std::fill(y.begin(), y.end(), cd(0.0));
        for (int line = 0; line < m.nlines; ++line) {
          const int tp = full[size_t(line)] / st.R_in, k = full[size_t(line)] % st.R_in;
          const cd x = cur[size_t(seg(st.in_pat, grp, tp, st.B, st.ch, st.R_in, c) + k)];
          for (int q = 0; q < m.len; ++q) y[size_t(q)] += item_at(ph.arena, m, line, q) * x;
        }
        if (st.out_pat == mbf::PAT_LEAF) {
          leaf_u_forward(st, grp, y, st.R_out, u);
        } else {
          for (int t = 0; t < c; ++t)
            for (int k2 = 0; k2 < st.R_out; ++k2)
              nxt[size_t(seg(st.out_pat, grp, t, st.B, st.ch, st.R_out, c) + k2)] += y[size_t(t * st.R_out + k2)];
        }
      }
      std::swap(cur, nxt);
    }
  }

  // K^*: the stages in reverse order, every item conjugate-transposed
  void simt_adjoint(const cd* u, cd* g) const {
    const int S = ph.plan.n_stages;
    std::vector<cd> cur(size_t(nL * rmax), 0.0), nxt(cur.size());
    for (int e = S - 1; e >= 1; --e) {
      const Stage& st = ph.plan.st[e];
      std::fill(nxt.begin(), nxt.end(), cd(0.0));
      std::vector<cd> y(size_t(c * st.R_out));
      for (int64_t grp = 0; grp < st.n_groups; ++grp) {
        std::fill(y.begin(), y.end(), cd(0.0));
        if (st.out_pat == mbf::PAT_LEAF) {   // (U^L)^* from u (natural X order)
          const Item& lx = item(st, grp, 1);
          for (int a = 0; a < (lx.nlines ? lx.len : 0); ++a) {
            const int64_t p = lx.base + a;
            const int t = leaf_child(f.x_off, grp, c, p);
            for (int k = 0; k < lx.nlines; ++k)
              y[size_t(t * st.R_out + k)] += std::conj(item_at(ph.arena, lx, k, a)) * u[f.x_perm[p]];
          }
        } else {
          for (int t = 0; t < c; ++t)
            for (int k2 = 0; k2 < st.R_out; ++k2)
              y[size_t(t * st.R_out + k2)] = cur[size_t(seg(st.out_pat, grp, t, st.B, st.ch, st.R_out, c) + k2)];
        }
        const Item& m = item(st, grp, st.main_idx);
        const std::vector<int> full = main_lines(st, m);
        for (int line = 0; line < m.nlines; ++line) {
          const int tp = full[size_t(line)] / st.R_in, k = full[size_t(line)] % st.R_in;
          cd s = 0;
          for (int q = 0; q < m.len; ++q) s += std::conj(item_at(ph.arena, m, line, q)) * y[size_t(q)];
          nxt[size_t(seg(st.in_pat, grp, tp, st.B, st.ch, st.R_in, c) + k)] += s;
        }
      }
      std::swap(cur, nxt);
    }
    const Stage& s0 = ph.plan.st[0];   // V^L to natural Omega order
    for (int64_t grp = 0; grp < s0.n_groups; ++grp) {
      const Item& it = item(s0, grp, 0);
      for (int b = 0; b < it.nlines; ++b) {
        const int64_t p = it.base + b;
        const int t = leaf_child(f.w_off, grp, c, p);
        const int64_t o = seg(s0.out_pat, grp, t, s0.B, s0.ch, s0.R_out, c);
        cd s = 0;
        for (int k = 0; k < it.len; ++k) s += std::conj(item_at(ph.arena, it, b, k)) * cur[size_t(o + k)];
        g[f.w_perm[p]] += s;
      }
    }
  }

  // Tensor path: the leaf items of the SIMT arena, the G/H levels from the split tiles.
  // Rows and columns of the rank padding must hold zeros.
  void tc_forward(const cd* g, cd* u) const {
    std::vector<cd> cur(size_t(nL * rmax), 0.0), nxt(cur.size());
    leaf_forward(g, cur);
    const int S = ph.plan.n_stages;
    if (ph.tcplan.n_stages != S - 1) fail(MBF_ERR_INVALID, "layout: tile plan does not match the stage plan");
    for (int e = 1; e < S; ++e) {
      const Stage& st = ph.plan.st[e];
      const TCStage& ts = ph.tcplan.st[e - 1];
      if (ts.R_in != st.R_in || ts.R_out != st.R_out || ts.n_groups != st.n_groups)
        fail(MBF_ERR_INVALID, "layout: tile stage differs from its stage");
      if (ts.base + int64_t(ts.n_groups) * ts.tile_bytes > int64_t(ph.tc_arena.size()))
        fail(MBF_ERR_INVALID, "layout: tiles beyond the arena");
      std::fill(nxt.begin(), nxt.end(), cd(0.0));
      std::vector<cd> y(size_t(ts.M_t));
      for (int64_t grp = 0; grp < ts.n_groups; ++grp) {
        const uint8_t* tile = ph.tc_arena.data() + size_t(ts.base) + size_t(grp) * size_t(ts.tile_bytes);
        std::fill(y.begin(), y.end(), cd(0.0));
        for (int k = 0; k < ts.K_pad; ++k) {
          const int tp = k / ts.R8_in, kk = k % ts.R8_in;
          const bool pad_col = k >= ts.K_t || kk >= ts.R_in;
          const cd x = pad_col ? cd(0.0) : cur[size_t(seg(ts.in_pat, grp, tp, ts.B, ts.ch, ts.R_in, c) + kk)];
          for (int m = 0; m < ts.M_t; ++m) {
            const cd v = tile_at(tile, ts, m, k);
            if ((pad_col || m % ts.R8_out >= ts.R_out) && v != cd(0.0))
              fail(MBF_ERR_INVALID, "layout: nonzero tile entry in the rank padding");
            y[size_t(m)] += v * x;
          }
        }
        if (ts.last) {
          leaf_u_forward(st, grp, y, ts.R8_out, u);
        } else {
          for (int t = 0; t < c; ++t)
            for (int k2 = 0; k2 < ts.R_out; ++k2)
              nxt[size_t(seg(ts.out_pat, grp, t, ts.B, ts.ch, ts.R_out, c) + k2)] += y[size_t(t * ts.R8_out + k2)];
        }
      }
      std::swap(cur, nxt);
    }
  }

  // Tensor adjoint: (U^L)^* from the leaf items of the last stage, then the stages of the
  // adjoint plan, stage e reading forward stage S - 1 - e's tile of the same group
  // conjugate-transposed (the device converts the tiles once; here they are read in
  // place), then V^L to natural Omega order.
  void tc_adjoint(const cd* u, cd* g) const {
    const mbf::TCPlan& fp = ph.tcplan;
    const mbf::TCPlan& ap = ph.tcplan_adj;
    const int S = ph.plan.n_stages;
    if (ap.n_stages != fp.n_stages || ap.n_stages != S - 1) fail(MBF_ERR_INVALID, "layout: adjoint plan size");
    std::vector<cd> cur(size_t(nL * rmax), 0.0), nxt(cur.size());
    const Stage& sl = ph.plan.st[S - 1];
    const TCStage& a0 = ap.st[0];
    for (int64_t grp = 0; grp < sl.n_groups; ++grp) {
      const Item& lx = item(sl, grp, 1);
      for (int a = 0; a < (lx.nlines ? lx.len : 0); ++a) {
        const int64_t p = lx.base + a;
        const int t = leaf_child(f.x_off, grp, c, p);
        const int64_t o = seg(a0.in_pat, grp, t, a0.B, a0.ch, a0.R_in, c);
        for (int k = 0; k < lx.nlines; ++k) cur[size_t(o + k)] += std::conj(item_at(ph.arena, lx, k, a)) * u[f.x_perm[p]];
      }
    }
    for (int e = 0; e < ap.n_stages; ++e) {
      const TCStage& as = ap.st[e];
      const TCStage& fs = fp.st[fp.n_stages - 1 - e];
      if (as.M_t != fs.K_t || as.K_pad != fs.M_t || as.R_in != fs.R_out || as.R_out != fs.R_in ||
          as.R8_in != fs.R8_out || as.R8_out != fs.R8_in || as.in_pat != fs.out_pat || as.out_pat != fs.in_pat ||
          as.B != fs.B || as.ch != fs.ch || as.n_groups != fs.n_groups)
        fail(MBF_ERR_INVALID, "layout: adjoint stage is not the transposed forward stage");
      std::fill(nxt.begin(), nxt.end(), cd(0.0));
      std::vector<cd> y(size_t(as.M_t));
      for (int64_t grp = 0; grp < as.n_groups; ++grp) {
        const uint8_t* tile = ph.tc_arena.data() + size_t(fs.base) + size_t(grp) * size_t(fs.tile_bytes);
        std::fill(y.begin(), y.end(), cd(0.0));
        for (int k = 0; k < as.K_pad; ++k) {
          const int tp = k / as.R8_in, kk = k % as.R8_in;
          if (kk >= as.R_in) continue;
          const cd x = cur[size_t(seg(as.in_pat, grp, tp, as.B, as.ch, as.R_in, c) + kk)];
          for (int m = 0; m < as.M_t; ++m) y[size_t(m)] += std::conj(tile_at(tile, fs, k, m)) * x;
        }
        if (as.last) {   // V^L: the leaf stage's items hold conj(V)
          const Stage& s0 = ph.plan.st[0];
          const Item& it = item(s0, grp, 0);
          for (int b = 0; b < it.nlines; ++b) {
            const int64_t p = it.base + b;
            const int t = leaf_child(f.w_off, grp, c, p);
            cd s = 0;
            for (int k = 0; k < it.len; ++k) s += std::conj(item_at(ph.arena, it, b, k)) * y[size_t(t * as.R8_out + k)];
            g[f.w_perm[p]] += s;
          }
        } else {
          for (int t = 0; t < c; ++t)
            for (int k2 = 0; k2 < as.R_out; ++k2)
              nxt[size_t(seg(as.out_pat, grp, t, as.B, as.ch, as.R_out, c) + k2)] += y[size_t(t * as.R8_out + k2)];
        }
      }
      std::swap(cur, nxt);
    }
  }
};

}  // namespace

extern "C" {

mbf_status mbf_debug_layout_apply(const mbf_factors_t* f, int32_t path, int32_t adjoint, const void* in, void* out,
                                  int64_t nrhs) {
  return mbf::abi_guard([&] {
    if (!f || (nrhs > 0 && (!in || !out))) fail(MBF_ERR_INVALID, "NULL argument");
    if (nrhs < 0) fail(MBF_ERR_INVALID, "nrhs < 0");
    if (path != 0 && path != 1) fail(MBF_ERR_INVALID, "path must be 0 (SIMT arena) or 1 (tensor tiles)");
    mbf::PackedHost ph;
    mbf::pack_host(*f, ph);
    if (path == 1 && !ph.tc_unavailable.empty()) fail(MBF_ERR_INVALID, "tensor tiles unavailable: " + ph.tc_unavailable);
    if (path == 1 && adjoint && !ph.tc_adj_unavailable.empty())
      fail(MBF_ERR_INVALID, "tensor adjoint unavailable: " + ph.tc_adj_unavailable);
    const Interp ip(*f, ph);
    const int64_t n_src = adjoint ? f->n_out : f->n_in, n_dst = adjoint ? f->n_in : f->n_out;
    const cd* src = static_cast<const cd*>(in);
    cd* dst = static_cast<cd*>(out);
    for (int64_t r = 0; r < nrhs; ++r) {
      cd* o = dst + r * n_dst;
      std::fill(o, o + n_dst, cd(0.0));
      if (path == 1)
        adjoint ? ip.tc_adjoint(src + r * n_src, o) : ip.tc_forward(src + r * n_src, o);
      else if (adjoint)
        ip.simt_adjoint(src + r * n_src, o);
      else
        ip.simt_forward(src + r * n_src, o);
    }
  });
}

mbf_status mbf_factors_device_bytes(const mbf_factors_t* f, int64_t* simt_bytes, int64_t* tensor_bytes) {
  return mbf::abi_guard([&] {
    if (!f) fail(MBF_ERR_INVALID, "NULL argument");
    mbf::PackedHost ph;
    mbf::pack_host(*f, ph);
    if (simt_bytes) *simt_bytes = int64_t(ph.arena.size() + ph.items.size() * sizeof(Item));
    if (tensor_bytes) *tensor_bytes = ph.tc_unavailable.empty() ? int64_t(ph.tc_arena.size()) : 0;
  });
}

}  // extern "C"
