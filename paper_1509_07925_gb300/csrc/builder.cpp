// Host FP64 construction of the butterfly factorization (Case (ii): entries by
// evaluation).  Middle level: §2.3 with the SVD via random sampling of §2.1 and
// the form of eq. (lowrank1).  Recursion: §2.4.1 (U side) and §2.4.2 (V side) --
// splitting (eq. splitandmerge), merging (eq. blocks), truncating (eq. blockF /
// RSh2, form of eq. lowrank2) and assembling into the padded factor set.
//
// Memory: the U side is processed one middle-level X node i at a time (all
// U^h_{i,j}, then the subtree below i); the V side one Omega node j at a time,
// recomputing the middle-level blocks K^h_{i,j} from the same per-block seed.  No
// full U^h or V^h is ever held (the interleaved construction noted in §2.5).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <exception>
#include <mutex>
#include <numeric>
#include <random>
#include <thread>

#include "mbf_internal.hpp"

namespace mbf {

namespace {

struct LowRank {
  Mat U;                    // orthonormal columns U_0
  std::vector<double> s;    // singular values (descending)
  Mat V;                    // orthonormal columns V_0
};

uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Hermitian Gram matrix A^* A (upper triangle computed, lower mirrored).
Mat gram_hn(const Mat& A) {
  Mat C(A.n, A.n);
  for (int64_t j = 0; j < A.n; ++j) {
    const cd* b = A.col(j);
    for (int64_t i = 0; i <= j; ++i) {
      C(i, j) = dot_hn(A.col(i), b, A.m);
      C(j, i) = std::conj(C(i, j));
    }
  }
  return C;
}

// Number of Gram eigenvalues kept: at most r, and only those above cut * w_0.
int64_t keep_count(const std::vector<double>& w, int64_t r, double cut) {
  if (w.empty() || !(w[0] > 0)) return 0;
  int64_t k = 0;
  while (k < int64_t(w.size()) && k < r && w[size_t(k)] > cut * w[0]) ++k;
  return k;
}

// Rank-r truncated SVD Z ~ U_0 diag(s) V_0^* from the eigendecomposition of the
// smaller Gram matrix.  Eigenvalues below gram_cut * lambda_1 are dropped (the Gram
// form resolves singular values down to about sqrt(gram_cut) sigma_1).
LowRank truncated_svd(const Mat& Z, int64_t r, double gram_cut) {
  LowRank out;
  const int64_t m = Z.m, n = Z.n;
  std::vector<double> w;
  Mat E;
  if (m == 0 || n == 0) { out.U = Mat(m, 0); out.V = Mat(n, 0); return out; }
  if (n <= m) {
    eig_herm(gram_hn(Z), w, E);
    const int64_t k = keep_count(w, r, gram_cut);
    out.V = Mat(n, k);
    for (int64_t j = 0; j < k; ++j) std::copy(E.col(j), E.col(j) + n, out.V.col(j));
    Mat ZV = matmul(Z, out.V);
    out.U = Mat(m, k);
    out.s.resize(size_t(k));
    for (int64_t j = 0; j < k; ++j) {
      out.s[size_t(j)] = std::sqrt(w[size_t(j)]);
      for (int64_t i = 0; i < m; ++i) out.U(i, j) = ZV(i, j) / out.s[size_t(j)];
    }
  } else {
    eig_herm(gram_hn(adjoint(Z)), w, E);
    const int64_t k = keep_count(w, r, gram_cut);
    out.U = Mat(m, k);
    for (int64_t j = 0; j < k; ++j) std::copy(E.col(j), E.col(j) + m, out.U.col(j));
    Mat ZhU = matmul_hn(Z, out.U);
    out.V = Mat(n, k);
    out.s.resize(size_t(k));
    for (int64_t j = 0; j < k; ++j) {
      out.s[size_t(j)] = std::sqrt(w[size_t(j)]);
      for (int64_t i = 0; i < n; ++i) out.V(i, j) = ZhU(i, j) / out.s[size_t(j)];
    }
  }
  return out;
}

// B ~ Ufac Gfac in the form of eq. (lowrank2): Ufac = U_0 Sigma_0, Gfac = V_0^*.
void truncate_form2(const Mat& B, int64_t r, double gram_cut, Mat& Ufac, Mat& Gfac) {
  const int64_t m = B.m, n = B.n;
  std::vector<double> w;
  Mat E;
  if (m == 0 || n == 0) { Ufac = Mat(m, 0); Gfac = Mat(0, n); return; }
  if (n <= m) {
    eig_herm(gram_hn(B), w, E);
    const int64_t k = keep_count(w, r, gram_cut);
    Mat V0(n, k);
    for (int64_t j = 0; j < k; ++j) std::copy(E.col(j), E.col(j) + n, V0.col(j));
    Ufac = matmul(B, V0);          // U_0 Sigma_0 = B V_0
    Gfac = adjoint(V0);
  } else {
    eig_herm(gram_hn(adjoint(B)), w, E);
    const int64_t k = keep_count(w, r, gram_cut);
    Mat U0(m, k);
    for (int64_t j = 0; j < k; ++j) std::copy(E.col(j), E.col(j) + m, U0.col(j));
    Ufac = Mat(m, k);
    std::vector<double> s(static_cast<size_t>(k));
    for (int64_t j = 0; j < k; ++j) {
      s[size_t(j)] = std::sqrt(w[size_t(j)]);
      for (int64_t i = 0; i < m; ++i) Ufac(i, j) = U0(i, j) * s[size_t(j)];
    }
    Mat UhB = matmul_hn(U0, B);    // Sigma_0 V_0^* = U_0^* B
    Gfac = Mat(k, n);
    for (int64_t jj = 0; jj < n; ++jj)
      for (int64_t i = 0; i < k; ++i) Gfac(i, jj) = UhB(i, jj) / s[size_t(i)];
  }
}

// Sorted union of `fixed` with random other indices of [0, total), `size` in all.
std::vector<int64_t> supplement(const std::vector<int64_t>& fixed, int64_t total, int64_t size,
                                std::mt19937_64& rng) {
  size = std::min(size, total);
  std::vector<char> used(size_t(total), 0);
  std::vector<int64_t> out;
  for (int64_t f : fixed)
    if (!used[size_t(f)]) { used[size_t(f)] = 1; out.push_back(f); }
  std::vector<int64_t> pool;
  for (int64_t q = 0; q < total; ++q)
    if (!used[size_t(q)]) pool.push_back(q);
  int64_t need = size - int64_t(out.size());
  for (int64_t q = 0; q < need && q < int64_t(pool.size()); ++q) {
    std::uniform_int_distribution<int64_t> pick(q, int64_t(pool.size()) - 1);
    std::swap(pool[size_t(q)], pool[size_t(pick(rng))]);
    out.push_back(pool[size_t(q)]);
  }
  std::sort(out.begin(), out.end());
  return out;
}

std::vector<int64_t> iota_n(int64_t n) {
  std::vector<int64_t> v(static_cast<size_t>(n));
  std::iota(v.begin(), v.end(), 0);
  return v;
}

template <class Entries>
LowRank svd_sampling(const Entries& entries, int64_t m, int64_t n, int64_t r, std::mt19937_64& rng,
                     const mbf_build_opts_t& o, double gram_cut) {
  const int64_t s = int64_t(o.sample_factor) * r;
  if (m == 0 || n == 0 || r == 0) return truncated_svd(Mat(m, n), r, gram_cut);
  if (s >= m || s >= n) return truncated_svd(entries(iota_n(m), iota_n(n)), r, gram_cut);
  std::vector<int64_t> rows_rep, cols_rep;
  const std::vector<int64_t> all_r = iota_n(m), all_c = iota_n(n);
  for (int round = 0; round < o.max_rounds; ++round) {
    // representative columns from a pivoted QR of the sampled rows, then rows from
    // a pivoted QR of the (adjoint of the) sampled columns (§2.1, first stage)
    const auto I = supplement(rows_rep, m, s, rng);
    auto new_cols = pivoted_qr(entries(I, all_c), r, 0.0, nullptr);
    std::sort(new_cols.begin(), new_cols.end());
    const auto J = supplement(new_cols, n, s, rng);
    auto new_rows = pivoted_qr(adjoint(entries(all_r, J)), r, 0.0, nullptr);
    std::sort(new_rows.begin(), new_rows.end());
    const bool stable = new_rows == rows_rep && new_cols == cols_rep;
    rows_rep = std::move(new_rows);
    cols_rep = std::move(new_cols);
    if (stable) break;
  }
  // bases of the column and row spaces (§2.1, second stage)
  Mat Qc, Qr;
  pivoted_qr(entries(all_r, cols_rep), r, 1e-14, &Qc);
  pivoted_qr(adjoint(entries(rows_rep, all_c)), r, 1e-14, &Qr);
  // M from the restriction to I_row x I_col (§2.1, third stage)
  const auto Irow = supplement(rows_rep, m, s, rng);
  const auto Icol = supplement(cols_rep, n, s, rng);
  Mat Zs = entries(Irow, Icol);
  Mat M = matmul(matmul(pinv(rows_of(Qc, Irow), 1e-15 * double(Irow.size())), Zs),
                 pinv(adjoint(rows_of(Qr, Icol)), 1e-15 * double(Icol.size())));
  // SVD of M (§2.1, last stage)
  Mat Um, Vm;
  std::vector<double> sm;
  svd_small(M, Um, sm, Vm);
  int64_t k = 0;
  while (k < int64_t(sm.size()) && k < r && sm[size_t(k)] > o.tol * sm[0]) ++k;
  LowRank out;
  Mat Uk(Um.m, k), Vk(Vm.m, k);
  for (int64_t j = 0; j < k; ++j) {
    std::copy(Um.col(j), Um.col(j) + Um.m, Uk.col(j));
    std::copy(Vm.col(j), Vm.col(j) + Vm.m, Vk.col(j));
  }
  out.U = matmul(Qc, Uk);
  out.V = matmul(Qr, Vk);
  out.s.assign(sm.begin(), sm.begin() + k);
  return out;
}

// SVD via random matrix-vector multiplication (§2.1, first procedure), from the products
// Y = Z C (m x p) and W = Z^* R (n x p) with the Gaussian matrices C (n x p), R (m x p):
// Q_col, Q_row from pivoted QRs of Y and W (first r columns), M = (R^* Q_col)^+ (W^* C)
// (Q_row^* C)^+ (R^* Z C = W^* C), and the SVD of M, truncated at rank r and tol sigma_1.
LowRank svd_matvec(const Mat& Y, const Mat& W, const Mat& C, const Mat& R, int64_t r, double tol) {
  LowRank out;
  const int64_t m = Y.m, n = W.m;
  if (m == 0 || n == 0 || r == 0) {
    out.U = Mat(m, 0);
    out.V = Mat(n, 0);
    return out;
  }
  Mat Qc, Qr;
  pivoted_qr(Y, r, 1e-14, &Qc);
  pivoted_qr(W, r, 1e-14, &Qr);
  const Mat A1 = matmul_hn(R, Qc);     // R^* Q_col
  const Mat A2 = matmul_hn(W, C);      // W^* C = R^* Z C
  const Mat A3 = matmul_hn(Qr, C);     // Q_row^* C
  const Mat M = matmul(matmul(pinv(A1, 1e-15 * double(A1.m)), A2), pinv(A3, 1e-15 * double(A3.n)));
  Mat Um, Vm;
  std::vector<double> sm;
  svd_small(M, Um, sm, Vm);
  int64_t k = 0;
  while (k < int64_t(sm.size()) && k < r && sm[size_t(k)] > tol * sm[0]) ++k;
  Mat Uk(Um.m, k), Vk(Vm.m, k);
  for (int64_t q = 0; q < k; ++q) {
    std::copy(Um.col(q), Um.col(q) + Um.m, Uk.col(q));
    std::copy(Vm.col(q), Vm.col(q) + Vm.m, Vk.col(q));
  }
  out.U = matmul(Qc, Uk);
  out.V = matmul(Qr, Vk);
  out.s.assign(sm.begin(), sm.begin() + k);
  return out;
}

// Complex Gaussian matrix (a + i b)/sqrt(2), m x p, from a seeded generator.
Mat gaussian(int64_t m, int64_t p, uint64_t seed) {
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  Mat G(m, p);
  for (int64_t q = 0; q < m * p; ++q) {
    const double a = nd(rng), b = nd(rng);
    G.a[size_t(q)] = cd(a, b) / std::sqrt(2.0);
  }
  return G;
}

template <class F>
void parallel_for(int64_t count, int threads, F&& fn) {
  std::atomic<int64_t> next{0};
  std::exception_ptr err;
  std::mutex mu;
  auto worker = [&]() {
    for (;;) {
      const int64_t q = next.fetch_add(1);
      if (q >= count) return;
      try {
        fn(q);
      } catch (...) {
        std::lock_guard<std::mutex> lk(mu);
        if (!err) err = std::current_exception();
        next.store(count);
        return;
      }
    }
  };
  const int nt = int(std::max<int64_t>(1, std::min<int64_t>(threads, count)));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  if (err) std::rethrow_exception(err);
}

}  // namespace

// The X tree (uniform) and the Omega tree of a problem (§2.2; §3.2 polar; §4.2 square
// over a corona).  Frequencies: grid digit - n / 2 per axis, natural row-major order.
void problem_trees(const mbf_problem_t& prob, Tree& xt, Tree& wt) {
  const int d = prob.dim, n = prob.n, L = prob.L;
  if (d != 2 && d != 3) fail(MBF_ERR_INVALID, "dim must be 2 or 3");
  if (L < 2 || (L % 2) != 0) fail(MBF_ERR_INVALID, "L must be even and >= 2");
  if (prob.tree != MBF_TREE_POINTS) {
    if (n < 2 || (n & (n - 1)) != 0) fail(MBF_ERR_INVALID, "n must be a power of two");
    xt = tree_uniform(n, d, L);
  }
  if (prob.tree == MBF_TREE_UNIFORM) {
    wt = tree_uniform(n, d, L);
  } else if (prob.tree == MBF_TREE_POLAR) {
    if (d != 2) fail(MBF_ERR_INVALID, "polar tree needs dim 2");
    wt = tree_polar(n, L);
  } else if (prob.tree == MBF_TREE_POINTS) {
    if (!prob.x_pts || !prob.w_pts || prob.n_x_pts <= 0 || prob.n_w_pts <= 0)
      fail(MBF_ERR_INVALID, "explicit point sets need x_pts and w_pts");
    if (!(prob.w_side > 0)) fail(MBF_ERR_INVALID, "explicit point sets need w_side > 0");
    std::vector<double> xp(prob.x_pts, prob.x_pts + prob.n_x_pts * d), wp(prob.w_pts, prob.w_pts + prob.n_w_pts * d);
    for (double v : xp)
      if (!(v >= 0.0 && v < 1.0)) fail(MBF_ERR_INVALID, "x_pts outside [0,1)^dim");
    for (double v : wp)
      if (!(v >= prob.w_lo && v < prob.w_lo + prob.w_side)) fail(MBF_ERR_INVALID, "w_pts outside the square");
    std::vector<int64_t> xi(size_t(prob.n_x_pts)), wi(size_t(prob.n_w_pts));
    for (int64_t q = 0; q < prob.n_x_pts; ++q) xi[size_t(q)] = q;
    for (int64_t q = 0; q < prob.n_w_pts; ++q) wi[size_t(q)] = q;
    xt = tree_square(xp, xi, d, 0.0, 1.0, L);
    wt = tree_square(wp, wi, d, prob.w_lo, prob.w_side, L);
  } else if (prob.tree == MBF_TREE_SQUARE) {
    if (!prob.w_index || prob.n_w <= 0) fail(MBF_ERR_INVALID, "square tree needs w_index");
    if (!(prob.w_side > 0)) fail(MBF_ERR_INVALID, "square tree needs w_side > 0");
    const int64_t N = Tree::ipow(n, d);
    std::vector<int64_t> idx(prob.w_index, prob.w_index + prob.n_w);
    std::vector<double> pts(static_cast<size_t>(prob.n_w * d));
    for (int64_t q = 0; q < prob.n_w; ++q) {
      if (idx[size_t(q)] < 0 || idx[size_t(q)] >= N) fail(MBF_ERR_INVALID, "w_index out of range");
      int64_t rest = idx[size_t(q)];
      for (int k = d - 1; k >= 0; --k) {
        pts[size_t(q * d + k)] = double(rest % n) - double(n / 2);
        rest /= n;
      }
    }
    wt = tree_square(pts, idx, d, prob.w_lo, prob.w_side, L);
  } else {
    fail(MBF_ERR_INVALID, "unknown tree kind");
  }
}

// Shapes of the padded factor set of a problem (the interchange layout of mbf_factors_t):
// padded rank caps R_h = min(r, max |A^h|, max |B^h|), R_{l+1} = min(r, max |node at l+1|,
// c R_l) on each side, leaf arrays at the largest leaf, every array zero.
void layout_factor_set(int d, int L, int64_t r, int64_t N_out, int64_t N_in, const Tree& xt, const Tree& wt,
                       FactorSet& fs) {
  const int c = 1 << d, h = L / 2;
  auto max_size = [&](const Tree& T, int l) {
    int64_t mx = 0;
    for (int64_t i = 0; i < Tree::ipow(c, l); ++i) mx = std::max(mx, T.size(l, i));
    return mx;
  };
  fs.d = d;
  fs.L = L;
  fs.n_out = N_out;
  fs.n_in = N_in;
  fs.n_w = int64_t(wt.perm.size());
  fs.RU.assign(size_t(L + 1), 0);
  fs.RV.assign(size_t(L + 1), 0);
  const int64_t Rh = std::max<int64_t>(1, std::min({r, max_size(xt, h), max_size(wt, L - h)}));
  fs.RU[size_t(h)] = fs.RV[size_t(h)] = int32_t(Rh);
  for (int l = h; l < L; ++l) {
    fs.RU[size_t(l + 1)] = int32_t(std::max<int64_t>(1, std::min({r, max_size(xt, l + 1), c * int64_t(fs.RU[size_t(l)])})));
    fs.RV[size_t(l + 1)] = int32_t(std::max<int64_t>(1, std::min({r, max_size(wt, l + 1), c * int64_t(fs.RV[size_t(l)])})));
  }
  fs.max_leaf_x = int32_t(std::max<int64_t>(1, max_size(xt, L)));
  fs.max_leaf_w = int32_t(std::max<int64_t>(1, max_size(wt, L)));
  const int64_t nL = Tree::ipow(c, L);
  fs.UL.assign(size_t(nL * fs.max_leaf_x * fs.RU[size_t(L)]), cd(0));
  fs.VL.assign(size_t(nL * fs.max_leaf_w * fs.RV[size_t(L)]), cd(0));
  fs.G.resize(size_t(L - h));
  fs.H.resize(size_t(L - h));
  for (int l = h; l < L; ++l) {
    fs.G[size_t(l - h)].assign(size_t(nL * c * fs.RU[size_t(l + 1)] * fs.RU[size_t(l)]), cd(0));
    fs.H[size_t(l - h)].assign(size_t(nL * c * fs.RV[size_t(l + 1)] * fs.RV[size_t(l)]), cd(0));
  }
  fs.S.assign(size_t(Tree::ipow(c, 2 * h) * Rh), 0.0);
  fs.x_perm = xt.perm;
  fs.x_off = xt.off;
  fs.w_perm = wt.perm;
  fs.w_off = wt.off;
}

// Algorithmic nonzeros of the unpadded factors (§2.5: the apply cost) from the true
// ranks rank[side][level][node * c^(L - level) + other].
int64_t factor_nnz(int c, int L, const Tree& xt, const Tree& wt, const std::vector<std::vector<int32_t>>& kU,
                   const std::vector<std::vector<int32_t>>& kV) {
  const int h = L / 2;
  const int64_t nL = Tree::ipow(c, L), nh = Tree::ipow(c, h);
  int64_t nnz = 0;
  for (int64_t q = 0; q < nL; ++q) {
    nnz += (xt.off[size_t(q + 1)] - xt.off[size_t(q)]) * kU[size_t(L)][size_t(q)];
    nnz += (wt.off[size_t(q + 1)] - wt.off[size_t(q)]) * kV[size_t(L)][size_t(q)];
  }
  for (int64_t q = 0; q < nh * nh; ++q) nnz += kU[size_t(h)][size_t(q)];
  for (int side = 0; side < 2; ++side) {
    auto& K = side == 0 ? kU : kV;
    for (int l = h; l < L; ++l) {
      const int64_t njp = Tree::ipow(c, L - l - 1);
      for (int64_t node = 0; node < Tree::ipow(c, l); ++node)
        for (int64_t jp = 0; jp < njp; ++jp) {
          int64_t kin = 0;
          for (int tp = 0; tp < c; ++tp) kin += K[size_t(l)][size_t(node * njp * c + c * jp + tp)];
          for (int t = 0; t < c; ++t) nnz += kin * K[size_t(l + 1)][size_t((c * node + t) * njp + jp)];
        }
    }
  }
  return nnz;
}

namespace {

struct Builder {
  const mbf_problem_t& prob;
  mbf_entry_fn fn;
  void* ctx;
  // Case (i) (§2.3): the operator is known only through products with K and K^*
  mbf_apply_fn afn = nullptr;
  int64_t p_over = 8;          // oversampling k of the random products
  Mat KC;                      // [n_out][c^h p]: K C^P_j for every Omega node j (natural rows)
  Mat KhR;                     // [n_in][c^h p]: K^* R^P_i for every X node i
  mbf_build_opts_t opts;
  int d, n, L, h, c;
  int64_t r;
  double gram_cut;
  Tree xt, wt;
  std::vector<double> xcoord;   // [N_x][d]
  std::vector<double> wcoord;   // coordinates of input point q (natural index) [n_in][d]
  FactorSet fs;
  // true ranks: rank[side][level] as [c^l][c^(L-l)]
  std::vector<std::vector<int32_t>> kU, kV;

  Builder(const mbf_problem_t& p, mbf_entry_fn f, void* cx, const mbf_build_opts_t& o)
      : prob(p), fn(f), ctx(cx), opts(o) {}

  static int64_t ip(int64_t b, int e) { return Tree::ipow(b, e); }

  Mat eval_block(const std::vector<int64_t>& xr, const std::vector<int64_t>& wc) const {
    const int64_t m = int64_t(xr.size()), nn = int64_t(wc.size());
    std::vector<double> xs(static_cast<size_t>(m * d)), ws(static_cast<size_t>(nn * d));
    for (int64_t a = 0; a < m; ++a)
      for (int k = 0; k < d; ++k) xs[size_t(a * d + k)] = xcoord[size_t(xr[size_t(a)] * d + k)];
    for (int64_t b = 0; b < nn; ++b)
      for (int k = 0; k < d; ++k) ws[size_t(b * d + k)] = wcoord[size_t(wc[size_t(b)] * d + k)];
    Mat Z(m, nn);
    if (m > 0 && nn > 0) fn(xs.data(), m, ws.data(), nn, d, reinterpret_cast<double*>(Z.a.data()), ctx);
    return Z;
  }

  // Middle-level block K^h_{i,j} (§2.3) by the SVD via random sampling; identical
  // for the U and the V pass because the generator depends on (seed, i, j) only.
  // Case (i) random matrices: C_j (|B_j| x p) and R_i (|A_i| x p), seeded per node.
  Mat case1_C(int64_t j) const {
    return gaussian(wt.size(L - h, j), r + p_over, mix64(opts.seed ^ 0x4331000000000000ULL ^ uint64_t(j)));
  }
  Mat case1_R(int64_t i) const {
    return gaussian(xt.size(h, i), r + p_over, mix64(opts.seed ^ 0x5231000000000000ULL ^ uint64_t(i)));
  }

  // Case (i): K C^P_j and K^* R^P_i for all nodes through the black box (§2.3), the
  // zero-padded random matrices applied in chunks of at most 256 vectors.
  void case1_products() {
    const int64_t nh = ip(c, h), p = r + p_over;
    const int64_t n_out = fs.n_out, n_in = fs.n_in;
    KC = Mat(n_out, nh * p);
    KhR = Mat(n_in, nh * p);
    for (int side = 0; side < 2; ++side) {
      const int64_t len_in = side == 0 ? n_in : n_out, len_out = side == 0 ? n_out : n_in;
      Mat& dst = side == 0 ? KC : KhR;
      const int64_t total = nh * p;
      for (int64_t v0 = 0; v0 < total; v0 += 256) {
        const int64_t nv = std::min<int64_t>(256, total - v0);
        std::vector<double> in(size_t(2 * nv * len_in), 0.0), out(size_t(2 * nv * len_out), 0.0);
        for (int64_t node = v0 / p; node <= (v0 + nv - 1) / p; ++node) {
          const Mat G = side == 0 ? case1_C(node) : case1_R(node);
          const Tree& T = side == 0 ? wt : xt;
          const int lev = side == 0 ? L - h : h;
          const int64_t b0 = T.begin(lev, node);
          for (int64_t q = 0; q < p; ++q) {
            const int64_t v = node * p + q - v0;
            if (v < 0 || v >= nv) continue;
            for (int64_t a = 0; a < G.m; ++a) {
              const int64_t nat = T.perm[size_t(b0 + a)];
              in[size_t(2 * (v * len_in + nat))] = G(a, q).real();
              in[size_t(2 * (v * len_in + nat) + 1)] = G(a, q).imag();
            }
          }
        }
        afn(in.data(), out.data(), nv, side, ctx);
        for (int64_t v = 0; v < nv; ++v)
          for (int64_t row = 0; row < len_out; ++row)
            dst(row, v0 + v) = cd(out[size_t(2 * (v * len_out + row))], out[size_t(2 * (v * len_out + row) + 1)]);
      }
    }
  }

  LowRank middle(int64_t i, int64_t j) const {
    const int64_t xb = xt.begin(h, i), xe = xt.end(h, i);
    const int64_t wb = wt.begin(L - h, j), we = wt.end(L - h, j);
    if (afn) {
      // Case (i): Y = K^h_{i,j} C_j = rows A_i of K C^P_j; W = (K^h_{i,j})^* R_i = rows B_j of
      // K^* R^P_i (§2.3); then the SVD via random matrix-vector multiplication (§2.1)
      const int64_t p = r + p_over;
      Mat Y(xe - xb, p), W(we - wb, p);
      for (int64_t q = 0; q < p; ++q) {
        for (int64_t a = 0; a < Y.m; ++a) Y(a, q) = KC(xt.perm[size_t(xb + a)], j * p + q);
        for (int64_t b = 0; b < W.m; ++b) W(b, q) = KhR(wt.perm[size_t(wb + b)], i * p + q);
      }
      return svd_matvec(Y, W, case1_C(j), case1_R(i), r, opts.tol);
    }
    std::mt19937_64 rng(mix64(opts.seed ^ mix64(uint64_t(i) * 0x10001ULL + uint64_t(j) + 1)));
    auto entries = [&](const std::vector<int64_t>& ri, const std::vector<int64_t>& ci) {
      std::vector<int64_t> xr(ri.size()), wc(ci.size());
      for (size_t a = 0; a < ri.size(); ++a) xr[a] = xt.perm[size_t(xb + ri[a])];
      for (size_t b = 0; b < ci.size(); ++b) wc[b] = wt.perm[size_t(wb + ci[b])];
      return eval_block(xr, wc);
    };
    return svd_sampling(entries, xe - xb, we - wb, r, rng, opts, gram_cut);
  }

  // One side of the recursive factorization for the middle-level node `own` of the
  // tree `T`: side 0 = U (own = X node i), side 1 = V (own = Omega node j).
  void side_pass(int side, int64_t own) {
    const Tree& T = side == 0 ? xt : wt;
    auto& R = side == 0 ? fs.RU : fs.RV;
    auto& mats = side == 0 ? fs.G : fs.H;
    auto& ranks = side == 0 ? kU : kV;
    const int64_t nh = ip(c, h);
    // U^h_{i,j} = U_0 Sigma_0 (or V^h_{j,i} = V_0 Sigma_0), eq. (Kij)
    std::vector<Mat> cur(static_cast<size_t>(nh));
    for (int64_t other = 0; other < nh; ++other) {
      const LowRank lr = side == 0 ? middle(own, other) : middle(other, own);
      const Mat& B = side == 0 ? lr.U : lr.V;
      const int64_t k = int64_t(lr.s.size());
      Mat F(B.m, k);
      for (int64_t q = 0; q < k; ++q)
        for (int64_t a = 0; a < B.m; ++a) F(a, q) = B(a, q) * lr.s[size_t(q)];
      cur[size_t(other)] = std::move(F);
      ranks[size_t(h)][size_t(own * nh + other)] = int32_t(k);
      if (side == 0)
        for (int64_t q = 0; q < k; ++q)
          fs.S[size_t((own * nh + other) * R[size_t(h)] + q)] = 1.0 / lr.s[size_t(q)];
    }
    // recursion l = h .. L-1 within the subtree of `own`
    for (int l = h; l < L; ++l) {
      const int64_t nloc = ip(c, l - h), nj = ip(c, L - l), njp = nj / c;
      const int64_t R1 = R[size_t(l)], R2 = R[size_t(l + 1)];
      std::vector<cd>& A = mats[size_t(l - h)];
      std::vector<Mat> nxt(static_cast<size_t>(nloc * c * njp));
      for (int64_t a = 0; a < nloc; ++a) {
        const int64_t node = own * nloc + a;
        const int64_t nb = T.begin(l, node);
        for (int t = 0; t < c; ++t) {
          const int64_t child = c * node + t;
          const int64_t cb = T.begin(l + 1, child) - nb, ce = T.end(l + 1, child) - nb;
          for (int64_t jp = 0; jp < njp; ++jp) {
            // merging (eq. blocks): [U^{l,t}_{node, c jp + 0} ... U^{l,t}_{node, c jp + c-1}]
            int64_t cols = 0;
            for (int tp = 0; tp < c; ++tp) cols += cur[size_t(a * nj + c * jp + tp)].n;
            Mat Bm(ce - cb, cols);
            int64_t col0 = 0;
            std::vector<int64_t> widths(static_cast<size_t>(c));
            for (int tp = 0; tp < c; ++tp) {
              const Mat& P = cur[size_t(a * nj + c * jp + tp)];
              widths[size_t(tp)] = P.n;
              for (int64_t q = 0; q < P.n; ++q)
                for (int64_t rr = cb; rr < ce; ++rr) Bm(rr - cb, col0 + q) = P(rr, q);
              col0 += P.n;
            }
            Mat Unew, Gm;
            truncate_form2(Bm, r, gram_cut, Unew, Gm);   // truncating, eq. (blockF)/(RSh2)
            const int64_t k2 = Gm.m;
            ranks[size_t(l + 1)][size_t(child * njp + jp)] = int32_t(k2);
            // assembling: padded [node][jp][t][k2][tp][k]
            int64_t q0 = 0;
            for (int tp = 0; tp < c; ++tp) {
              for (int64_t q = 0; q < widths[size_t(tp)]; ++q)
                for (int64_t kk = 0; kk < k2; ++kk) {
                  const int64_t off = ((((node * njp + jp) * c + t) * R2 + kk) * c + tp) * R1 + q;
                  A[size_t(off)] = Gm(kk, q0 + q);
                }
              q0 += widths[size_t(tp)];
            }
            nxt[size_t((a * c + t) * njp + jp)] = std::move(Unew);
          }
        }
      }
      cur = std::move(nxt);
    }
    // leaves: U^L_i (or V^L_j), rows in tree order
    const int64_t nleaf = ip(c, L - h);
    const int64_t RL = R[size_t(L)];
    const int32_t mx = side == 0 ? fs.max_leaf_x : fs.max_leaf_w;
    std::vector<cd>& Leaf = side == 0 ? fs.UL : fs.VL;
    for (int64_t a = 0; a < nleaf; ++a) {
      const int64_t leaf = own * nleaf + a;
      const Mat& P = cur[size_t(a)];
      for (int64_t row = 0; row < P.m; ++row)
        for (int64_t q = 0; q < P.n; ++q) Leaf[size_t((leaf * mx + row) * RL + q)] = P(row, q);
    }
  }

  void run() {
    d = prob.dim;
    n = prob.n;
    L = prob.L;
    r = prob.r;
    c = 1 << d;
    h = L / 2;
    if (d != 2 && d != 3) fail(MBF_ERR_INVALID, "dim must be 2 or 3");
    if (prob.tree != MBF_TREE_POINTS && (n < 2 || (n & (n - 1)) != 0))
      fail(MBF_ERR_INVALID, "n must be a power of two");
    if (L < 2 || (L % 2) != 0) fail(MBF_ERR_INVALID, "L must be even and >= 2");
    if (r < 1) fail(MBF_ERR_INVALID, "r must be >= 1");
    if (!fn && !afn) fail(MBF_ERR_INVALID, "entry function is NULL");
    if (opts.sample_factor <= 0) opts.sample_factor = 3;
    if (opts.max_rounds <= 0) opts.max_rounds = 3;
    if (!(opts.tol > 0)) opts.tol = 1e-14;
    if (opts.threads <= 0) opts.threads = int(std::max(1u, std::thread::hardware_concurrency()));
    gram_cut = std::max(opts.tol * opts.tol, 1e-13);

    int64_t N_out = 0, N_in = 0;
    if (prob.tree == MBF_TREE_POINTS) {
      // explicit point sets (§2.6): coordinates as given, natural order = array order
      N_out = prob.n_x_pts;
      N_in = prob.n_w_pts;
      if (prob.x_pts && prob.w_pts && N_out > 0 && N_in > 0) {
        xcoord.assign(prob.x_pts, prob.x_pts + N_out * d);
        wcoord.assign(prob.w_pts, prob.w_pts + N_in * d);
      }
    } else {
      int64_t N = 1;
      for (int k = 0; k < d; ++k) N *= n;
      N_out = N_in = N;
      xcoord.resize(size_t(N * d));
      wcoord.resize(size_t(N * d));
      for (int64_t p = 0; p < N; ++p) {
        int64_t q = p;
        for (int k = d - 1; k >= 0; --k) {
          const int64_t digit = q % n;
          q /= n;
          xcoord[size_t(p * d + k)] = double(digit) / double(n);
          wcoord[size_t(p * d + k)] = double(digit) - double(n / 2);
        }
      }
    }
    problem_trees(prob, xt, wt);

    layout_factor_set(d, L, r, N_out, N_in, xt, wt, fs);
    kU.assign(size_t(L + 1), {});
    kV.assign(size_t(L + 1), {});
    const int64_t nL = ip(c, L);
    for (int l = h; l <= L; ++l) {
      kU[size_t(l)].assign(size_t(nL), 0);
      kV[size_t(l)].assign(size_t(nL), 0);
    }

    if (afn) case1_products();
    const int64_t nh = ip(c, h);
    parallel_for(nh, opts.threads, [&](int64_t i) { side_pass(0, i); });
    parallel_for(nh, opts.threads, [&](int64_t j) { side_pass(1, j); });

    const int64_t nnz = factor_nnz(c, L, xt, wt, kU, kV);
    fs.nnz = nnz;
  }
};

}  // namespace

FactorSet build_factors(const mbf_problem_t& prob, mbf_entry_fn fn, void* ctx,
                        const mbf_build_opts_t& opts) {
  Builder b(prob, fn, ctx, opts);
  b.run();
  return std::move(b.fs);
}

FactorSet build_factors_from_applies(const mbf_problem_t& prob, mbf_apply_fn afn, void* ctx,
                                     const mbf_build_opts_t& opts) {
  if (!afn) fail(MBF_ERR_INVALID, "apply function is NULL");
  if (prob.tree == MBF_TREE_SQUARE) fail(MBF_ERR_INVALID, "construction from applies takes whole grids or point sets");
  Builder b(prob, nullptr, ctx, opts);
  b.afn = afn;
  b.run();
  return std::move(b.fs);
}

mbf_factors_t FactorSet::view() {
  mbf_factors_t v{};
  v.dim = d;
  v.L = L;
  v.n_out = n_out;
  v.n_in = n_in;
  v.n_w = n_w;
  v.x_perm = x_perm.data();
  v.x_off = x_off.data();
  v.w_perm = w_perm.data();
  v.w_off = w_off.data();
  v.RU = RU.data();
  v.RV = RV.data();
  v.max_leaf_x = max_leaf_x;
  v.max_leaf_w = max_leaf_w;
  v.UL = reinterpret_cast<const double*>(UL.data());
  v.VL = reinterpret_cast<const double*>(VL.data());
  Gp.clear();
  Hp.clear();
  for (auto& g : G) Gp.push_back(reinterpret_cast<const double*>(g.data()));
  for (auto& hh : H) Hp.push_back(reinterpret_cast<const double*>(hh.data()));
  v.G = Gp.data();
  v.H = Hp.data();
  v.S = S.data();
  v.nnz = nnz;
  return v;
}

}  // namespace mbf
