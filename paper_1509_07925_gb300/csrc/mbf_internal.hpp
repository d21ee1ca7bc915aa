// Internal declarations shared by the host translation units of libmbf.
#pragma once

#include <complex>
#include <cstdint>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "mbf.h"

namespace mbf {

using cd = std::complex<double>;

// Error carried to the C ABI boundary, where it becomes an mbf_status.
struct Error : std::runtime_error {
  mbf_status code;
  Error(mbf_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};
[[noreturn]] inline void fail(mbf_status c, const std::string& m) { throw Error(c, m); }
void set_last_error(const std::string& m);

// Runs fn at the C ABI boundary: an mbf::Error becomes its status, a failed host
// allocation MBF_ERR_OOM and any other exception MBF_ERR_INVALID; mbf_last_error() then
// returns the message ("" after a success).  No exception crosses the ABI.
template <class F>
mbf_status abi_guard(F&& fn) noexcept {
  try {
    fn();
    set_last_error("");
    return MBF_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return MBF_ERR_OOM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return MBF_ERR_INVALID;
  }
}

// ---------------------------------------------------------------- trees (§2.2)
// A Z-order tree of depth L stored as the permutation tree order -> point index
// plus the c^L + 1 leaf offsets.  Node i of level l owns leaves
// [i c^(L-l), (i+1) c^(L-l)) and the tree-order range [off[..], off[..]).
struct Tree {
  int d = 2, L = 0, c = 4;
  std::vector<int64_t> perm;   // tree order -> natural index
  std::vector<int64_t> off;    // leaf offsets
  int64_t begin(int level, int64_t i) const { return off[i * ipow(c, L - level)]; }
  int64_t end(int level, int64_t i) const { return off[(i + 1) * ipow(c, L - level)]; }
  int64_t size(int level, int64_t i) const { return end(level, i) - begin(level, i); }
  static int64_t ipow(int64_t b, int e) { int64_t r = 1; while (e-- > 0) r *= b; return r; }
};
Tree tree_uniform(int n, int d, int L);
Tree tree_polar(int n, int L);
Tree tree_square(const std::vector<double>& xi, const std::vector<int64_t>& index, int d,
                 double lo, double side, int L);
int64_t morton(const int64_t* cell, int d, int L);
// The X tree and the Omega tree of a problem, as the builder makes them.
void problem_trees(const mbf_problem_t& prob, Tree& xt, Tree& wt);

// ---------------------------------------------------------------- host factor set
// Owning version of mbf_factors_t (same layout).
struct FactorSet {
  int d = 2, L = 0;
  int64_t n_out = 0, n_in = 0, n_w = 0;
  std::vector<int64_t> x_perm, x_off, w_perm, w_off;
  std::vector<int32_t> RU, RV;
  int32_t max_leaf_x = 1, max_leaf_w = 1;
  std::vector<cd> UL, VL;
  std::vector<std::vector<cd>> G, H;
  std::vector<double> S;
  int64_t nnz = 0;
  std::vector<const double*> Gp, Hp;   // pointer tables for the view
  mbf_factors_t view();
};
// Consistency checks of a factor set (shapes, offsets, permutations, the apply's
// limits); throws MBF_ERR_INVALID.
void validate(const mbf_factors_t& f);
// Factor files (factor_file.cpp): write a validated factor set; read one back
// (MBF_ERR_IO for a missing, truncated, foreign or corrupt file).
void save_factors(const mbf_factors_t& f, const std::string& path);
FactorSet load_factors(const std::string& path);
// build_factors with the checkpoint of opts.factor_file: load the file if it exists
// (checked against the problem), else build and write it.
FactorSet build_or_load(const mbf_problem_t& prob, mbf_entry_fn fn, void* ctx, const mbf_build_opts_t& opts);

// ---------------------------------------------------------------- dense linear algebra
// Column-major complex matrix.
struct Mat {
  int64_t m = 0, n = 0;
  std::vector<cd> a;
  Mat() = default;
  Mat(int64_t m_, int64_t n_) : m(m_), n(n_), a(size_t(m_ * n_)) {}
  cd& operator()(int64_t i, int64_t j) { return a[size_t(i + m * j)]; }
  const cd& operator()(int64_t i, int64_t j) const { return a[size_t(i + m * j)]; }
  cd* col(int64_t j) { return a.data() + m * j; }
  const cd* col(int64_t j) const { return a.data() + m * j; }
};
// sum_i conj(a_i) b_i (linalg.cpp: explicit real arithmetic, a reduction the compiler
// may vectorise).
cd dot_hn(const cd* a, const cd* b, int64_t n);
Mat matmul(const Mat& A, const Mat& B);                 // A B
Mat matmul_hn(const Mat& A, const Mat& B);              // A^* B
Mat adjoint(const Mat& A);
Mat rows_of(const Mat& A, const std::vector<int64_t>& rows);
// Householder QR with column pivoting, stopped after kmax steps or when the
// largest remaining column norm falls below tol * the first.  Returns pivots and,
// if Q != nullptr, the first k orthonormal columns.
std::vector<int64_t> pivoted_qr(const Mat& A, int64_t kmax, double tol, Mat* Q);
// Hermitian eigendecomposition (cyclic Jacobi): A = V diag(w) V^*, w descending.
void eig_herm(const Mat& A, std::vector<double>& w, Mat& V);
// Thin SVD A = U diag(s) V^* (s descending) via one-sided Jacobi; small matrices.
void svd_small(const Mat& A, Mat& U, std::vector<double>& s, Mat& V);
// Moore-Penrose pseudo-inverse with relative cutoff rcond * s_max.
Mat pinv(const Mat& A, double rcond);

// ---------------------------------------------------------------- builder
FactorSet build_factors(const mbf_problem_t& prob, mbf_entry_fn fn, void* ctx,
                        const mbf_build_opts_t& opts);
// Case (i) of §1.1 / §2.3: the middle level from products with K and K^* only.
FactorSet build_factors_from_applies(const mbf_problem_t& prob, mbf_apply_fn afn, void* ctx,
                                     const mbf_build_opts_t& opts);
// Padded factor-set shapes (ranks capped per level, zero arrays) and the algorithmic
// nonzeros from true ranks rank[level][node * c^(L - level) + other] (builder.cpp).
void layout_factor_set(int d, int L, int64_t r, int64_t N_out, int64_t N_in, const Tree& xt, const Tree& wt,
                       FactorSet& fs);
int64_t factor_nnz(int c, int L, const Tree& xt, const Tree& wt, const std::vector<std::vector<int32_t>>& kU,
                   const std::vector<std::vector<int32_t>>& kV);

}  // namespace mbf
