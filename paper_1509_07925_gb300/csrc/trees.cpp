// Z-order trees over point sets (§2.2, Fig. 1; non-uniform point sets §2.6) and
// the polar image of Omega (§3.1, eq. polar).
#include <algorithm>
#include <cmath>

#include "mbf_internal.hpp"

namespace mbf {

// Z-order index at level L: one base-2^d digit per level, the first coordinate
// supplying the most significant bit of each digit (Fig. 1: t = 2 bit(x_1) + bit(x_2)).
int64_t morton(const int64_t* cell, int d, int L) {
  int64_t m = 0;
  for (int b = L - 1; b >= 0; --b) {
    int64_t digit = 0;
    for (int k = 0; k < d; ++k) digit |= ((cell[k] >> b) & 1) << (d - 1 - k);
    m = (m << d) | digit;
  }
  return m;
}

// Counting sort of points by leaf; ties keep the order of `index` (natural order).
static Tree make_tree(const std::vector<int64_t>& leaf, const std::vector<int64_t>& index, int d,
                      int L) {
  Tree t;
  t.d = d;
  t.L = L;
  t.c = 1 << d;
  const int64_t nl = Tree::ipow(t.c, L);
  t.off.assign(size_t(nl + 1), 0);
  for (int64_t q : leaf) t.off[size_t(q + 1)]++;
  for (int64_t q = 0; q < nl; ++q) t.off[size_t(q + 1)] += t.off[size_t(q)];
  std::vector<int64_t> pos(t.off.begin(), t.off.end() - 1);
  t.perm.assign(leaf.size(), 0);
  for (size_t p = 0; p < leaf.size(); ++p) t.perm[size_t(pos[size_t(leaf[p])]++)] = index[p];
  return t;
}

static int ilog2(int64_t n) {
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return l;
}

Tree tree_uniform(int n, int d, int L) {
  const int shift = ilog2(n) - L;
  if (shift < 0) fail(MBF_ERR_INVALID, "tree depth L exceeds log2(n)");
  int64_t N = 1;
  for (int k = 0; k < d; ++k) N *= n;
  std::vector<int64_t> leaf(static_cast<size_t>(N)), index(static_cast<size_t>(N));
  int64_t cell[3];
  for (int64_t p = 0; p < N; ++p) {
    int64_t r = p;
    for (int k = d - 1; k >= 0; --k) {
      cell[k] = (r % n) >> shift;
      r /= n;
    }
    leaf[size_t(p)] = morton(cell, d, L);
    index[size_t(p)] = p;
  }
  return make_tree(leaf, index, d, L);
}

static Tree tree_unit_cube(const std::vector<double>& p, const std::vector<int64_t>& index, int d,
                           int L) {
  const int64_t npts = int64_t(index.size());
  const int64_t side = int64_t(1) << L;
  std::vector<int64_t> leaf(static_cast<size_t>(npts));
  int64_t cell[3];
  for (int64_t q = 0; q < npts; ++q) {
    for (int k = 0; k < d; ++k) {
      int64_t c = int64_t(std::floor(p[size_t(q * d + k)] * double(side)));
      cell[k] = std::min(std::max<int64_t>(c, 0), side - 1);
    }
    leaf[size_t(q)] = morton(cell, d, L);
  }
  return make_tree(leaf, index, d, L);
}

// Tree over P = p(Omega): p_1 = sqrt(2)|xi|/n (clamped to 1), p_2 = atan2(xi_2, xi_1)/(2 pi)
// mod 1, the inverse of eq. (polar).  Points keep their natural Omega index.
Tree tree_polar(int n, int L) {
  const int64_t N = int64_t(n) * n;
  std::vector<double> p(static_cast<size_t>(2 * N));
  std::vector<int64_t> index(static_cast<size_t>(N));
  const double two_pi = 2.0 * 3.14159265358979323846;
  for (int64_t q = 0; q < N; ++q) {
    const double x1 = double(q / n) - n / 2, x2 = double(q % n) - n / 2;
    double p1 = std::sqrt(2.0) * std::sqrt(x1 * x1 + x2 * x2) / double(n);
    double p2 = std::atan2(x2, x1) / two_pi;
    p2 = p2 - std::floor(p2);
    if (p2 >= 1.0) p2 = 0.0;
    p[size_t(2 * q)] = std::min(p1, 1.0);
    p[size_t(2 * q + 1)] = p2;
    index[size_t(q)] = q;
  }
  return tree_unit_cube(p, index, 2, L);
}

Tree tree_square(const std::vector<double>& xi, const std::vector<int64_t>& index, int d,
                 double lo, double side, int L) {
  std::vector<double> p(xi.size());
  for (size_t q = 0; q < xi.size(); ++q) p[q] = (xi[q] - lo) / side;
  return tree_unit_cube(p, index, d, L);
}

}  // namespace mbf
