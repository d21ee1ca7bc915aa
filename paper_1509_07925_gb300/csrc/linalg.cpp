// Dense complex FP64 linear algebra for the host builder: pivoted Householder QR,
// Hermitian eigensolver (Householder tridiagonalisation + implicit QL), one-sided
// Jacobi SVD and the pseudo-inverse.  These are the primitives of §2.1 (truncated
// SVD, pivoted QR, pseudo-inverse); all arithmetic is FP64.
#include <algorithm>
#include <cmath>
#include <limits>
#include <numeric>

#include "mbf_internal.hpp"

namespace mbf {

static inline double norm2(const cd* x, int64_t n) {
  const double* a = reinterpret_cast<const double*>(x);
  double s = 0;
#pragma omp simd reduction(+ : s)
  for (int64_t i = 0; i < 2 * n; ++i) s += a[i] * a[i];
  return s;
}

cd dot_hn(const cd* a, const cd* b, int64_t n) {
  const double* x = reinterpret_cast<const double*>(a);
  const double* y = reinterpret_cast<const double*>(b);
  double re = 0, im = 0;
#pragma omp simd reduction(+ : re, im)
  for (int64_t i = 0; i < n; ++i) {
    re += x[2 * i] * y[2 * i] + x[2 * i + 1] * y[2 * i + 1];
    im += x[2 * i] * y[2 * i + 1] - x[2 * i + 1] * y[2 * i];
  }
  return cd(re, im);
}

// w -= tau (v^* w) v for one column w of length n: the reflector I - tau v v^* applied
// to w, in explicit real arithmetic on the interleaved (re, im) pairs (std::complex's
// operator* carries NaN-recovery branches that keep these loops from vectorising).
static inline void reflect(const cd* v, double tau, cd* w, int64_t n) {
  const double* a = reinterpret_cast<const double*>(v);
  double* b = reinterpret_cast<double*>(w);
  const cd s = dot_hn(v, w, n) * tau;
  const double sr = s.real(), si = s.imag();
  for (int64_t i = 0; i < n; ++i) {
    b[2 * i] -= sr * a[2 * i] - si * a[2 * i + 1];
    b[2 * i + 1] -= sr * a[2 * i + 1] + si * a[2 * i];
  }
}

Mat matmul(const Mat& A, const Mat& B) {
  if (A.n != B.m) fail(MBF_ERR_INVALID, "matmul: shape mismatch");
  Mat C(A.m, B.n);
  for (int64_t j = 0; j < B.n; ++j) {
    double* c = reinterpret_cast<double*>(C.col(j));
    for (int64_t k = 0; k < A.n; ++k) {
      const cd b = B(k, j);
      if (b == cd(0)) continue;
      const double br = b.real(), bi = b.imag();
      const double* a = reinterpret_cast<const double*>(A.col(k));
      for (int64_t i = 0; i < A.m; ++i) {
        c[2 * i] += a[2 * i] * br - a[2 * i + 1] * bi;
        c[2 * i + 1] += a[2 * i] * bi + a[2 * i + 1] * br;
      }
    }
  }
  return C;
}

Mat matmul_hn(const Mat& A, const Mat& B) {
  if (A.m != B.m) fail(MBF_ERR_INVALID, "matmul_hn: shape mismatch");
  Mat C(A.n, B.n);
  for (int64_t j = 0; j < B.n; ++j)
    for (int64_t i = 0; i < A.n; ++i) C(i, j) = dot_hn(A.col(i), B.col(j), A.m);
  return C;
}

Mat adjoint(const Mat& A) {
  Mat B(A.n, A.m);
  for (int64_t j = 0; j < A.n; ++j)
    for (int64_t i = 0; i < A.m; ++i) B(j, i) = std::conj(A(i, j));
  return B;
}

Mat rows_of(const Mat& A, const std::vector<int64_t>& rows) {
  Mat B(int64_t(rows.size()), A.n);
  for (int64_t j = 0; j < A.n; ++j)
    for (size_t i = 0; i < rows.size(); ++i) B(int64_t(i), j) = A(rows[i], j);
  return B;
}

// Householder reflector H = I - tau v v^* with H x = beta e_1; v[0] = 1 convention is
// not used: v is returned unnormalised together with tau = 2 / (v^* v).
static void householder(const cd* x, int64_t n, std::vector<cd>& v, double& tau, cd& beta) {
  v.assign(x, x + n);
  const double alpha = std::sqrt(norm2(x, n));
  if (alpha == 0.0) { tau = 0; beta = 0; return; }
  const cd phase = std::abs(x[0]) > 0 ? x[0] / std::abs(x[0]) : cd(1.0);
  beta = -phase * alpha;
  v[0] -= beta;
  const double vv = norm2(v.data(), n);
  tau = vv > 0 ? 2.0 / vv : 0.0;
}

std::vector<int64_t> pivoted_qr(const Mat& A, int64_t kmax, double tol, Mat* Q) {
  const int64_t m = A.m, n = A.n;
  kmax = std::min({kmax, m, n});
  Mat W = A;
  std::vector<int64_t> piv(static_cast<size_t>(n));
  std::iota(piv.begin(), piv.end(), 0);
  // squared norms of the trailing parts of the columns, downdated after each step by
  // the entry the step removes; recomputed where cancellation has consumed all but a
  // sqrt(eps) fraction of the norm since it was last computed (the rule of LAPACK's
  // xGEQP3 / xLAQP2), cn_ref holding that last computed value
  std::vector<double> cn(static_cast<size_t>(n)), cn_ref(static_cast<size_t>(n));
  for (int64_t j = 0; j < n; ++j) cn_ref[size_t(j)] = cn[size_t(j)] = norm2(W.col(j), m);
  const double tol3z = std::sqrt(std::numeric_limits<double>::epsilon());
  std::vector<std::vector<cd>> vs;
  std::vector<double> taus;
  double first = -1;
  int64_t k = 0;
  std::vector<cd> v;
  for (; k < kmax; ++k) {
    int64_t p = k;
    for (int64_t j = k + 1; j < n; ++j)
      if (cn[size_t(j)] > cn[size_t(p)]) p = j;
    const double best = std::sqrt(cn[size_t(p)]);
    if (first < 0) first = best;
    if (best == 0.0 || best <= tol * first) break;
    if (p != k) {
      std::swap(piv[size_t(p)], piv[size_t(k)]);
      std::swap(cn[size_t(p)], cn[size_t(k)]);
      std::swap(cn_ref[size_t(p)], cn_ref[size_t(k)]);
      std::swap_ranges(W.col(k), W.col(k) + m, W.col(p));
    }
    double tau;
    cd beta;
    householder(W.col(k) + k, m - k, v, tau, beta);
    // apply H to the trailing columns
    for (int64_t j = k; j < n; ++j) reflect(v.data(), tau, W.col(j) + k, m - k);
    for (int64_t j = k + 1; j < n; ++j) {
      double& c = cn[size_t(j)];
      if (c == 0.0) continue;
      const double left = c - std::norm(W(k, j));
      if (left <= tol3z * cn_ref[size_t(j)]) {
        c = norm2(W.col(j) + k + 1, m - k - 1);
        cn_ref[size_t(j)] = c;
      } else {
        c = left;
      }
    }
    vs.push_back(v);
    taus.push_back(tau);
  }
  if (Q) {
    *Q = Mat(m, k);
    for (int64_t j = 0; j < k; ++j) (*Q)(j, j) = 1.0;
    for (int64_t q = k - 1; q >= 0; --q) {
      const auto& vq = vs[size_t(q)];
      const double tau = taus[size_t(q)];
      for (int64_t j = 0; j < k; ++j) reflect(vq.data(), tau, Q->col(j) + q, m - q);
    }
  }
  piv.resize(size_t(k));
  return piv;
}

// Symmetric tridiagonal eigenproblem by implicit single-shift QR sweeps with the
// Wilkinson shift (Golub & Van Loan, "Matrix Computations", §8.3).  T has diagonal d
// and off-diagonal e (e[k] couples k and k+1).  Each sweep chases the bulge created
// by the shifted first rotation down the unreduced block [lo, hi]; converged
// off-diagonals are zeroed from the bottom.  Rotations accumulate into the real
// column-major n x n matrix Z (T_original = Z T_final Z^T).
static void tridiag_qr(std::vector<double>& d, std::vector<double>& e, std::vector<double>& Z,
                       int64_t n) {
  const double eps = std::numeric_limits<double>::epsilon();
  auto small = [&](int64_t k) {
    return std::fabs(e[size_t(k)]) <= eps * (std::fabs(d[size_t(k)]) + std::fabs(d[size_t(k + 1)]));
  };
  int64_t hi = n - 1;
  int guard = 0;
  while (hi > 0 && guard < int(64 * n + 64)) {
    if (small(hi - 1)) { e[size_t(hi - 1)] = 0.0; --hi; continue; }
    int64_t lo = hi - 1;
    while (lo > 0 && !small(lo - 1)) --lo;
    ++guard;
    // Wilkinson shift from the trailing 2 x 2 block of [lo, hi]
    const double delta = 0.5 * (d[size_t(hi - 1)] - d[size_t(hi)]);
    const double off = e[size_t(hi - 1)];
    const double den = delta + (delta >= 0 ? 1.0 : -1.0) * std::hypot(delta, off);
    const double mu = d[size_t(hi)] - (den != 0.0 ? off * off / den : 0.0);
    double x = d[size_t(lo)] - mu, z = e[size_t(lo)];
    for (int64_t k = lo; k < hi; ++k) {
      const double rr = std::hypot(x, z);
      const double cs = rr > 0 ? x / rr : 1.0, sn = rr > 0 ? z / rr : 0.0;
      if (k > lo) e[size_t(k - 1)] = rr;
      const double a = d[size_t(k)], b = d[size_t(k + 1)], f = e[size_t(k)];
      d[size_t(k)] = cs * cs * a + 2.0 * cs * sn * f + sn * sn * b;
      d[size_t(k + 1)] = sn * sn * a - 2.0 * cs * sn * f + cs * cs * b;
      e[size_t(k)] = cs * sn * (b - a) + (cs * cs - sn * sn) * f;
      if (k + 1 < hi) {
        x = e[size_t(k)];
        z = sn * e[size_t(k + 1)];
        e[size_t(k + 1)] *= cs;
      }
      double* zk = Z.data() + n * k;
      double* zk1 = Z.data() + n * (k + 1);
      for (int64_t q = 0; q < n; ++q) {
        const double u = zk[q], w = zk1[q];
        zk[q] = cs * u + sn * w;
        zk1[q] = -sn * u + cs * w;
      }
    }
  }
}

void eig_herm(const Mat& A0, std::vector<double>& w, Mat& V) {
  const int64_t n = A0.n;
  Mat A = A0;
  Mat Q(n, n);
  for (int64_t i = 0; i < n; ++i) Q(i, i) = 1.0;
  std::vector<cd> v, p(static_cast<size_t>(n)), wv(static_cast<size_t>(n));
  std::vector<cd> sub(size_t(std::max<int64_t>(n - 1, 0)));
  // Householder tridiagonalisation A = Q T Q^*, T Hermitian tridiagonal.
  for (int64_t k = 0; k + 1 < n; ++k) {
    const int64_t m = n - k - 1;
    double tau;
    cd beta;
    householder(A.col(k) + k + 1, m, v, tau, beta);
    sub[size_t(k)] = (tau == 0.0) ? A(k + 1, k) : beta;
    if (tau == 0.0) continue;
    // p = tau * A22 v
    for (int64_t i = 0; i < m; ++i) p[size_t(i)] = 0;
    for (int64_t j = 0; j < m; ++j) {
      const cd vj = v[size_t(j)];
      const cd* a = A.col(k + 1 + j) + k + 1;
      for (int64_t i = 0; i < m; ++i) p[size_t(i)] += a[i] * vj;
    }
    for (int64_t i = 0; i < m; ++i) p[size_t(i)] *= tau;
    cd K = 0;
    for (int64_t i = 0; i < m; ++i) K += std::conj(v[size_t(i)]) * p[size_t(i)];
    K *= 0.5 * tau;
    for (int64_t i = 0; i < m; ++i) wv[size_t(i)] = p[size_t(i)] - K * v[size_t(i)];
    // A22 -= v w^* + w v^*
    for (int64_t j = 0; j < m; ++j) {
      cd* a = A.col(k + 1 + j) + k + 1;
      const cd cw = std::conj(wv[size_t(j)]), cv = std::conj(v[size_t(j)]);
      for (int64_t i = 0; i < m; ++i) a[i] -= v[size_t(i)] * cw + wv[size_t(i)] * cv;
    }
    // Q[:, k+1:] = Q[:, k+1:] H
    for (int64_t i = 0; i < n; ++i) {
      cd s = 0;
      for (int64_t j = 0; j < m; ++j) s += Q(i, k + 1 + j) * v[size_t(j)];
      s *= tau;
      for (int64_t j = 0; j < m; ++j) Q(i, k + 1 + j) -= s * std::conj(v[size_t(j)]);
    }
  }
  // Make the subdiagonal real and nonnegative with a diagonal unitary similarity.
  std::vector<double> d(static_cast<size_t>(n)), e(size_t(n), 0.0);
  std::vector<cd> phase(size_t(n), cd(1.0));
  for (int64_t k = 0; k < n; ++k) d[size_t(k)] = A(k, k).real();
  for (int64_t k = 0; k + 1 < n; ++k) {
    const double a = std::abs(sub[size_t(k)]);
    e[size_t(k)] = a;
    phase[size_t(k + 1)] = a > 0 ? phase[size_t(k)] * sub[size_t(k)] / a : phase[size_t(k)];
  }
  std::vector<double> Z(size_t(n * n), 0.0);
  for (int64_t i = 0; i < n; ++i) Z[size_t(i + n * i)] = 1.0;
  tridiag_qr(d, e, Z, n);
  std::vector<int64_t> order(static_cast<size_t>(n));
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return d[size_t(a)] > d[size_t(b)]; });
  w.resize(size_t(n));
  V = Mat(n, n);
  // eigenvectors of A: Q D Z
  for (int64_t jj = 0; jj < n; ++jj) {
    const int64_t j = order[size_t(jj)];
    w[size_t(jj)] = d[size_t(j)];
    const double* z = Z.data() + n * j;
    cd* out = V.col(jj);
    for (int64_t k = 0; k < n; ++k) {
      const cd dz = phase[size_t(k)] * z[k];
      if (dz == cd(0)) continue;
      const cd* q = Q.col(k);
      for (int64_t i = 0; i < n; ++i) out[i] += q[i] * dz;
    }
  }
}

// Columns (x, y) <- (c x - sn y', sn x + c y') with y' = y (pr + i pi): the complex
// Jacobi rotation of svd_small, in explicit real arithmetic.
static inline void rotate_pair(cd* xp, cd* yp, int64_t n, double c, double sn, double pr, double pi) {
  double* x = reinterpret_cast<double*>(xp);
  double* y = reinterpret_cast<double*>(yp);
  for (int64_t i = 0; i < n; ++i) {
    const double xr = x[2 * i], xi = x[2 * i + 1];
    const double yr = y[2 * i] * pr - y[2 * i + 1] * pi, yi = y[2 * i] * pi + y[2 * i + 1] * pr;
    x[2 * i] = c * xr - sn * yr;
    x[2 * i + 1] = c * xi - sn * yi;
    y[2 * i] = sn * xr + c * yr;
    y[2 * i + 1] = sn * xi + c * yi;
  }
}

void svd_small(const Mat& A, Mat& U, std::vector<double>& s, Mat& V) {
  const int64_t m = A.m, n = A.n;
  Mat W = A;
  V = Mat(n, n);
  for (int64_t i = 0; i < n; ++i) V(i, i) = 1.0;
  const double eps = 1e-15;
  for (int sweep = 0; sweep < 40; ++sweep) {
    bool rotated = false;
    for (int64_t p = 0; p + 1 < n; ++p) {
      for (int64_t q = p + 1; q < n; ++q) {
        cd* ap = W.col(p);
        cd* aq = W.col(q);
        // |a_p|^2, |a_q|^2 and a_p^* a_q in one pass (explicit arithmetic, vectorisable)
        const double* xa = reinterpret_cast<const double*>(ap);
        const double* xb = reinterpret_cast<const double*>(aq);
        double alpha = 0, beta = 0, gr = 0, gi = 0;
#pragma omp simd reduction(+ : alpha, beta, gr, gi)
        for (int64_t i = 0; i < m; ++i) {
          alpha += xa[2 * i] * xa[2 * i] + xa[2 * i + 1] * xa[2 * i + 1];
          beta += xb[2 * i] * xb[2 * i] + xb[2 * i + 1] * xb[2 * i + 1];
          gr += xa[2 * i] * xb[2 * i] + xa[2 * i + 1] * xb[2 * i + 1];
          gi += xa[2 * i] * xb[2 * i + 1] - xa[2 * i + 1] * xb[2 * i];
        }
        const cd gamma(gr, gi);
        const double g = std::abs(gamma);
        if (g == 0.0 || g <= eps * std::sqrt(alpha * beta)) continue;
        rotated = true;
        const cd ph = gamma / g;             // a_q e^{-i phi} makes a_p^* a_q real
        const double zeta = (beta - alpha) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        rotate_pair(ap, aq, m, c, sn, ph.real(), -ph.imag());
        rotate_pair(V.col(p), V.col(q), n, c, sn, ph.real(), -ph.imag());
      }
    }
    if (!rotated) break;
  }
  std::vector<double> sv(static_cast<size_t>(n));
  for (int64_t j = 0; j < n; ++j) sv[size_t(j)] = std::sqrt(norm2(W.col(j), m));
  std::vector<int64_t> order(static_cast<size_t>(n));
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return sv[size_t(a)] > sv[size_t(b)]; });
  const int64_t k = std::min(m, n);
  U = Mat(m, k);
  Mat V2(n, k);
  s.assign(size_t(k), 0.0);
  for (int64_t jj = 0; jj < k; ++jj) {
    const int64_t j = order[size_t(jj)];
    s[size_t(jj)] = sv[size_t(j)];
    std::copy(V.col(j), V.col(j) + n, V2.col(jj));
    if (sv[size_t(j)] > 0)
      for (int64_t i = 0; i < m; ++i) U(i, jj) = W(i, j) / sv[size_t(j)];
  }
  V = std::move(V2);
}

Mat pinv(const Mat& A, double rcond) {
  Mat U, V;
  std::vector<double> s;
  if (A.m >= A.n) {
    svd_small(A, U, s, V);
  } else {
    Mat At = adjoint(A);
    svd_small(At, V, s, U);  // A^* = V S U^*  =>  A = U S V^*
  }
  const double smax = s.empty() ? 0.0 : s[0];
  Mat P(A.n, A.m);
  for (size_t k = 0; k < s.size(); ++k) {
    if (!(s[k] > rcond * smax) || s[k] == 0.0) continue;
    const double inv = 1.0 / s[k];
    for (int64_t j = 0; j < A.m; ++j) {
      const cd uj = std::conj(U(j, int64_t(k))) * inv;
      for (int64_t i = 0; i < A.n; ++i) P(i, j) += V(i, int64_t(k)) * uj;
    }
  }
  return P;
}

}  // namespace mbf
