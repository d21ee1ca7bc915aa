// Built-in kernel evaluators K(x, xi) for the builder (Case (ii) of §1.1: entries
// in O(1) work).  Phases are reduced modulo 1 before multiplying by 2 pi so that
// large |xi| keep full relative accuracy.
#include <cmath>

#include "mbf.h"

namespace {
constexpr double kTwoPi = 6.283185307179586476925286766559;

inline void expi(double phase, double* out) {
  const double f = phase - std::floor(phase);
  out[0] = std::cos(kTwoPi * f);
  out[1] = std::sin(kTwoPi * f);
}
}  // namespace

extern "C" {

// exp(-2 pi i x.xi): the d-dimensional DFT kernel (§1.1).
void mbf_kernel_dft(const double* x, int64_t m, const double* xi, int64_t n, int32_t dim,
                    double* out, void*) {
  for (int64_t b = 0; b < n; ++b) {
    for (int64_t a = 0; a < m; ++a) {
      double ph = 0;
      for (int k = 0; k < dim; ++k) ph += x[a * dim + k] * xi[b * dim + k];
      expi(-ph, out + 2 * (a + m * b));
    }
  }
}

// exp(2 pi i (x.xi + c(x)|xi|)), c(x) = (2 + sin 2 pi x_1 sin 2 pi x_2)/16: the isotropic
// case c_1 = c_2 of the Example-1 phase (§3.3).
void mbf_kernel_fio_iso(const double* x, int64_t m, const double* xi, int64_t n, int32_t dim,
                        double* out, void*) {
  (void)dim;
  double cx[512];
  const int64_t chunk = 512;
  for (int64_t a0 = 0; a0 < m; a0 += chunk) {
    const int64_t a1 = a0 + chunk < m ? a0 + chunk : m;
    for (int64_t a = a0; a < a1; ++a)
      cx[a - a0] = (2.0 + std::sin(kTwoPi * x[2 * a]) * std::sin(kTwoPi * x[2 * a + 1])) / 16.0;
    for (int64_t b = 0; b < n; ++b) {
      const double x1 = xi[2 * b], x2 = xi[2 * b + 1];
      const double r = std::sqrt(x1 * x1 + x2 * x2);
      for (int64_t a = a0; a < a1; ++a) {
        const double ph = x[2 * a] * x1 + x[2 * a + 1] * x2 + cx[a - a0] * r;
        expi(ph, out + 2 * (a + m * b));
      }
    }
  }
}

// Example 1 (§3.3, eq. example1phi): exp(2 pi i (x.xi + sqrt(c_1^2 xi_1^2 + c_2^2 xi_2^2))),
// c_1 = (2 + sin 2pi x_1 sin 2pi x_2)/16, c_2 = (2 + cos 2pi x_1 cos 2pi x_2)/16.
void mbf_kernel_fio_ellip(const double* x, int64_t m, const double* xi, int64_t n, int32_t dim,
                          double* out, void*) {
  (void)dim;
  for (int64_t a = 0; a < m; ++a) {
    const double s1 = std::sin(kTwoPi * x[2 * a]), s2 = std::sin(kTwoPi * x[2 * a + 1]);
    const double k1 = std::cos(kTwoPi * x[2 * a]), k2 = std::cos(kTwoPi * x[2 * a + 1]);
    const double c1 = (2.0 + s1 * s2) / 16.0, c2 = (2.0 + k1 * k2) / 16.0;
    for (int64_t b = 0; b < n; ++b) {
      const double x1 = xi[2 * b], x2 = xi[2 * b + 1];
      const double ph = x[2 * a] * x1 + x[2 * a + 1] * x2 +
                        std::sqrt(c1 * c1 * x1 * x1 + c2 * c2 * x2 * x2);
      expi(ph, out + 2 * (a + m * b));
    }
  }
}

}  // extern "C"
