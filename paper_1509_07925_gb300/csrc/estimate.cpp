// Error estimator of the numerical sections (§3.3 and §4.3): the relative L2 error of
// the factored operator against the direct sum u(x) = sum_xi K(x, xi) g(xi) (§1.1,
// eq. kernel) on a random set S of output points,
//     e = sqrt( sum_{x in S} |u_f(x) - u(x)|^2 / sum_{x in S} |u(x)|^2 ).
// u_f comes from one FP32 apply of the resident operator on the device; u(x) from FP64
// entry evaluations on the host through the same entry function the builder takes.
// The input g has iid complex standard normal entries on the Omega points the operator
// covers (zero elsewhere), drawn from a seeded counter-based generator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "mbf_internal.hpp"
#include "op_internal.hpp"

namespace mbf {
namespace {

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// 2014): one 64-bit output per counter value.
uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
double unit_open(uint64_t bits) { return (double(bits >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

// Complex standard normal (a + i b)/sqrt(2) by the Box-Muller transform of two uniforms.
void complex_normal(uint64_t seed, uint64_t k, double* re, double* im) {
  const double u1 = unit_open(splitmix64(seed ^ (2 * k))), u2 = unit_open(splitmix64(seed ^ (2 * k + 1)));
  const double rad = std::sqrt(-2.0 * std::log(u1)) / std::sqrt(2.0);
  *re = rad * std::cos(6.283185307179586 * u2);
  *im = rad * std::sin(6.283185307179586 * u2);
}

void check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(MBF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int grid_side(int64_t N, int d) {
  const int n = int(std::llround(std::pow(double(N), 1.0 / d)));
  if (Tree::ipow(n, d) != N) fail(MBF_ERR_INVALID, "estimate: point count is not n^d");
  return n;
}

}  // namespace

double estimate_error(mbf_op_s* op, mbf_entry_fn fn, void* ctx, int32_t n_samples, uint64_t seed,
                      cudaStream_t st) {
  if (!fn) fail(MBF_ERR_INVALID, "estimate: NULL entry function");
  if (n_samples <= 0) fail(MBF_ERR_INVALID, "estimate: n_samples must be positive");
  const int d = op->d;
  const int nx = grid_side(op->n_out, d), nw = grid_side(op->n_in, d);
  // the Omega points the operator covers
  std::vector<int32_t> wp(size_t(op->n_w));
  check(cudaMemcpy(wp.data(), op->d_w_perm, wp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost), "read w_perm");
  std::vector<float> g(size_t(2 * op->n_in), 0.0f);
  for (size_t k = 0; k < wp.size(); ++k) {
    double re, im;
    complex_normal(seed, uint64_t(wp[k]), &re, &im);
    g[2 * size_t(wp[k])] = float(re);
    g[2 * size_t(wp[k]) + 1] = float(im);
  }
  // one FP32 apply on the device
  void *dg = nullptr, *du = nullptr;
  if (cudaMalloc(&dg, g.size() * sizeof(float)) != cudaSuccess) fail(MBF_ERR_OOM, "estimate: cudaMalloc");
  if (cudaMalloc(&du, size_t(op->n_out) * 2 * sizeof(float)) != cudaSuccess) {
    cudaFree(dg);
    fail(MBF_ERR_OOM, "estimate: cudaMalloc");
  }
  std::vector<float> u(size_t(2 * op->n_out));
  try {
    check(cudaMemcpyAsync(dg, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice, st), "estimate H2D");
    const int32_t prec = op->simt_unavailable.empty() ? MBF_PREC_FP32_SIMT : MBF_PREC_AUTO;
    apply_dev(op, dg, du, 1, prec, st, false, 0);
    check(cudaMemcpyAsync(u.data(), du, u.size() * sizeof(float), cudaMemcpyDeviceToHost, st), "estimate D2H");
    check(cudaStreamSynchronize(st), "estimate sync");
  } catch (...) {
    cudaFree(dg);
    cudaFree(du);
    throw;
  }
  cudaFree(dg);
  cudaFree(du);
  int status = 0;
  check(cudaMemcpy(&status, op->ws.status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  if (status != 0) fail(MBF_ERR_TIMEOUT, "estimate: a device wait of the apply gave up");

  // S: n_samples distinct outputs (partial Fisher-Yates on a counter-based stream)
  const int64_t m = std::min<int64_t>(n_samples, op->n_out);
  std::vector<int64_t> idx(size_t(op->n_out));
  for (int64_t i = 0; i < op->n_out; ++i) idx[size_t(i)] = i;
  for (int64_t i = 0; i < m; ++i) {
    const uint64_t r = splitmix64(seed ^ 0x5a5a5a5a5a5a5a5aull ^ uint64_t(i) * 0x100000001b3ull);
    const int64_t j = i + int64_t(r % uint64_t(op->n_out - i));
    std::swap(idx[size_t(i)], idx[size_t(j)]);
  }
  // Omega points as coordinates, and the applied g (the FP32 values) in FP64
  std::vector<double> xi(size_t(wp.size()) * d), gv(2 * wp.size());
  for (size_t k = 0; k < wp.size(); ++k) {
    int64_t q = wp[k];
    for (int a = d - 1; a >= 0; --a) {
      xi[k * d + size_t(a)] = double(q % nw) - nw / 2;
      q /= nw;
    }
    gv[2 * k] = g[2 * size_t(wp[k])];
    gv[2 * k + 1] = g[2 * size_t(wp[k]) + 1];
  }
  std::vector<double> num(size_t(m), 0.0), den(size_t(m), 0.0);
  const unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), unsigned(m)));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) {
    th.emplace_back([&, t] {
      const int64_t chunk = 4096;
      std::vector<double> ent(size_t(2 * chunk));
      for (int64_t s = t; s < m; s += nt) {
        const int64_t xr = idx[size_t(s)];
        double x[3];
        int64_t q = xr;
        for (int a = d - 1; a >= 0; --a) {
          x[a] = double(q % nx) / nx;
          q /= nx;
        }
        double sr = 0, si = 0;
        for (int64_t b0 = 0; b0 < int64_t(wp.size()); b0 += chunk) {
          const int64_t nb = std::min<int64_t>(chunk, int64_t(wp.size()) - b0);
          fn(x, 1, xi.data() + size_t(b0) * d, nb, d, ent.data(), ctx);
          for (int64_t b = 0; b < nb; ++b) {
            const double kr = ent[2 * size_t(b)], ki = ent[2 * size_t(b) + 1];
            const double gr = gv[2 * size_t(b0 + b)], gi = gv[2 * size_t(b0 + b) + 1];
            sr += kr * gr - ki * gi;
            si += kr * gi + ki * gr;
          }
        }
        const double er = double(u[2 * size_t(xr)]) - sr, ei = double(u[2 * size_t(xr) + 1]) - si;
        num[size_t(s)] = er * er + ei * ei;
        den[size_t(s)] = sr * sr + si * si;
      }
    });
  }
  for (auto& x : th) x.join();
  double sn = 0, sd = 0;
  for (int64_t s = 0; s < m; ++s) {
    sn += num[size_t(s)];
    sd += den[size_t(s)];
  }
  const double eps = sd > 0 ? std::sqrt(sn / sd) : 0.0;
  op->eps = eps;
  op->eps_samples = int32_t(m);
  return eps;
}

}  // namespace mbf
