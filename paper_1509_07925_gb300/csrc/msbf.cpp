// Multiscale butterfly factorization (§4): the corona split of Omega (eq.
// domaindecomp), one butterfly factorization per corona on a square Omega tree (§4.2
// step 2), and the dense centre; the apply is the sum of eq. (f1):
//     u = K_C (R_C g) + sum_t BF_t (R_t g).
// Each BF_t is an ordinary resident operator whose Omega tree holds only the points of
// Omega_t, so its leaf gathers are R_t; its result is added into u (accumulating
// apply).  K_C is evaluated once through the entry callback and kept in HBM.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "mbf_internal.hpp"
#include "msbf.hpp"
#include "op_internal.hpp"

struct mbf_msbf_s {
  int device = 0;
  std::vector<mbf_op_s*> parts;
  std::vector<int32_t> part_t, part_L;
  bool own = false;
  float2* d_Kc = nullptr;     // [n_c][n_out] complex64
  int32_t* d_idx = nullptr;   // centre points (natural Omega indices)
  int64_t n_c = 0, n_out = 0, n_in = 0;
};

namespace {

using mbf::fail;

void cuda_ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(MBF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void msbf_free(mbf_msbf_s* m) {
  if (!m) return;
  if (m->own)
    for (mbf_op_s* p : m->parts) mbf_op_destroy(p);
  cudaFree(m->d_Kc);
  cudaFree(m->d_idx);
  delete m;
}

// Upload the centre: Kc host complex128 [n_c][n_out] (c-major), idx [n_c].
void upload_centre(mbf_msbf_s* m, const double* Kc, const int64_t* idx, int64_t n_c) {
  m->n_c = n_c;
  if (n_c == 0) return;
  std::vector<float2> k(size_t(n_c * m->n_out));
  for (size_t q = 0; q < k.size(); ++q) k[q] = make_float2(float(Kc[2 * q]), float(Kc[2 * q + 1]));
  std::vector<int32_t> ix(static_cast<size_t>(n_c));
  for (int64_t c = 0; c < n_c; ++c) {
    if (idx[c] < 0 || idx[c] >= m->n_in) fail(MBF_ERR_INVALID, "centre index out of range");
    ix[size_t(c)] = int32_t(idx[c]);
  }
  cuda_ok(cudaMalloc(&m->d_Kc, k.size() * sizeof(float2)), "cudaMalloc centre kernel");
  cuda_ok(cudaMemcpy(m->d_Kc, k.data(), k.size() * sizeof(float2), cudaMemcpyHostToDevice), "upload centre kernel");
  cuda_ok(cudaMalloc(&m->d_idx, ix.size() * sizeof(int32_t)), "cudaMalloc centre index");
  cuda_ok(cudaMemcpy(m->d_idx, ix.data(), ix.size() * sizeof(int32_t), cudaMemcpyHostToDevice), "upload centre index");
}

// Corona index of each Omega point (eq. domaindecomp): n/2^(t+2) < max_k |xi_k| <= n/2^(t+1),
// for the t with n/2^(t+2) >= n_center/2; -1 for the centre.
std::vector<int> corona_of(int n, int n_center, int& T) {
  const int64_t N = int64_t(n) * n;
  std::vector<int> t_of(size_t(N), -1);
  T = 0;
  for (int t = 0;; ++t) {
    const double lo = double(n) / std::ldexp(1.0, t + 2), hi = double(n) / std::ldexp(1.0, t + 1);
    if (lo < 0.5 * n_center || lo < 0.5) break;
    T = t + 1;
    for (int64_t p = 0; p < N; ++p) {
      const double x1 = double(p / n) - n / 2, x2 = double(p % n) - n / 2;
      const double mx = std::max(std::fabs(x1), std::fabs(x2));
      if (mx > lo && mx <= hi) t_of[size_t(p)] = t;
    }
  }
  return t_of;
}

}  // namespace

extern "C" {

mbf_status mbf_msbf_create(const mbf_op_t* parts, int32_t n_parts, const double* center_kernel,
                           const int64_t* center_index, int64_t n_center_points, int32_t take_ownership,
                           mbf_msbf_t* out) {
  return mbf::abi_guard([&] {
    if (!out || (n_parts > 0 && !parts) || n_parts < 0) fail(MBF_ERR_INVALID, "bad parts");
    if (n_center_points < 0 || (n_center_points > 0 && (!center_kernel || !center_index)))
      fail(MBF_ERR_INVALID, "bad centre");
    if (n_parts == 0 && n_center_points == 0) fail(MBF_ERR_INVALID, "empty multiscale operator");
    auto* m = new mbf_msbf_s();
    try {
      cuda_ok(cudaGetDevice(&m->device), "cudaGetDevice");
      for (int32_t i = 0; i < n_parts; ++i) {
        if (!parts[i]) fail(MBF_ERR_INVALID, "NULL part");
        if (i == 0) {
          m->n_out = parts[i]->n_out;
          m->n_in = parts[i]->n_in;
        } else if (parts[i]->n_out != m->n_out || parts[i]->n_in != m->n_in) {
          fail(MBF_ERR_INVALID, "parts act on different point sets");
        }
        m->parts.push_back(parts[i]);
        m->part_t.push_back(i);
        m->part_L.push_back(parts[i]->L);
      }
      if (n_parts == 0) fail(MBF_ERR_INVALID, "a centre alone needs mbf_build_msbf (point counts unknown)");
      upload_centre(m, center_kernel, center_index, n_center_points);
      m->own = take_ownership != 0;
    } catch (...) {
      m->own = false;
      msbf_free(m);
      throw;
    }
    *out = m;
  });
}

mbf_status mbf_build_msbf(const mbf_problem_t* prob, mbf_entry_fn fn, void* ctx, const mbf_build_opts_t* opts,
                          int32_t n_center, mbf_msbf_t* out) {
  return mbf::abi_guard([&] {
    if (!prob || !fn || !out) fail(MBF_ERR_INVALID, "NULL argument");
    if (prob->dim != 2) fail(MBF_ERR_INVALID, "the multiscale split is two-dimensional (§4)");
    const int n = prob->n;
    if (n < 4 || (n & (n - 1))) fail(MBF_ERR_INVALID, "n must be a power of two >= 4");
    if (n_center < 1) fail(MBF_ERR_INVALID, "n_center must be >= 1");
    const int L = int(std::lround(std::log2(double(n))));
    int T = 0;
    const std::vector<int> t_of = corona_of(n, n_center, T);
    const int64_t N = int64_t(n) * n;
    mbf_build_opts_t o{};
    if (opts) o = *opts;
    auto* m = new mbf_msbf_s();
    m->own = true;
    try {
      cuda_ok(cudaGetDevice(&m->device), "cudaGetDevice");
      m->n_out = m->n_in = N;
      std::vector<int64_t> centre;
      for (int64_t p = 0; p < N; ++p)
        if (t_of[size_t(p)] < 0) centre.push_back(p);
      for (int t = 0; t < T; ++t) {
        const int Lt = 2 * ((L - t) / 2);
        if (Lt < 2) fail(MBF_ERR_INVALID, "corona too deep for a tree of depth >= 2");
        std::vector<int64_t> idx;
        for (int64_t p = 0; p < N; ++p)
          if (t_of[size_t(p)] == t) idx.push_back(p);
        mbf_problem_t pt = *prob;
        pt.L = Lt;
        pt.tree = MBF_TREE_SQUARE;
        pt.n_w = int64_t(idx.size());
        pt.w_index = idx.data();
        pt.w_lo = -double(n) / std::ldexp(1.0, t + 1);
        pt.w_side = double(n) / std::ldexp(1.0, t);
        mbf_build_opts_t ot = o;
        ot.seed = o.seed + 101 * uint64_t(t + 1);
        const std::string part_file = o.factor_file && *o.factor_file ? std::string(o.factor_file) + ".t" +
                                                                            std::to_string(t)
                                                                      : std::string();
        ot.factor_file = part_file.empty() ? nullptr : part_file.c_str();
        mbf::FactorSet fs = mbf::build_or_load(pt, fn, ctx, ot);
        mbf_factors_t v = fs.view();
        mbf_op_t op = nullptr;
        const mbf_status s = mbf_op_create(&v, &op);
        if (s != MBF_OK) fail(s, mbf_last_error());
        m->parts.push_back(op);
        m->part_t.push_back(t);
        m->part_L.push_back(Lt);
      }
      // K_C through the entry callback: x = natural grid / n, xi = centre frequencies
      const int64_t nc = int64_t(centre.size());
      std::vector<double> Kc(size_t(2 * nc * N));
      if (nc > 0) {
        std::vector<double> xs(size_t(2 * N)), xi(size_t(2 * nc));
        for (int64_t p = 0; p < N; ++p) {
          xs[size_t(2 * p)] = double(p / n) / n;
          xs[size_t(2 * p + 1)] = double(p % n) / n;
        }
        for (int64_t c = 0; c < nc; ++c) {
          xi[size_t(2 * c)] = double(centre[size_t(c)] / n) - n / 2;
          xi[size_t(2 * c + 1)] = double(centre[size_t(c)] % n) - n / 2;
        }
        // block (all x) x (one centre point) is column-major m x 1 = the row c of Kc
        for (int64_t c = 0; c < nc; ++c) fn(xs.data(), N, xi.data() + 2 * c, 1, 2, Kc.data() + 2 * c * N, ctx);
      }
      upload_centre(m, Kc.data(), centre.data(), nc);
    } catch (...) {
      msbf_free(m);
      throw;
    }
    *out = m;
  });
}

mbf_status mbf_msbf_apply(mbf_msbf_t m, const void* g, void* u, int64_t nrhs, int32_t precision, void* stream) {
  return mbf::abi_guard([&] {
    if (!m || !g || !u) fail(MBF_ERR_INVALID, "NULL argument");
    if (nrhs < 0 || nrhs > (int64_t(1) << 24)) fail(MBF_ERR_INVALID, "nrhs out of range");
    if (nrhs == 0) return;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // centre first (it initialises u), then every corona's BF adds into u
    cuda_ok(mbf::launch_center_fwd(m->d_Kc, m->d_idx, int(m->n_c), static_cast<const float2*>(g), m->n_in,
                                   static_cast<float2*>(u), m->n_out, int(nrhs), false, st),
            "centre launch");
    for (mbf_op_s* p : m->parts) mbf::apply_dev(p, g, u, nrhs, precision, st, false, 0, true);
  });
}

mbf_status mbf_msbf_apply_adjoint(mbf_msbf_t m, const void* u, void* g, int64_t nrhs, int32_t precision,
                                  void* stream) {
  return mbf::abi_guard([&] {
    if (!m || !g || !u) fail(MBF_ERR_INVALID, "NULL argument");
    if (nrhs < 0 || nrhs > (int64_t(1) << 24)) fail(MBF_ERR_INVALID, "nrhs out of range");
    if (nrhs == 0) return;
    if (precision == MBF_PREC_TF32) fail(MBF_ERR_INVALID, "TF32 operands apply the forward operator only");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the parts and the centre write disjoint entries of g (they partition Omega)
    cuda_ok(cudaMemsetAsync(g, 0, size_t(nrhs) * size_t(m->n_in) * sizeof(float2), st), "cudaMemsetAsync");
    cuda_ok(mbf::launch_center_adj(m->d_Kc, m->d_idx, int(m->n_c), static_cast<const float2*>(u), m->n_out,
                                   static_cast<float2*>(g), m->n_in, int(nrhs), st),
            "centre launch");
    for (mbf_op_s* p : m->parts) mbf::apply_dev(p, u, g, nrhs, precision, st, true, 0, true);
  });
}

mbf_status mbf_msbf_info(mbf_msbf_t m, mbf_msbf_info_t* info) {
  return mbf::abi_guard([&] {
    if (!m || !info) fail(MBF_ERR_INVALID, "NULL argument");
    *info = mbf_msbf_info_t{};
    info->n_parts = int32_t(m->parts.size());
    info->n_out = m->n_out;
    info->n_in = m->n_in;
    info->n_center_points = m->n_c;
    int64_t nnz = m->n_c * m->n_out;
    for (size_t i = 0; i < m->parts.size() && i < 16; ++i) {
      info->part_t[i] = m->part_t[i];
      info->part_L[i] = m->part_L[i];
      info->part_points[i] = m->parts[i]->n_w;
      info->part_nnz[i] = m->parts[i]->nnz;
      nnz += m->parts[i]->nnz;
    }
    info->nnz_algorithmic = nnz;
    info->bytes_algorithmic = 8 * nnz;
  });
}

mbf_status mbf_msbf_part(mbf_msbf_t m, int32_t i, mbf_op_t* op) {
  return mbf::abi_guard([&] {
    if (!m || !op || i < 0 || i >= int32_t(m->parts.size())) fail(MBF_ERR_INVALID, "bad part index");
    *op = m->parts[size_t(i)];
  });
}

mbf_status mbf_msbf_destroy(mbf_msbf_t m) {
  return mbf::abi_guard([&] { msbf_free(m); });
}

}  // extern "C"
