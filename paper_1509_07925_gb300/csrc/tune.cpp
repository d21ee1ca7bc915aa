// Autotuner for one operator (the paper has no counterpart): times the FP32 SIMT apply
// over RHS counts and the tensor-core panel over (panel buffers, A-ring depth) on the
// device, keeps the fastest configuration and the RHS count from which MBF_PREC_AUTO
// switches to the tensor cores.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "apply.hpp"
#include "op_internal.hpp"

namespace {

using mbf::fail;

void cuda_ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(MBF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};
struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Device time of one apply (median-free: best of `reps` after one warm-up).
double time_apply(mbf_op_s* op, const void* g, void* u, int64_t nrhs, int32_t prec, cudaStream_t st, Events& ev,
                  int reps) {
  mbf::apply_dev(op, g, u, nrhs, prec, st, false, 0);
  double best = 1e30;
  for (int r = 0; r < reps; ++r) {
    cuda_ok(cudaEventRecord(ev.a, st), "event");
    mbf::apply_dev(op, g, u, nrhs, prec, st, false, 0);
    cuda_ok(cudaEventRecord(ev.b, st), "event");
    cuda_ok(cudaEventSynchronize(ev.b), "event sync");
    float ms = 0.f;
    cuda_ok(cudaEventElapsedTime(&ms, ev.a, ev.b), "elapsed");
    best = std::min(best, double(ms));
  }
  return best;
}

}  // namespace

extern "C" mbf_status mbf_op_tune(mbf_op_t op, void* stream, mbf_tune_result_t* out) {
  return mbf::abi_guard([&] {
    if (!op || !out) fail(MBF_ERR_INVALID, "NULL argument");
    *out = mbf_tune_result_t{};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    constexpr int kMaxRhs = 64;
    DevBuf g, u;
    cuda_ok(cudaMalloc(&g.p, size_t(kMaxRhs) * size_t(op->n_in) * sizeof(float2)), "cudaMalloc");
    cuda_ok(cudaMalloc(&u.p, size_t(kMaxRhs) * size_t(op->n_out) * sizeof(float2)), "cudaMalloc");
    // inputs: every float = 0x3c3c3c3c (about 0.0115), a finite nonzero pattern
    cuda_ok(cudaMemsetAsync(g.p, 0x3c, size_t(kMaxRhs) * size_t(op->n_in) * sizeof(float2), st), "memset");
    Events ev;
    cuda_ok(cudaEventCreate(&ev.a), "event");
    cuda_ok(cudaEventCreate(&ev.b), "event");
    const int rhs_list[] = {1, 2, 4, 8, 16, 32, 64};
    for (int R : rhs_list) {
      if (!op->simt_unavailable.empty()) break;   // tensor-only operator
      out->simt_rhs[out->n_simt] = R;
      out->simt_ms[out->n_simt] = time_apply(op, g.p, u.p, R, MBF_PREC_FP32_SIMT, st, ev, 3);
      ++out->n_simt;
    }
    out->tc_min_rhs = 1 << 30;
    if (op->tc_unavailable.empty()) {
      int optin = 0;
      cuda_ok(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, op->device), "attr");
      const int keep_nsa = op->tc_nsa, keep_nxb = op->tc_nxb;
      const size_t keep_smem = op->tc_smem;
      double best = 1e30;
      int best_nsa = keep_nsa, best_nxb = keep_nxb;
      size_t best_smem = keep_smem;
      // panel buffers 2 and 3; for each, the deepest ring depths that fit first (at most
      // 8 configurations in all: 5 with two buffers, 3 with three)
      for (int nxb = 2; nxb <= 3; ++nxb) {
        int deepest = 0;
        for (int nsa = 2; nsa <= 16; nsa += 2)
          if (mbf::tc_smem_bytes(nsa, nxb, op->tc_nsets, op->tc_mt_max, op->tc_kpad_max) <= size_t(optin)) deepest = nsa;
        const int quota = nxb == 2 ? 5 : 3;
        for (int nsa = std::max(2, deepest - 2 * (quota - 1)); nsa <= deepest && out->n_slots < 8; nsa += 2) {
          op->tc_nsa = nsa;
          op->tc_nxb = nxb;
          op->tc_smem = std::max(mbf::tc_smem_bytes(nsa, nxb, op->tc_nsets, op->tc_mt_max, op->tc_kpad_max),
                                 size_t(optin) / 2 + 1024);
          double ms = 0.0;
          try {
            ms = time_apply(op, g.p, u.p, kMaxRhs, MBF_PREC_BF16X3, st, ev, 3);
          } catch (...) {
            op->tc_nsa = keep_nsa;
            op->tc_nxb = keep_nxb;
            op->tc_smem = keep_smem;
            throw;
          }
          out->slots[out->n_slots] = nsa;
          out->panel_buffers[out->n_slots] = nxb;
          out->tc_ms[out->n_slots] = ms;
          ++out->n_slots;
          if (ms < best) {
            best = ms;
            best_nsa = nsa;
            best_nxb = nxb;
            best_smem = op->tc_smem;
          }
        }
      }
      op->tc_nxb = best_nxb;
      out->tc_buffers_chosen = best_nxb;
      op->tc_nsa = best_nsa;
      op->tc_smem = best_smem;
      out->tc_slots_chosen = best_nsa;
      // one 64-RHS panel costs `best` for any RHS count up to 64
      for (int i = 0; i < out->n_simt; ++i)
        if (out->simt_ms[i] > best) {
          out->tc_min_rhs = out->simt_rhs[i];
          break;
        }
      if (out->tc_min_rhs > kMaxRhs) out->tc_min_rhs = kMaxRhs + 1;
      if (!op->simt_unavailable.empty()) out->tc_min_rhs = 1;
      op->tc_min_rhs = out->tc_min_rhs;
    }
    cuda_ok(cudaStreamSynchronize(st), "sync");
    int dev_status = 0;
    cuda_ok(cudaMemcpy(&dev_status, op->ws.status, sizeof(int), cudaMemcpyDeviceToHost), "status");
    if (dev_status != 0) {
      cudaMemset(op->ws.status, 0, sizeof(int));
      fail(MBF_ERR_TIMEOUT, "a device wait gave up while tuning");
    }
  });
}
