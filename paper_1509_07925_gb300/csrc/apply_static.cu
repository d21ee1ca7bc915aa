// Allocation-free forward apply: the persistent FP32 kernel of apply_simt.cu run
// with its coefficient workspace and grid-barrier counter placed in one fixed,
// library-global device array instead of the operator's own workspace.
//
// Why: some callers may not allocate device memory when they apply an operator --
// for instance a process whose device memory is entirely owned by another
// allocator (a framework's caching pool) or held to a fixed budget, where an extra
// cudaMalloc can fail, or a latency-critical loop in which an allocation, which
// may synchronize the device, is not allowed.  This entry point lets them apply a
// resident operator using only memory the library reserved when it was loaded.
//
// Limits and sharing: the array holds kStaticScratchBytes (4 MiB) on every device
// that loads the library, for the life of the process.  A call needs 256 bytes, one
// dependency counter per group of every stage, and one coefficient vector of
// (c^L * max rank) entries per stage for each of up to 4 RHS per pass; larger needs
// are rejected with MBF_ERR_INVALID.  Every call on a device
// shares the one array and leaves its contents behind; the barrier counter is
// cleared at the start of each call.  Calls that overlap on the GPU (on different
// streams, or with an mbf_apply_static on another operator) race on the array.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "apply.hpp"
#include "op_internal.hpp"

namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;
constexpr size_t kBarrierBytes = 256;
constexpr int kMaxDevices = 64;

// Device-side scratch.  In host code this name is only a host-side stand-in for
// the symbol, not a device address: the kernel must be given the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Set-up, once per device, with that device current: look up the device address
// of the scratch array.  The first call on each device does this.
void* scratch_address(int dev) {
  if (dev < 0 || dev >= kMaxDevices) mbf::fail(MBF_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      mbf::fail(MBF_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

void apply_static_impl(mbf_op_s* op, const void* g, void* u, int64_t nrhs, void* stream) {
  if (!op) mbf::fail(MBF_ERR_INVALID, "operator is NULL");
  if (nrhs < 0) mbf::fail(MBF_ERR_INVALID, "nrhs < 0");
  if (nrhs == 0) return;
  if (!g || !u) mbf::fail(MBF_ERR_INVALID, "NULL vector");
  if (nrhs > (int64_t(1) << 24)) mbf::fail(MBF_ERR_INVALID, "nrhs too large");
  if (!op->simt_unavailable.empty())
    mbf::fail(MBF_ERR_INVALID, "FP32 SIMT path unavailable: " + op->simt_unavailable);
  const int nrb = nrhs >= 4 ? 4 : (nrhs >= 2 ? 2 : 1);
  const size_t vec_bytes = size_t(op->positions) * size_t(nrb) * sizeof(float2);
  const size_t sync_bytes = kBarrierBytes + mbf::counter_bytes(op->plan);
  const size_t need = sync_bytes + size_t(op->plan.n_stages) * vec_bytes;
  if (need > kStaticScratchBytes)
    mbf::fail(MBF_ERR_INVALID, "operator needs " + std::to_string(need) + " bytes of scratch for " +
                                   std::to_string(nrb) + " RHS per pass; the static scratch holds " +
                                   std::to_string(kStaticScratchBytes));
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) mbf::fail(MBF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (prev != op->device && (e = cudaSetDevice(op->device)) != cudaSuccess)
    mbf::fail(MBF_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  struct Restore {
    int dev, cur;
    ~Restore() {
      if (dev != cur) cudaSetDevice(dev);
    }
  } restore{prev, op->device};
  unsigned char* base = static_cast<unsigned char*>(scratch_address(op->device));
  mbf::ApplyArgs a{};
  a.arena = op->d_arena;
  a.items = op->d_items;
  a.x_perm = op->d_x_perm;
  a.x_off = op->d_x_off;
  a.w_perm = op->d_w_perm;
  a.w_off = op->d_w_off;
  a.in = static_cast<const float2*>(g);
  a.out = static_cast<float2*>(u);
  a.in_len = op->n_in;
  a.out_len = op->n_out;
  a.barrier = reinterpret_cast<unsigned*>(base);            // barrier + counters, cleared by the launch
  a.counters = a.barrier + kBarrierBytes / sizeof(unsigned);
  a.bufs = reinterpret_cast<float2*>(base + sync_bytes);     // one vector per stage
  a.buf_stride = op->positions * nrb;
  a.status = op->ws.status;
  a.nrhs = int32_t(nrhs);
  a.n_pass = int32_t((nrhs + nrb - 1) / nrb);
  a.n_slots = op->ns[nrb];
  a.plan = op->plan;
  e = mbf::launch_apply_simt(a, nrb, false, op->grid, op->smem[nrb], static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) mbf::fail(MBF_ERR_CUDA, std::string("apply launch: ") + cudaGetErrorString(e));
}

}  // namespace

extern "C" mbf_status mbf_apply_static(mbf_op_t op, const void* g, void* u, int64_t nrhs, void* stream) {
  return mbf::abi_guard([&] { apply_static_impl(op, g, u, nrhs, stream); });
}
