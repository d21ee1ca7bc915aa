// Host/device interface of the apply kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "layout.hpp"

namespace mbf {

struct ApplyArgs {
  const uint8_t* arena;
  const Item* items;
  const int32_t* x_perm;
  const int32_t* x_off;
  const int32_t* w_perm;
  const int32_t* w_off;
  const float2* in;        // forward: g [nrhs][n_in]; adjoint: u [nrhs][n_out]
  float2* out;             // forward: u; adjoint: g
  int64_t in_len, out_len;
  float2* bufs;            // stage e writes bufs + e * buf_stride ([pos][NRB]); stage e+1 reads it
  int64_t buf_stride;
  unsigned int* counters;  // [stage][group]: input segments written so far (zeroed per launch)
  unsigned int* barrier;   // grid barrier between passes (zeroed per launch)
  int* status;             // 0 = ok; nonzero = a device wait ran out of time (sticky)
  int32_t nrhs, n_pass, n_slots, pad_;
  Plan plan;
};

enum DeviceStatus : int {
  ST_OK = 0,
  ST_BARRIER_TIMEOUT = 1,
  ST_FULL_TIMEOUT = 2,
  ST_EMPTY_TIMEOUT = 3,
  ST_BAD_ITEM = 4,
  ST_DEP_TIMEOUT = 5
};

size_t simt_smem_bytes(int nrb, int ns);
int simt_threads(int nrb);
cudaError_t simt_config(int nrb, int* grid, int* ns, size_t* smem);
cudaError_t launch_apply_simt(const ApplyArgs& a, int nrb, bool adj, int grid, size_t smem,
                              cudaStream_t stream);
// Bytes of dependency counters for a plan (S stages x groups, rounded up to 256).
size_t counter_bytes(const Plan& plan);

}  // namespace mbf
