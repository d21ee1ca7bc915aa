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

constexpr int kTcMaxNR = 64;   // RHS per tensor-core panel

struct TCArgs {
  const uint8_t* arena;
  const float2* x_in;      // input of main stage 0: [pos][NR]
  float2* bufs;            // output of main stage e: bufs + e * buf_stride, [pos][NR]
  int64_t buf_stride;
  unsigned* counters;      // [stage][group], zeroed per launch
  int* status;
  int32_t NR, nsa;         // RHS per panel (32 or 64); A ring slots
  int32_t mpad, kpad_max;  // rows of an A slot plane (128 or 256); largest K_pad
  TCPlan plan;
};

struct LeafArgs {
  const uint8_t* arena;    // packed arena of the SIMT path (leaf items)
  const Item* items;
  int64_t item_base;       // item of group 0; group g's item is item_base + g * item_stride
  const int32_t* perm;
  const int32_t* off;
  const float2* vec;       // forward: g [nrhs][len_vec]; U^L: input W [pos][NR]
  float2* outp;            // forward: Y [pos][NR]; U^L: u [nrhs][len_out]
  int64_t len_vec, len_out;
  int32_t nrhs, rhs0, NR, c;
  int32_t R, item_stride;
};

size_t simt_smem_bytes(int nrb, int ns);
int simt_threads(int nrb);
cudaError_t simt_config(int nrb, int* grid, int* ns, size_t* smem);
cudaError_t launch_apply_simt(const ApplyArgs& a, int nrb, bool adj, int grid, size_t smem,
                              cudaStream_t stream);
// Bytes of dependency counters for a plan (S stages x groups, rounded up to 256).
size_t counter_bytes(const Plan& plan);

// tensor-core path (apply_tc.cu)
size_t tc_smem_bytes(int nsa, int mpad, int NR, int kpad_max);
size_t tc_counter_bytes(const TCPlan& plan);
size_t leaf_smem_bytes(int R, int c);
cudaError_t launch_apply_tc(const TCArgs& a, int grid, size_t smem, cudaStream_t stream);
cudaError_t launch_leaf(const LeafArgs& a, bool u_side, int n_groups, cudaStream_t stream);

}  // namespace mbf
