// Host/device interface of the apply kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "layout.hpp"

namespace mbf {

// Per-RHS row addresses of an apply's input and output, for up to kRowTab RHS: a served
// batch applies its requests' rows where the callers put them, with no staging copies.
// in[r] (n_in entries) and out[r] (n_out entries) for RHS r < nrhs.
constexpr int kRowTab = 64;
struct RowTable {
  const float2* in[kRowTab];
  float2* out[kRowTab];
};

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
  int32_t nrhs, n_pass, n_slots;
  int32_t accumulate;      // 1: out += result (the caller initialised out), 0: out = result
  // Failure-detection test hook (mbf_op_debug_stall); zero leaves the apply unchanged.
  // stall_stage1 = 1 + s: the dependency wait of group 0 of stage s (execution order)
  // waits for one more producer than exists, so that it can only end by running out of
  // time.  wait_ns > 0: every wait on a dependency counter, the pass barrier or a chunk
  // gives up after wait_ns instead of kTimeoutNs.
  uint64_t wait_ns;
  int32_t stall_stage1, stall_pad_;
  int32_t use_rows, rows_pad_;   // 1: in / out rows from `rows` (nrhs <= kRowTab)
  RowTable rows;
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


// Vectors between the tensor-core stages are "split blocks": block P of a level holds
// the R8 coefficients of one tree-node pair for the kTcNR right-hand sides of a panel
// as bf16 pairs hi = bf16(x), lo = bf16(x - hi), laid out as the MMA's K-major A
// operand with the real and imaginary parts of RHS n interleaved on M (rows
// m = 2 n + ri, ri = 0 real, 1 imaginary):
//   byte (hl, k, m) = hl R8 256 + (k / 8) 2048 + (m / 8) 128 + (m % 8) 16 + (k % 8) 2.
// A consumer copies each hi / lo half of a block into shared memory as it is.
constexpr int kTcNR = 64;   // RHS per tensor-core panel
MBF_HD int64_t split_block_bytes(int R8) { return int64_t(R8) * kTcNR * 8; }
// With TF32 operands the same block holds FP32 (TF32-rounded) values instead, byte
//   (k, m) = (k / 4) 2048 + (m / 8) 128 + (m % 8) 16 + (k % 4) 4
// (the MMA's K-major A operand for 32-bit types): the same R8 x 512 bytes.

struct TCArgs {
  const uint8_t* arena;
  const uint8_t* x_in;     // input of main stage 0 (split blocks)
  uint8_t* bufs;           // output of main stage e < S - 1: bufs + e * buf_stride (split blocks)
  float* y_out;            // output of the last main stage: row block * R + k, [re 64 | im 64] floats
  int64_t buf_stride;      // bytes
  unsigned* counters;      // [stage][group], zeroed per launch
  int* status;
  int32_t nsa, nxb;        // A ring slots; panel buffers (1 or 2)
  int32_t nsets, mt_max;   // accumulator sets (1 or 2, 2 mt_max TMEM columns each); largest M_t
  int32_t kpad_max, pad_;  // largest K_pad
  TCPlan plan;
};

struct LeafArgs {
  const uint8_t* arena;    // packed arena of the SIMT path (leaf items)
  const Item* items;
  int64_t item_base;       // item of group 0; group g's item is item_base + g * item_stride
  const int32_t* perm;     // U^L: tree -> natural x index; permute: natural -> tree Omega index
  const int32_t* off;      // leaf offsets (tree order)
  const float2* vec;       // (V^L)^*: panel in tree order [point][64]; permute: g [nrhs][len_vec]
  const float* wl;         // U^L: level-L coefficients, row block * R + k, [re 64 | im 64] floats
  float2* outp;            // U^L: u [nrhs][len_out]; permute: panel in tree order
  uint8_t* outs;           // (V^L)^*: split blocks of the level-L vector (block c g + t)
  int64_t len_vec, len_out;
  int32_t nrhs, rhs0, c, R;
  int32_t R8, item_stride;
  int32_t accumulate;       // U^L: 1 adds into u
  int32_t pts_cap;          // (V^L)^*: points staged per round (leaf_pts_cap of the largest leaf)
  int32_t leaf_split;       // U^L side: 1 = one CTA per leaf (ragged trees), 0 = one per group
  int32_t gather;           // (V^L)^* side: 1 = vec is [nrhs][len_vec] in natural order, read through
                            // nat; 0 = the tree-ordered panel
  int32_t nat_stride;       // (V^L)^* gather: entries per leaf in nat
  const int32_t* nat;       // (V^L)^* gather: leaf j's natural indices at nat[j * nat_stride + b]
  int32_t use_rows, rows_pad_;   // 1: (V^L)^* gather reads rows.in[rhs], U^L writes rows.out[rhs]
  RowTable rows;
};

size_t simt_smem_bytes(int nrb, int ns);
int simt_threads(int nrb);
cudaError_t simt_config(int nrb, int* grid, int* ns, size_t* smem);
cudaError_t launch_apply_simt(const ApplyArgs& a, int nrb, bool adj, int grid, size_t smem,
                              cudaStream_t stream);
// Bytes of dependency counters for a plan (S stages x groups, rounded up to 256).
size_t counter_bytes(const Plan& plan);

// tensor-core path (apply_tc.cu)
size_t tc_smem_bytes(int nsa, int nxb, int nsets, int mt_max, int kpad_max);
size_t tc_counter_bytes(const TCPlan& plan);
// Dynamic shared memory of a leaf kernel; the (V^L)^* side stages pts_cap points a round.
size_t leaf_smem_bytes(int R, int c, bool u_side, int pts_cap = 64);
// Points per round of the (V^L)^* leaf kernel for leaves of at most max_leaf_points
// points: rounded up to 8, within [8, 64].
int leaf_pts_cap(int64_t max_leaf_points);
bool leaf_fits(int R8, int c);   // leaf kernels: R8 <= 64, c <= 8
// tf32: TF32 tiles and vectors (kind::tf32 MMAs), else split-BF16x3.
cudaError_t launch_apply_tc(const TCArgs& a, int grid, size_t smem, cudaStream_t stream, bool tf32);
// TF32 tiles (two FP32 planes per K16 chunk) converted from n_chunks split-BF16 chunks of M_t rows.
cudaError_t launch_tf32_tiles(const uint8_t* src, uint8_t* dst, int64_t n_chunks, int M_t, cudaStream_t stream);
// U^L side: one CTA per group of c leaves; (V^L)^* side: one CTA per leaf (c n_groups CTAs).
// xpose: the adjoint's leaf products (U^* from the U^L items, V from the (V^L)^* items).
cudaError_t launch_leaf(const LeafArgs& a, bool u_side, int n_groups, cudaStream_t stream, bool tf32 = false,
                        bool xpose = false);
// Adjoint (conjugate-transposed) split-BF16 tiles of one stage from its forward tiles.
cudaError_t launch_adjoint_tiles(const uint8_t* src, uint8_t* dst, int n_groups, int M_t, int K_t, cudaStream_t stream);
// vec = g [nrhs][len_vec], perm = inverse tree permutation (natural -> tree, -1 if absent),
// outp = panel in tree order [tree point][64]
cudaError_t launch_permute_in(const LeafArgs& a, cudaStream_t stream);

}  // namespace mbf
