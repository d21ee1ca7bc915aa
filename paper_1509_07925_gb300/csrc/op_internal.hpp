// Definition of the resident operator object, shared by the host translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "layout.hpp"
#include "mbf_internal.hpp"

struct mbf_factors_s {
  mbf::FactorSet fs;
};

namespace mbf {
struct RowTable;   // apply.hpp

// Scratch of one apply in flight: the SIMT kernel's coefficient vectors, grid-barrier
// word and dependency counters, the status word its waits report to, and the tensor
// path's vectors, counters and tree-ordered input panel (allocated on first tensor
// use).  An operator owns one, and lends further ones from a pool it keeps to the
// server, so that batches of one operator can run at the same time.
struct Workspace {
  float2* bufs = nullptr;          // one coefficient vector per stage, 4 RHS wide
  unsigned* barrier = nullptr;     // barrier word, then (256 bytes on) the dependency counters
  int* status = nullptr;
  uint8_t* tc_bufs = nullptr;      // S_main + 1 vectors of c^L blocks x R8 x 64 entries (8 bytes each)
  unsigned* tc_counters = nullptr;
  float2* tc_gt = nullptr;         // input panel in Omega-tree order [n_w][64]
};
}  // namespace mbf

struct mbf_op_s {
  uint64_t serial = 0;              // unique per operator created in this process
  int device = 0;
  int d = 2, c = 4, L = 0, h = 0;
  int64_t n_out = 0, n_in = 0, n_w = 0;
  std::vector<int32_t> RU, RV;
  mbf::Plan plan{};
  int64_t nnz = 0, bytes_packed = 0;
  int64_t positions = 0;            // longest coefficient vector (c^L max R)
  uint8_t* d_arena = nullptr;
  mbf::Item* d_items = nullptr;
  int32_t *d_x_perm = nullptr, *d_x_off = nullptr, *d_w_perm = nullptr, *d_w_off = nullptr;
  int64_t leaf_pts_x = 0, leaf_pts_w = 0;   // points of the largest X / Omega leaf
  // per leaf, the natural indices of its points (tree order), padded to a stride of the
  // largest leaf rounded up to 8: the leaf kernels' gathers need no offset load first
  int32_t *d_x_nat = nullptr, *d_w_nat = nullptr;
  int32_t x_nat_stride = 0, w_nat_stride = 0;
  int32_t split_x = 0, split_w = 0;         // U^L-side leaf kernels: one CTA per leaf (ragged tree)
  mbf::Workspace ws;                // the scratch of the operator's own applies
  int grid = 0, ns[5] = {0, 0, 0, 0, 0};
  size_t smem[5] = {0, 0, 0, 0, 0};
  // tensor-core path: arena of split-bf16 tiles of the main stages, its plan, and the
  // panel workspace (allocated on first use)
  mbf::TCPlan tcplan{};
  uint8_t* d_tc_arena = nullptr;
  uint8_t* d_tc_arena_tf32 = nullptr; // the same tiles as TF32 planes (converted on first TF32 apply)
  int64_t tc_bytes = 0;
  int tc_mt_max = 16, tc_kpad_max = 16, tc_nsa = 2, tc_nxb = 2, tc_nsets = 2;
  size_t tc_smem = 0;
  int32_t* d_w_inv = nullptr;         // natural Omega index -> tree position (-1: not in the tree)
  std::string tc_unavailable;         // why the tensor path cannot run for this operator ("" if it can)
  std::string simt_unavailable;       // why the FP32 SIMT path cannot (leaves beyond its limits; "" if it can)
  // adjoint on the tensor cores: the stages reversed with conjugate-transposed tiles
  // (converted on the device from the forward tiles on the first adjoint apply)
  mbf::TCPlan tcplan_adj{};
  uint8_t* d_tc_arena_adj = nullptr;
  int tca_mt_max = 16, tca_kpad_max = 16, tca_nsa = 2, tca_nxb = 2, tca_nsets = 2;
  size_t tca_smem = 0;
  int32_t* d_x_inv = nullptr;         // natural x index -> X-tree position
  std::string tc_adj_unavailable;     // why the adjoint cannot run on the tensor cores
  int sms = 0;                        // SMs of the device (the persistent grids)
  int64_t tc_min_rhs = 8;             // AUTO: tensor cores from this many RHS (tuner may change it)
  std::vector<int64_t> nnz_stage;     // nonzero factor entries per forward stage
  int64_t nnz_leaf_x = 0;             // of which U^L
  // kernel timing (mbf_op_set_profiling): events bracketing each launch, by kind
  bool prof_on = false;
  struct ProfRec { int kind; cudaEvent_t e0, e1; };
  std::vector<ProfRec> prof_pending;
  int64_t prof_launches[8] = {};
  double prof_ms[8] = {};
  // staging for mbf_apply_host
  float2 *d_stage_in = nullptr, *d_stage_out = nullptr;
  size_t stage_in_bytes = 0, stage_out_bytes = 0;
  // pipeline of mbf_apply_host_batch: two staging pairs (input b, output b), the
  // host-to-device and device-to-host copy streams, and per pair the events "input
  // copied", "applied" and "output copied"
  float2* d_pipe_in[2] = {nullptr, nullptr};
  float2* d_pipe_out[2] = {nullptr, nullptr};
  size_t pipe_in_bytes = 0, pipe_out_bytes = 0;
  cudaStream_t pipe_st[2] = {nullptr, nullptr};
  cudaEvent_t pipe_ev[3][2] = {};
  // error estimate against the direct sum (mbf_op_estimate_error; -1 until made)
  double eps = -1.0;
  int32_t eps_samples = 0;
  // failure-detection test hook of the FP32 SIMT apply (mbf_op_debug_stall)
  int32_t dbg_stall_stage1 = 0;
  uint64_t dbg_wait_ns = 0;
  // workspaces lent to concurrent batches (the server): the operator's own one first,
  // then further ones, allocated on first need and kept until the operator is destroyed
  std::mutex ws_mu;
  bool ws_own_lent = false;
  std::vector<mbf::Workspace*> ws_pool;
  std::vector<bool> ws_pool_lent;
};


namespace mbf {
void set_last_error(const std::string& m);
// Internal entry points shared with the server and the tuner.  All throw mbf::Error.
bool uses_tensor(const mbf_op_s* op, int64_t nrhs, int32_t precision, bool adj);
void tc_prepare(mbf_op_s* op);
// Allocate a workspace for `op` (its SIMT parts; ws_prepare_tc adds the tensor path's,
// once) and free one.  Throw mbf::Error (MBF_ERR_OOM) on a failed allocation.
void ws_init(const mbf_op_s* op, Workspace& w);
void ws_prepare_tc(const mbf_op_s* op, Workspace& w);
void ws_free(Workspace& w);
// Borrow a workspace of `op` for one apply in flight (its own one if free, else one of its
// pool, allocated if every one is lent; with the tensor path's parts when `tensor`), and
// give it back.  Thread safe.
Workspace* ws_acquire(mbf_op_s* op, bool tensor);
void ws_release(mbf_op_s* op, Workspace* w);
int64_t tc_vec_bytes(const mbf_op_s* op);
// Apply on the device; grid > 0 caps the persistent kernels' CTA count (an SM share);
// accumulate adds the result into out (which the caller initialised).
// ws: the workspace to use (nullptr: the operator's own).  rows: per-RHS input and
// output rows instead of in / out (forward, device buffers, nrhs <= kRowTab).
void apply_dev(mbf_op_s* op, const void* in, void* out, int64_t nrhs, int32_t precision, cudaStream_t st,
               bool adj, int grid, bool accumulate = false, Workspace* ws = nullptr, const RowTable* rows = nullptr);
// The packed layouts of a factor set, made on the host by the same packers and checks
// that mbf_op_create runs before it uploads them: the SIMT plan, items and arena, and
// the tensor path's tile plan and arena (unless the tiles do not fit: tc_unavailable
// says why).  No device is touched.  Throws mbf::Error on an invalid factor set.
struct PackedHost {
  Plan plan{};
  std::vector<Item> items;
  std::vector<uint8_t> arena;
  TCPlan tcplan{};
  std::vector<uint8_t> tc_arena;
  TCPlan tcplan_adj{};   // the tensor adjoint's plan over the same tiles, transposed
  std::string simt_unavailable, tc_unavailable, tc_adj_unavailable;
};
void pack_host(const mbf_factors_t& f, PackedHost& out);
// The error estimator of §3.3 (estimate.cpp); keeps the result in op->eps.
double estimate_error(mbf_op_s* op, mbf_entry_fn fn, void* ctx, int32_t n_samples, uint64_t seed,
                      cudaStream_t st);
}  // namespace mbf
