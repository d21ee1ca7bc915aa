// Persistent SIMT apply of a butterfly factorization on sm_103a (single- and
// few-RHS path, FP32 arithmetic on complex64 factors).
//
// One CTA per SM walks every stage of eq. (gbf) -- (V^L)^*, (H^l)^*, M^h, G^l, U^L --
// in order (or the reverse, conjugated, for K^*).  Warp 0 is the producer: one
// lane streams the stage's factor chunks global -> shared with cp.async.bulk into
// a ring of 16 KB slots, each guarded by a full/empty mbarrier pair.  Factor data
// does not depend on the vectors, so the producer runs ahead across stage
// boundaries and keeps HBM busy while the consumers wait at the grid barrier.
// Warps 1..8 are consumers: they gather a group's input segments, multiply by the
// streamed block and scatter the result, then meet the other CTAs at a bounded
// grid barrier before the next stage.  Every wait gives up after kTimeoutNs, sets
// the status word and drains its own copies in flight before the CTA exits.
#include <cuda_runtime.h>

#include <cstdint>

#include "apply.hpp"

namespace mbf {

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory"); }
// Barrier among the consumer warps that also returns the OR of `v` over them, so
// every consumer takes the same branch afterwards.
__device__ __forceinline__ bool consumer_or(int v) {
  uint32_t res;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(res)
      : "r"(v), "n"(kConsumers)
      : "memory");
  return res != 0;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ float2 ld_cg(const float2* p) { return __ldcg(p); }

// Wait for phase `parity` of barrier b; false after kTimeoutNs or if abort is raised.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer();
  for (;;) {
    if (mbar_try(b, parity)) return true;
    if (*abort) return false;
    if (gtimer() - t0 > kTimeoutNs) return false;
  }
}

__device__ __forceinline__ void set_status(int* status, volatile int* abort, int code) {
  atomicCAS(status, 0, code);
  *abort = 1;
}

__device__ __forceinline__ int64_t pat_off(int pat, int g, int t, const Stage& s, int R, int c) {
  const int a = g / s.B, b = g - (g / s.B) * s.B;
  if (pat == PAT_SPLIT) return (int64_t(c * a + t) * s.B + b) * R;
  if (pat == PAT_CONTIG) return (int64_t(c) * g + t) * R;
  return (int64_t(c * b + t) * s.ch + a) * R;  // PAT_CORNER
}

struct Shared {
  uint64_t* full;
  uint64_t* empty;
  float2* xin;     // [kMaxLen][NRB] group input
  float2* yout;    // [kMaxLen][NRB] group output
  float2* red;     // [kConsumers][NRB] partial sums
  float2* xleaf;   // [kMaxLeaf][NRB] gathered leaf values
  volatile int* abort;
  volatile int* issued;
  volatile int* producer_done;
  uint8_t* ring;
};

// Consumer-side ring cursor.
struct Cursor {
  uint32_t kc;       // chunks consumed so far
  int ns;
};

template <int NRB>
struct Acc {
  float2 v[NRB];
};

// ---------------------------------------------------------------- consumers
// y[e] += sum_l T[l][e] x[l] over the item's lines (lines are inputs), thread (e, part).
// On exit dst[e] (e < len) holds the sum; all consumers synchronised.
template <int NRB, bool CONJ>
__device__ void axpy_item(const Item& it, const float2* __restrict__ x, float2* dst, Shared& sh,
                          Cursor& cur, int ctid, int* status) {
  const int len = it.len, nlines = it.nlines, lpc = it.lpc;
  const int parts = kConsumers / len;
  const int e = ctid % len, part = ctid / len;
  const bool active = part < parts;
  Acc<NRB> acc;
#pragma unroll
  for (int r = 0; r < NRB; ++r) acc.v[r] = make_float2(0.f, 0.f);
  const int lane = ctid & 31;
  for (int l0 = 0; l0 < nlines; l0 += lpc) {
    const int nl = min(lpc, nlines - l0);
    const int slot = int(cur.kc % uint32_t(cur.ns));
    const uint32_t ph = (cur.kc / uint32_t(cur.ns)) & 1u;
    // a wait that gives up raises abort; the chunk is then processed as garbage so
    // that every consumer keeps the same control flow (results are discarded)
    if (!mbar_wait(&sh.full[slot], ph, sh.abort) && !*sh.abort) set_status(status, sh.abort, ST_FULL_TIMEOUT);
    const float* re = reinterpret_cast<const float*>(sh.ring + size_t(slot) * kSlotBytes);
    const float* im = re + pad4(int64_t(nl) * len);
    if (active) {
#pragma unroll 4
      for (int l = part; l < nl; l += parts) {
        const float ar = re[l * len + e];
        const float ai = CONJ ? -im[l * len + e] : im[l * len + e];
        const float2* xl = x + size_t(l0 + l) * NRB;
#pragma unroll
        for (int r = 0; r < NRB; ++r) {
          const float2 xv = xl[r];
          acc.v[r].x = fmaf(ar, xv.x, fmaf(-ai, xv.y, acc.v[r].x));
          acc.v[r].y = fmaf(ar, xv.y, fmaf(ai, xv.x, acc.v[r].y));
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sh.empty[slot]);
    ++cur.kc;
  }
  if (active) {
#pragma unroll
    for (int r = 0; r < NRB; ++r) sh.red[ctid * NRB + r] = acc.v[r];
  }
  consumer_sync();
  if (ctid < len) {
#pragma unroll
    for (int r = 0; r < NRB; ++r) {
      float2 s = make_float2(0.f, 0.f);
      for (int p = 0; p < parts; ++p) {
        const float2 v = sh.red[(p * len + ctid) * NRB + r];
        s.x += v.x;
        s.y += v.y;
      }
      dst[ctid * NRB + r] = s;
    }
  }
  consumer_sync();
}

// out(line) = sum_e T[line][e] x[e] (lines are outputs), one warp per line.
template <int NRB, bool CONJ, class Sink>
__device__ void dot_item(const Item& it, const float2* __restrict__ x, Sink sink, Shared& sh,
                         Cursor& cur, int ctid, int* status) {
  const int len = it.len, nlines = it.nlines, lpc = it.lpc;
  const int warp = ctid >> 5, lane = ctid & 31;
  for (int l0 = 0; l0 < nlines; l0 += lpc) {
    const int nl = min(lpc, nlines - l0);
    const int slot = int(cur.kc % uint32_t(cur.ns));
    const uint32_t ph = (cur.kc / uint32_t(cur.ns)) & 1u;
    if (!mbar_wait(&sh.full[slot], ph, sh.abort) && !*sh.abort) set_status(status, sh.abort, ST_FULL_TIMEOUT);
    const float* re = reinterpret_cast<const float*>(sh.ring + size_t(slot) * kSlotBytes);
    const float* im = re + pad4(int64_t(nl) * len);
    for (int l = warp; l < nl; l += kConsumerWarps) {
      Acc<NRB> acc;
#pragma unroll
      for (int r = 0; r < NRB; ++r) acc.v[r] = make_float2(0.f, 0.f);
      for (int e = lane; e < len; e += 32) {
        const float ar = re[l * len + e];
        const float ai = CONJ ? -im[l * len + e] : im[l * len + e];
#pragma unroll
        for (int r = 0; r < NRB; ++r) {
          const float2 xv = x[e * NRB + r];
          acc.v[r].x = fmaf(ar, xv.x, fmaf(-ai, xv.y, acc.v[r].x));
          acc.v[r].y = fmaf(ar, xv.y, fmaf(ai, xv.x, acc.v[r].y));
        }
      }
#pragma unroll
      for (int r = 0; r < NRB; ++r) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          acc.v[r].x += __shfl_xor_sync(0xffffffffu, acc.v[r].x, o);
          acc.v[r].y += __shfl_xor_sync(0xffffffffu, acc.v[r].y, o);
        }
      }
      if (lane == 0) sink(l0 + l, acc);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sh.empty[slot]);
    ++cur.kc;
  }
  consumer_sync();
}

// ---------------------------------------------------------------- kernel

template <int NRB, bool ADJ>
__global__ void __launch_bounds__(kThreads, 1) bf_apply_simt(const __grid_constant__ ApplyArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int ns = a.n_slots;
  Shared sh;
  sh.ring = smem;
  uint8_t* p = smem + size_t(ns) * kSlotBytes;
  sh.full = reinterpret_cast<uint64_t*>(p);
  sh.empty = sh.full + ns;
  p += 16 * size_t(ns);
  sh.xin = reinterpret_cast<float2*>(p);
  sh.yout = sh.xin + kMaxLen * NRB;
  sh.red = sh.yout + kMaxLen * NRB;
  sh.xleaf = sh.red + kConsumers * NRB;
  int* flags = reinterpret_cast<int*>(sh.xleaf + kMaxLeaf * NRB);
  sh.abort = flags;
  sh.issued = flags + 1;
  sh.producer_done = flags + 2;

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < ns; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], kConsumerWarps);
    }
    flags[0] = 0;
    flags[1] = 0;
    flags[2] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const Plan& plan = a.plan;
  const int S = plan.n_stages, c = plan.c;

  if (tid < 32) {
    // ------------------------------------------------------------ producer
    if (tid == 0) {
      uint32_t kc = 0;
      bool ok = true;
      for (int pass = 0; pass < a.n_pass && ok; ++pass) {
        for (int e = 0; e < S && ok; ++e) {
          const Stage& st = plan.st[ADJ ? S - 1 - e : e];
          for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x) {
            for (int mi = 0; mi < st.n_items && ok; ++mi) {
              const int idx = ADJ ? st.n_items - 1 - mi : mi;
              const Item it = a.items[st.item_base + int64_t(g) * st.n_items + idx];
              const uint8_t* src = a.arena + it.offset;
              for (int l0 = 0; l0 < it.nlines; l0 += it.lpc) {
                const int nl = min(int(it.lpc), int(it.nlines) - l0);
                const uint32_t bytes = uint32_t(chunk_bytes(nl, it.len));
                const int slot = int(kc % uint32_t(ns));
                const uint32_t ph = (kc / uint32_t(ns)) & 1u;
                if (*sh.abort) { ok = false; break; }
                if (!mbar_wait(&sh.empty[slot], ph ^ 1u, sh.abort)) {
                  if (!*sh.abort) set_status(a.status, sh.abort, ST_EMPTY_TIMEOUT);
                  ok = false;
                  break;
                }
                mbar_expect_tx(&sh.full[slot], bytes);
                bulk_g2s(sh.ring + size_t(slot) * kSlotBytes, src, bytes, &sh.full[slot]);
                src += bytes;
                ++kc;
                *sh.issued = int(kc);
              }
            }
          }
        }
      }
      __threadfence_block();
      *sh.producer_done = 1;
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int ctid = tid - 32;
  Cursor cur{0u, ns};
  unsigned nbar = 0;
  bool ok = true;
  for (int pass = 0; pass < a.n_pass && ok; ++pass) {
    const int rhs0 = pass * NRB;
    for (int e = 0; e < S && ok; ++e) {
      const Stage& st = plan.st[ADJ ? S - 1 - e : e];
      // grid-wide barrier between consecutive stages (and passes)
      if (pass > 0 || e > 0) {
        ++nbar;
        consumer_sync();
        if (ctid == 0) {
          __threadfence();
          atomicAdd(a.barrier, 1u);
          const unsigned target = nbar * gridDim.x;
          const uint64_t t0 = gtimer();
          while (ld_acquire(a.barrier) < target) {
            if (*reinterpret_cast<volatile int*>(a.status) != 0) { *sh.abort = 1; break; }
            if (gtimer() - t0 > kTimeoutNs) { set_status(a.status, sh.abort, ST_BARRIER_TIMEOUT); break; }
            __nanosleep(40);
          }
          __threadfence();
        }
        if (consumer_or(*sh.abort)) { ok = false; break; }
      }
      const float2* src = (e & 1) ? a.buf0 : a.buf1;   // previous stage's output
      float2* dst = (e & 1) ? a.buf1 : a.buf0;
      const int in_pat = ADJ ? st.out_pat : st.in_pat;
      const int out_pat = ADJ ? st.in_pat : st.out_pat;
      const int Rin = ADJ ? st.R_out : st.R_in;    // execution-sense segment lengths
      const int Rout = ADJ ? st.R_in : st.R_out;

      for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x) {
        if (in_pat != PAT_LEAF) {
          for (int q = ctid; q < c * Rin * NRB; q += kConsumers) {
            const int r = q % NRB, k = (q / NRB) % Rin, t = q / (NRB * Rin);
            const int64_t pos = pat_off(in_pat, g, t, st, Rin, c) + k;
            sh.xin[q] = ld_cg(src + pos * NRB + r);
          }
        }
        consumer_sync();
        for (int mi = 0; mi < st.n_items && ok; ++mi) {
          const int idx = ADJ ? st.n_items - 1 - mi : mi;
          const Item it = a.items[st.item_base + int64_t(g) * st.n_items + idx];
          const int max_lines = it.kind == ITEM_MAIN ? kMaxLen : kMaxLeaf;
          if (it.len > kMaxLen || it.len == 0 || it.nlines > max_lines) {
            set_status(a.status, sh.abort, ST_BAD_ITEM);
            ok = false;
            break;
          }
          const int leaf = c * g + it.t;
          if (it.kind == ITEM_MAIN) {
            if (!ADJ) {
              axpy_item<NRB, false>(it, sh.xin, sh.yout, sh, cur, ctid, a.status);
            } else {
              float2* yo = sh.yout;
              auto sink = [yo](int line, const Acc<NRB>& v) {
#pragma unroll
                for (int r = 0; r < NRB; ++r) yo[line * NRB + r] = v.v[r];
              };
              dot_item<NRB, true>(it, sh.xin, sink, sh, cur, ctid, a.status);
            }
            if (out_pat != PAT_LEAF) {
              for (int q = ctid; q < c * Rout * NRB; q += kConsumers) {
                const int r = q % NRB, k = (q / NRB) % Rout, t = q / (NRB * Rout);
                const int64_t pos = pat_off(out_pat, g, t, st, Rout, c) + k;
                dst[pos * NRB + r] = sh.yout[q];
              }
            }
          } else {
            const bool is_in = (!ADJ && it.kind == ITEM_LEAF_W) || (ADJ && it.kind == ITEM_LEAF_X);
            const int32_t* perm = it.kind == ITEM_LEAF_W ? a.w_perm : a.x_perm;
            const int32_t* off = it.kind == ITEM_LEAF_W ? a.w_off : a.x_off;
            const int base = off[leaf];
            if (is_in) {
              // gather the leaf's input values, then (V^L)^* (forward) or (U^L)^* (adjoint)
              for (int q = ctid; q < it.nlines * NRB; q += kConsumers) {
                const int r = q % NRB, l = q / NRB;
                const int rhs = rhs0 + r;
                sh.xleaf[q] = rhs < a.nrhs ? __ldg(a.in + int64_t(rhs) * a.in_len + perm[base + l])
                                           : make_float2(0.f, 0.f);
              }
              consumer_sync();
              axpy_item<NRB, ADJ>(it, sh.xleaf, sh.xin + it.t * it.len * NRB, sh, cur, ctid, a.status);
            } else {
              // U^L (forward) or V^L (adjoint) and the scatter to natural order
              float2* outp = a.out;
              const int64_t out_len = a.out_len;
              const int nrhs = a.nrhs;
              const int32_t* pp = perm + base;
              auto sink = [outp, out_len, nrhs, rhs0, pp](int line, const Acc<NRB>& v) {
                const int64_t col = pp[line];
#pragma unroll
                for (int r = 0; r < NRB; ++r)
                  if (rhs0 + r < nrhs) outp[int64_t(rhs0 + r) * out_len + col] = v.v[r];
              };
              dot_item<NRB, ADJ>(it, sh.yout + it.t * it.len * NRB, sink, sh, cur, ctid, a.status);
            }
          }
        }
        if (consumer_or(*sh.abort)) ok = false;
      }
    }
  }

  // Drain: on an abort, wait (bounded) for every copy this CTA issued but did not
  // consume, so no bulk copy is still writing shared memory when the CTA exits.
  if (!ok && ctid == 0) {
    const uint64_t t0 = gtimer();
    while (!*sh.producer_done && gtimer() - t0 < kTimeoutNs) __nanosleep(100);
    const uint32_t issued = uint32_t(*sh.issued);
    for (int s = 0; s < ns; ++s) {
      if (issued <= uint32_t(s)) continue;
      const uint32_t last = uint32_t(s) + ((issued - 1u - uint32_t(s)) / uint32_t(ns)) * uint32_t(ns);
      const uint32_t ph = (last / uint32_t(ns)) & 1u;
      const uint64_t t1 = gtimer();
      while (!mbar_try(&sh.full[s], ph) && gtimer() - t1 < kTimeoutNs) {
      }
    }
  }
}

// ---------------------------------------------------------------- host side

size_t simt_smem_bytes(int nrb, int ns) {
  return size_t(ns) * kSlotBytes + 16 * size_t(ns) +
         sizeof(float2) * size_t(nrb) * (2 * kMaxLen + kConsumers + kMaxLeaf) + 64;
}

template <int NRB, bool ADJ>
static cudaError_t launch_t(const ApplyArgs& a, int grid, size_t smem, cudaStream_t stream) {
  auto kern = bf_apply_simt<NRB, ADJ>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// Largest slot count that fits the opt-in shared memory, and the co-resident grid.
cudaError_t simt_config(int nrb, int* grid, int* ns, size_t* smem) {
  int dev = 0, sms = 0, optin = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return err;
  int slots = 16;
  while (slots > 2 && simt_smem_bytes(nrb, slots) > size_t(optin)) --slots;
  *ns = slots;
  *smem = simt_smem_bytes(nrb, slots);
  *grid = sms;   // one CTA per SM (the shared-memory footprint allows no more)
  return cudaSuccess;
}

cudaError_t launch_apply_simt(const ApplyArgs& a, int nrb, bool adj, int grid, size_t smem,
                              cudaStream_t stream) {
  cudaError_t err = cudaMemsetAsync(a.barrier, 0, sizeof(unsigned), stream);
  if (err != cudaSuccess) return err;
  switch (nrb * 2 + (adj ? 1 : 0)) {
    case 2: return launch_t<1, false>(a, grid, smem, stream);
    case 3: return launch_t<1, true>(a, grid, smem, stream);
    case 4: return launch_t<2, false>(a, grid, smem, stream);
    case 5: return launch_t<2, true>(a, grid, smem, stream);
    case 8: return launch_t<4, false>(a, grid, smem, stream);
    case 9: return launch_t<4, true>(a, grid, smem, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mbf
