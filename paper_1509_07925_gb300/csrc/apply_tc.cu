// Tensor-core apply of a butterfly factorization for panels of 64 right-hand sides
// (sm_103a: tcgen05 MMAs, TMEM accumulators, cp.async.bulk staging).
//
// Every group product of a G^l / (H^l)^* level, Y = T X with T complex (M_t x K_t) and X
// complex (K_t x 64), is computed transposed, Y^T = X^T T^T, on split-BF16 operands
// (T = T_hi + T_lo, X = X_hi + X_lo, products hi*hi + hi*lo + lo*hi, FP32 accumulation).
// The MMA's A operand interleaves the real and imaginary parts of X^T on M (row 2 n is
// X_re[:, n], row 2 n + 1 is X_im[:, n]: M = 128), its B operand is one plane of T
// (N = M_t), so two accumulators
//     D1 = A T_re^T,     D2 = A T_im^T
// give Y_re^T[n] = D1[2n] - D2[2n + 1] and Y_im^T[n] = D2[2n] + D1[2n + 1]: the two lanes
// of an output pair are neighbours in one warp.  With the tile's Re and Im planes
// adjacent, D1 | D2 is one MMA of N = 2 M_t: three MMAs per K = 16.
// The vectors between stages are kept as split blocks (apply.hpp), so a group's X is
// two contiguous runs per input block.
//
// Warp roles in a CTA (one per SM, persistent, cooperative):
//   warp 0     two lanes stream each group's tile, chunk by chunk (K = 16 columns,
//              4 planes), into a ring of shared-memory slots (full/empty mbarriers);
//   warp 1     allocates TMEM; runs the MMA loop (warp-uniform operands), one elected
//              lane issuing the MMAs into an accumulator set and the commits;
//   warp 2     lane 0 waits for a group's inputs (dependency counters), then one lane
//              per block half bulk-copies the c blocks into a panel buffer
//              (complete_tx on its mbarrier);
//   warps 4-7, 8-11   epilogue sets, one per accumulator set: read the accumulators
//              (tcgen05.ld, 32 columns of each half a round), pair the halves by warp
//              shuffles, split and store the group's output blocks, and hand them to
//   warp 12    the signal warp, which fences and counts them in for the consumers;
//   warps 3, 13  drop each group's consumed input blocks from L2 once its MMAs are done.
// The (V^L)^* and U^L leaf products run before and after it (leaf kernels below).
// Every wait is bounded; on a timeout the status word is set and all roles drain.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "apply.hpp"

namespace mbf {

namespace tc {

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t sa(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(sa(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sa(dst)),
      "l"(src), "r"(bytes), "r"(sa(bar))
      : "memory");
}
// Same, with an L2 eviction-priority policy for the source lines.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          sa(dst)),
      "l"(src), "r"(bytes), "r"(sa(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// 16-byte global -> shared copy through L2 (cp.async, the load/store path).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}
// Drop a 128-byte line from L2 without writing it back (its contents become undefined).
__device__ __forceinline__ void l2_discard(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Shared-memory matrix descriptor: start, leading (K-direction core-matrix) and
// stride (M/N-direction) byte offsets, fixed bit 46, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// FP32 -> TF32 (round to nearest, ties away from zero), kept in an FP32 container.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ uint4 tf32x4(const float* y) {
  return make_uint4(__float_as_uint(to_tf32(y[0])), __float_as_uint(to_tf32(y[1])), __float_as_uint(to_tf32(y[2])),
                    __float_as_uint(to_tf32(y[3])));
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
// Named barrier that also ORs a flag over the participating threads, so that every
// thread takes the same branch after it.
__device__ __forceinline__ bool named_sync_or(int id, int n, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(uint32_t(v)), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}


// 16 consecutive TMEM columns of this thread's lane (one row of the accumulator),
// written straight into the 16 FP32 registers (b32 operands take any 32-bit register).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
      : "r"(taddr));
}
// 32 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
        "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]),
        "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]),
        "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Uses of registers written by tcgen05.ld must not move above the tcgen05.wait::ld that
// completes them: after the wait, each register passes through an empty asm that the
// compiler must assume rewrites it (volatile asms keep their order).
template <int K>
__device__ __forceinline__ void tmem_hold(float (&x)[K], float (&y)[K]) {
#pragma unroll
  for (int j = 0; j < K; ++j) asm volatile("" : "+f"(x[j]));
#pragma unroll
  for (int j = 0; j < K; ++j) asm volatile("" : "+f"(y[j]));
}

// Two floats -> bf16x2 (round to nearest even), the first in the low half.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo_half, float hi_half) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_half), "f"(lo_half));
  return r;
}
// Split 8 floats into hi = bf16(x) and lo = bf16(x - hi) (4 words each).
__device__ __forceinline__ void split8(const float* y, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = pack_bf16x2(y[2 * i], y[2 * i + 1]);
    const float r0 = y[2 * i] - __uint_as_float(h[i] << 16), r1 = y[2 * i + 1] - __uint_as_float(h[i] & 0xffff0000u);
    l[i] = pack_bf16x2(r0, r1);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// One lane of the (converged) warp: true in exactly one lane.
__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile("{\n .reg .pred P;\n elect.sync _|P, 0xffffffff;\n selp.u32 %0, 1, 0, P;\n}\n" : "=r"(pred));
  return pred != 0;
}

// Block index (tree-node pair of the level) of segment t of group g under a pattern.
__device__ __forceinline__ int64_t pat_blk(int pat, int g, int t, const TCStage& s, int c) {
  const int a = g / s.B, b = g - (g / s.B) * s.B;
  if (pat == PAT_SPLIT) return int64_t(c * a + t) * s.B + b;
  if (pat == PAT_CONTIG) return int64_t(c) * g + t;
  return int64_t(c * b + t) * s.ch + a;  // PAT_CORNER
}
__device__ __forceinline__ int pat_group(int pat, int64_t P, const TCStage& s, int c) {
  if (pat == PAT_CONTIG) return int(P / c);
  if (pat == PAT_SPLIT) {
    const int64_t q = P / s.B;
    return int((q / c) * s.B + (P - q * s.B));
  }
  const int64_t q = P / s.ch;
  return int((P - q * s.ch) * s.B + q / c);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

// Bounded wait on an mbarrier phase.  Returns false on timeout or abort.
__device__ __forceinline__ bool wait_bar(uint64_t* b, uint32_t ph, volatile int* abort) {
  if (mbar_try(b, ph)) return true;
  const uint64_t t0 = gtimer();
  for (;;) {
    if (mbar_try(b, ph)) return true;
    if (*abort) return false;
    if (gtimer() - t0 > kTimeoutNs) return false;
  }
}

}  // namespace tc

constexpr int kTcThreads = 448;   // 14 warps (roles above)
constexpr int kAProducers = 2;    // lanes of warp 0 issuing the tile copies
constexpr int kMaxXBufs = 3;      // panel buffers at most (the autotuner picks 2 or 3)
constexpr int kTcChunk = 16;   // accumulator columns per epilogue step

// TF32: the vectors between stages are TF32 blocks (apply.hpp) and the tiles two FP32
// planes (Re, Im) per K16 chunk; kind::tf32 MMAs of K = 8.  Otherwise split-BF16x3.
template <bool TF32>
__global__ void __launch_bounds__(kTcThreads, 1) bf_apply_tc(const __grid_constant__ TCArgs a) {
  using namespace tc;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int nsa = a.nsa, nxb = a.nxb, nsets = a.nsets;
  const uint32_t a_slot = 4u * uint32_t(a.mt_max) * 32u;       // one K16 chunk of a tile (4 planes)
  const uint32_t x_buf = 2u * uint32_t(a.kpad_max) * 256u;      // hi + lo halves of a panel
  uint8_t* aring = smem;
  uint8_t* xbuf = aring + size_t(nsa) * a_slot;
  uint64_t* afull = reinterpret_cast<uint64_t*>(xbuf + size_t(nxb) * x_buf);
  uint64_t* aempty = afull + nsa;
  uint64_t* xfull = aempty + nsa;
  uint64_t* xempty = xfull + kMaxXBufs;
  uint64_t* dfull = xempty + kMaxXBufs;
  uint64_t* dempty = dfull + 2;
  uint64_t* stored = dempty + 2;     // [set]: the set's output blocks of a group are written
  uint64_t* signaled = stored + 2;   // [set]: the signal warp has counted them in
  uint64_t* done = signaled + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < nsa; ++i) {
      mbar_init(&afull[i], 1);
      mbar_init(&aempty[i], 1);
    }
    for (int s = 0; s < nxb; ++s) {
      mbar_init(&xfull[s], 1);
      mbar_init(&xempty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&dfull[s], 1);
      mbar_init(&dempty[s], 128);
    }
    for (int s2 = 0; s2 < 2; ++s2) {
      mbar_init(&stored[s2], 128);
      mbar_init(&signaled[s2], 1);
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(sa(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *tslot;
  const TCPlan& plan = a.plan;
  const int S = plan.n_stages, c = plan.c;
  const uint32_t set_cols = 2u * uint32_t(a.mt_max);   // D1 | D2 of one accumulator set

  if (warp == 0 && lane < kAProducers) {
    // ---------------------------------------------------------------- A tiles
    // (streamed once: first out of L2, so that the stage vectors stay there).  A thread
    // issues one bulk copy every few hundred ns whatever its size, so kAProducers lanes
    // share the chunks: lane p takes chunks ca = p mod kAProducers, i.e. the ring slots
    // of that residue (nsa is a multiple of kAProducers).
    const uint64_t pol = policy_evict_first();
    uint32_t ca = 0;
    bool ok = true;
    for (int e = 0; e < S && ok; ++e) {
      const TCStage& st = plan.st[e];
      const int nk = st.K_pad / 16;
      const uint32_t chunk = 4u * uint32_t(st.plane_bytes);
      for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x) {
        const uint8_t* src = a.arena + st.base + int64_t(g) * st.tile_bytes;
        for (int kk = 0; kk < nk; ++kk, ++ca) {
          if (int(ca % uint32_t(kAProducers)) != lane) continue;
          const uint32_t slot = ca % uint32_t(nsa), ph = (ca / uint32_t(nsa)) & 1u;
          if (!wait_bar(&aempty[slot], ph ^ 1u, abort)) {
            if (!*abort) {
              atomicCAS(a.status, 0, ST_EMPTY_TIMEOUT);
              *abort = 1;
            }
            ok = false;
            break;
          }
          mbar_expect_tx(&afull[slot], chunk);
          bulk_g2s_hint(aring + size_t(slot) * a_slot, src + int64_t(kk) * chunk, chunk, &afull[slot], pol);
        }
      }
    }
    // wait (bounded) for every copy of this lane still in flight
    for (uint32_t q = (ca > uint32_t(nsa) ? ca - uint32_t(nsa) : 0u); q < ca; ++q) {
      if (int(q % uint32_t(kAProducers)) != lane) continue;
      const uint32_t slot = q % uint32_t(nsa), ph = (q / uint32_t(nsa)) & 1u;
      const uint64_t t1 = gtimer();
      while (!mbar_try(&afull[slot], ph) && gtimer() - t1 < kTimeoutNs) {
      }
    }
  } else if (warp == 2) {
    // ---------------------------------------------------------------- X panels
    // Lane 0 waits for a group's panel buffer and its c input blocks (dependency
    // counters); then lanes 0 .. c kParts - 1 each issue one bulk copy of a block half
    // (split-BF16: the hi halves of the c blocks side by side, then the lo halves; TF32:
    // one run per block), all completing on the buffer's xfull barrier: a thread issues
    // one bulk copy every few hundred ns, so the copies go out from separate lanes.  The
    // consumed blocks are dropped from L2 later, by the discard warps, once the group's
    // MMAs are done.
    int j = 0;
    bool ok = true;
    for (int e = 0; e < S && ok; ++e) {
      const TCStage& st = plan.st[e];
      const uint8_t* src = e == 0 ? a.x_in : a.bufs + int64_t(e - 1) * a.buf_stride;
      const unsigned* cnt_in = a.counters + int64_t(e) * st.n_groups;
      const uint32_t half = TF32 ? uint32_t(st.R8_in) * 512u : uint32_t(st.R8_in) * 256u;
      const uint32_t xhalf = uint32_t(st.K_pad) * 256u;     // hi or lo half of the panel buffer
      const int64_t blk = split_block_bytes(st.R8_in);
      constexpr int kParts = TF32 ? 1 : 2;
      for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x, ++j) {
        const int xs = j % nxb;
        const uint32_t xu = uint32_t(j / nxb);
        bool fail = false;
        if (lane == 0) {
          fail = !wait_bar(&xempty[xs], (xu & 1u) ^ 1u, abort);
          // all c input blocks written by the previous stage
          if (!fail && e > 0) {
            const unsigned* cp = cnt_in + g;
            const uint64_t t0 = gtimer();
            while (ld_acquire(cp) < unsigned(c)) {
              if (*abort || *reinterpret_cast<volatile int*>(a.status) != 0) {
                fail = true;
                break;
              }
              if (gtimer() - t0 > kTimeoutNs) {
                atomicCAS(a.status, 0, ST_DEP_TIMEOUT);
                fail = true;
                break;
              }
              __nanosleep(32);
            }
          }
          if (fail) *abort = 1;
          else mbar_expect_tx(&xfull[xs], uint32_t(kParts * c) * half);
        }
        if (__shfl_sync(0xffffffffu, fail ? 1 : 0, 0)) {   // (also orders the expect before the copies)
          ok = false;
          break;
        }
        if (lane < kParts * c) {
          const int t = lane / kParts, hl = lane - t * kParts;
          const uint8_t* sb = src + int64_t(pat_blk(st.in_pat, g, t, st, c)) * blk;
          uint8_t* xb = xbuf + size_t(xs) * x_buf;
          bulk_g2s(xb + uint32_t(hl) * xhalf + uint32_t(t) * half, sb + int64_t(hl) * half, half, &xfull[xs]);
        }
      }
    }
    // wait (bounded) for the copies of the last groups still in flight
    if (lane == 0) {
      for (int q = (j > nxb ? j - nxb : 0); q < j; ++q) {
        const uint64_t t1 = gtimer();
        while (!mbar_try(&xfull[q % nxb], uint32_t(q / nxb) & 1u) && gtimer() - t1 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 3 || warp == 13) {
    // ---------------------------------------------------------------- L2 discards
    // Once a group's MMAs are done (its panel buffer's xempty phase), its c input blocks
    // are neither in shared memory nor read again: their lines are dropped from L2
    // without a write-back.  Each discard takes a while, so two warps share them.
    const int dt = (warp == 3 ? 0 : 32) + lane;
    int j = 0;
    bool ok = true;
    for (int e = 0; e < S && ok; ++e) {
      const TCStage& st = plan.st[e];
      const uint8_t* src = e == 0 ? a.x_in : a.bufs + int64_t(e - 1) * a.buf_stride;
      const int64_t blk = split_block_bytes(st.R8_in);
      for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x, ++j) {
        const int xs = j % nxb;
        const uint32_t xu = uint32_t(j / nxb);
        if (!__all_sync(0xffffffffu, wait_bar(&xempty[xs], xu & 1u, abort))) {
          ok = false;
          break;
        }
        for (int t = 0; t < c; ++t) {
          const uint8_t* sb = src + int64_t(pat_blk(st.in_pat, g, t, st, c)) * blk;
          for (int64_t q = dt; q < (blk >> 7); q += 64) l2_discard(sb + (q << 7));
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    // The whole warp runs the loop, so that descriptors and addresses are warp-uniform;
    // one elected lane issues the MMAs and the commits.
    uint32_t ca = 0;
    int j = 0;
    bool ok = true;
    const uint32_t abase = sa(aring), xbase0 = sa(xbuf);
    for (int e = 0; e < S && ok; ++e) {
      const TCStage& st = plan.st[e];
      const int nk = st.K_pad / 16;
      const uint32_t xhalf = uint32_t(st.K_pad) * 256u;
      const uint32_t pb = uint32_t(st.plane_bytes);
      // kind::f16, FP32 accumulate, BF16 A and B, both K-major, M = 128.  While 2 M_t <= 256
      // the Re and Im planes of the tile form one B operand of N = 2 M_t rows (three MMAs
      // per K16 fill D1 | D2 at once); wider tiles take N = M_t, one MMA per plane.
      // (TF32: kind::tf32, A and B TF32, K = 8 per MMA; planes Re, Im of M_t x 16 FP32)
      const bool stack = 2 * st.M_t <= 256;
      const uint32_t nmma = uint32_t(stack ? 2 * st.M_t : st.M_t);
      const uint32_t ab = TF32 ? 2u : 1u;   // operand format: BF16 = 1, TF32 = 2
      const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((nmma >> 3) << 17) | (uint32_t(128 >> 4) << 24);
      const uint32_t pbt = uint32_t(st.M_t) * 64u;   // TF32: one K16 chunk of one plane
      for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x, ++j) {
        const int xs = j % nxb, ds = j % nsets;
        const uint32_t xu = uint32_t(j / nxb), du = uint32_t(j / nsets);
        const bool got = wait_bar(&xfull[xs], xu & 1u, abort) && wait_bar(&dempty[ds], (du & 1u) ^ 1u, abort);
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0 && !*abort) {
            atomicCAS(a.status, 0, ST_FULL_TIMEOUT);
            *abort = 1;
          }
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d1 = taddr + uint32_t(ds) * set_cols, d2 = d1 + uint32_t(st.M_t);
        const uint32_t xb = xbase0 + uint32_t(xs) * x_buf;
        for (int kk = 0; kk < nk; ++kk, ++ca) {
          const uint32_t slot = ca % uint32_t(nsa), ph = (ca / uint32_t(nsa)) & 1u;
          if (!__all_sync(0xffffffffu, wait_bar(&afull[slot], ph, abort))) {
            if (lane == 0 && !*abort) {
              atomicCAS(a.status, 0, ST_FULL_TIMEOUT);
              *abort = 1;
            }
            ok = false;
            break;
          }
          // (the chunk was written by the bulk copy the mbarrier tracks: no tcgen05 fence)
          const uint32_t as = abase + slot * a_slot;
          if constexpr (TF32) {
            // A: K-major, 4 K (16 bytes) per core matrix: next 4 K at +2048, next 8 rows at
            // +128; chunk kk at +8192, its second K = 8 at +4096.  B: planes 0 Re, 1 Im,
            // next 4 K at +128, next 8 rows at +512; second K = 8 at +256.
            const uint64_t x0 = sdesc(xb + uint32_t(kk) * 8192u, 2048u, 128u);
            const uint64_t x1 = sdesc(xb + uint32_t(kk) * 8192u + 4096u, 2048u, 128u);
            const uint64_t r0 = sdesc(as, 128u, 512u), r1 = sdesc(as + 256u, 128u, 512u);
            const uint64_t i0 = sdesc(as + pbt, 128u, 512u), i1 = sdesc(as + pbt + 256u, 128u, 512u);
            const uint32_t acc0 = kk > 0 ? 1u : 0u;
            if (elect_one()) {
              mma_tf32(d1, x0, r0, idesc, acc0);   // stacked: r0 spans [Re; Im]
              mma_tf32(d1, x1, r1, idesc, 1u);
              if (!stack) {
                mma_tf32(d2, x0, i0, idesc, acc0);
                mma_tf32(d2, x1, i1, idesc, 1u);
              }
              mma_commit(&aempty[slot]);
            }
            __syncwarp();
            continue;
          }
          // A: panel half (hi / lo), K-major, next 8 K at +2048, next 8 rows at +128
          const uint64_t xh = sdesc(xb + uint32_t(kk) * 4096u, 2048u, 128u);
          const uint64_t xl = sdesc(xb + xhalf + uint32_t(kk) * 4096u, 2048u, 128u);
          // B: tile planes 0 Re hi, 1 Im hi, 2 Re lo, 3 Im lo; next 8 K at +128, next 8 rows at +256
          const uint64_t t0 = sdesc(as, 128u, 256u), t1 = sdesc(as + pb, 128u, 256u);
          const uint64_t t2 = sdesc(as + 2u * pb, 128u, 256u), t3 = sdesc(as + 3u * pb, 128u, 256u);
          const uint32_t acc0 = kk > 0 ? 1u : 0u;
          if (elect_one()) {
            if (stack) {          // t0 spans [Re hi; Im hi], t2 spans [Re lo; Im lo]
              mma_bf16(d1, xh, t0, idesc, acc0);
              mma_bf16(d1, xh, t2, idesc, 1u);
              mma_bf16(d1, xl, t0, idesc, 1u);
            } else {
              mma_bf16(d1, xh, t0, idesc, acc0);
              mma_bf16(d1, xh, t2, idesc, 1u);
              mma_bf16(d1, xl, t0, idesc, 1u);
              mma_bf16(d2, xh, t1, idesc, acc0);
              mma_bf16(d2, xh, t3, idesc, 1u);
              mma_bf16(d2, xl, t1, idesc, 1u);
            }
            mma_commit(&aempty[slot]);
          }
          __syncwarp();
        }
        if (!ok) break;
        if (elect_one()) {
          mma_commit(&dfull[ds]);
          mma_commit(&xempty[xs]);
        }
        __syncwarp();
      }
    }
    // every MMA this warp issued has completed before TMEM is freed
    if (elect_one()) mma_commit(done);
    __syncwarp();
    const uint64_t t1 = gtimer();
    while (!mbar_try(done, 0) && gtimer() - t1 < kTimeoutNs) {
    }
  } else if (warp >= 4 && (warp - 4) / 4 < nsets) {
    // ---------------------------------------------------------------- epilogue sets
    // TMEM lane tl is row tl of the panel: RHS n = tl / 2, real (ri = 0) or imaginary
    // (ri = 1) part, so the two halves of a complex output sit in adjacent lanes of one
    // warp and pair by a shuffle.  Each warp works on its own.
    const int set = (warp - 4) >> 2;             // 0: warps 4-7, 1: warps 8-11
    const int quarter = warp & 3;                // TMEM lane quarter this warp may access
    const int tl = quarter * 32 + lane;
    const int ri = tl & 1, n = tl >> 1;
    const uint32_t lane_base = uint32_t(32 * quarter) << 16;
    int j = 0;
    bool ok = true;
    for (int e = 0; e < S && ok; ++e) {
      const TCStage& st = plan.st[e];
      const bool last = st.last != 0;
      uint8_t* dst = a.bufs + int64_t(e) * a.buf_stride;
      const int64_t blk = split_block_bytes(st.R8_out);
      const uint32_t half = uint32_t(st.R8_out) * 256u;
      // pair, split and store the 16 accumulator columns c0 .. c0 + 15 (output rows of
      // the group) held in v1 (D1) and v2 (D2)
      auto emit = [&](int g, int c0, const float* v1, const float* v2) {
        float y[kTcChunk];
#pragma unroll
        for (int q = 0; q < kTcChunk; ++q) {
          // Y_re = D1[2n] - D2[2n + 1] (ri = 0), Y_im = D2[2n] + D1[2n + 1] (ri = 1)
          const float pv = __shfl_xor_sync(0xffffffffu, v2[q], 1);
          y[q] = ri == 0 ? v1[q] - pv : v1[q] + pv;
        }
#pragma unroll
        for (int r8 = 0; r8 < kTcChunk / 8; ++r8) {
          const int m0 = c0 + 8 * r8;
          const int t = m0 / st.R8_out, k2 = m0 - t * st.R8_out;
          const int64_t P = pat_blk(st.out_pat, g, t, st, c);
          if (last) {
            float* o = a.y_out + (P * st.R_out + k2) * (2 * kTcNR) + ri * kTcNR + n;
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (k2 + i < st.R_out) o[i * 2 * kTcNR] = y[8 * r8 + i];
          } else if (TF32) {   // two runs of 4 rows: byte (k / 4) 2048 + (m / 8) 128 + (m % 8) 16
            uint8_t* o = dst + P * blk + (k2 >> 2) * 2048 + (tl >> 3) * 128 + (tl & 7) * 16;
            *reinterpret_cast<uint4*>(o) = tf32x4(y + 8 * r8);
            *reinterpret_cast<uint4*>(o + 2048) = tf32x4(y + 8 * r8 + 4);
          } else {
            uint4 hi, lo;
            split8(y + 8 * r8, hi, lo);
            uint8_t* o = dst + P * blk + (k2 >> 3) * 2048 + (tl >> 3) * 128 + (tl & 7) * 16;
            *reinterpret_cast<uint4*>(o) = hi;
            *reinterpret_cast<uint4*>(o + half) = lo;
          }
        }
      };
      for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x, ++j) {
        if (j % nsets != set) continue;
        const uint32_t du = uint32_t(j / nsets);
        // wait for the MMAs of this group (every lane observes the phase)
        if (!__all_sync(0xffffffffu, wait_bar(&dfull[set], du & 1u, abort))) {
          if (lane == 0 && !*abort) {
            atomicCAS(a.status, 0, ST_FULL_TIMEOUT);
            *abort = 1;
          }
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d1 = taddr + uint32_t(set) * set_cols + lane_base, d2 = d1 + uint32_t(st.M_t);
        // 32 columns of D1 and of D2 a round (M_t is a multiple of 32); the accumulator set
        // is released to the MMA warp as soon as its last columns are in registers
        for (int c0 = 0; c0 < st.M_t; c0 += 32) {
          float v1[32], v2[32];
          tmem_ld32(d1 + uint32_t(c0), v1);
          tmem_ld32(d2 + uint32_t(c0), v2);
          tmem_wait_ld();
          tmem_hold(v1, v2);
          if (c0 + 32 >= st.M_t) {
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&dempty[set]);
          }
          emit(g, c0, v1, v2);
          emit(g, c0 + kTcChunk, v1 + kTcChunk, v2 + kTcChunk);
        }
        // hand the written blocks to the signal warp (which counts them in for the next
        // stage off this set's path); first make sure it took the set's previous group,
        // so that the two never get a full phase apart
        if (du > 0 && !wait_bar(&signaled[set], (du - 1) & 1u, abort)) {
          if (!*abort) {
            atomicCAS(a.status, 0, ST_FULL_TIMEOUT);
            *abort = 1;
          }
        } else {
          mbar_arrive(&stored[set]);   // release: the set's stores before the signal warp's fence
        }
      }
    }
  } else if (warp == 12) {
    // ---------------------------------------------------------------- signal warp
    // For each group in order: wait until its epilogue set has stored the output
    // blocks, make them visible GPU-wide (fence) and count them in for the consumers.
    int j = 0;
    bool ok = true;
    for (int e = 0; e < S && ok; ++e) {
      const TCStage& st = plan.st[e];
      const bool last = st.last != 0;
      const TCStage& nst = plan.st[e + 1 < S ? e + 1 : e];
      unsigned* cnt_out = a.counters + int64_t(e + 1) * nst.n_groups;
      for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x, ++j) {
        const int set = j % nsets;
        const uint32_t du = uint32_t(j / nsets);
        if (!__all_sync(0xffffffffu, wait_bar(&stored[set], du & 1u, abort))) {
          if (lane == 0 && !*abort) {
            atomicCAS(a.status, 0, ST_FULL_TIMEOUT);
            *abort = 1;
          }
          ok = false;
          break;
        }
        if (!last && lane < c) {
          __threadfence();
          const int64_t P = pat_blk(st.out_pat, g, lane, st, c);
          atomicAdd(cnt_out + pat_group(nst.in_pat, P, nst, c), 1u);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&signaled[set]);
      }
    }
  }
  // teardown: all roles are done with TMEM
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr));
}

// ------------------------------------------------------------------ leaf kernels
// U^L: one CTA per group (its c leaves), the group's points staged kLeafPts at a time;
// (V^L)^*: one CTA per leaf, its points staged up to LeafArgs::pts_cap at a time.
constexpr int kLeafThreads = 256;
constexpr int kLeafPts = 64;        // points staged per round (= kTcNR)
constexpr int kLeafMaxR8 = 64;      // largest leaf rank (rounded up to 8) of the tensor path
constexpr int kLeafMaxC = 8;        // children per node (3-D)

// Entry e of line ci lpc + li (chunk ci, line li within it) of a chunked item (split
// real / imaginary planes per chunk).
__device__ __forceinline__ float2 item_entry_cl(const uint8_t* base, const Item& it, int ci, int li, int e) {
  const int nl = min(int(it.lpc), int(it.nlines) - ci * int(it.lpc));
  const float* re = reinterpret_cast<const float*>(base + int64_t(ci) * chunk_bytes(it.lpc, it.len));
  const int64_t q = int64_t(li) * it.len + e;
  return make_float2(__ldg(re + q), __ldg(re + pad4(int64_t(nl) * it.len) + q));
}

// Entry e of line `line` of a chunked item.
__device__ __forceinline__ float2 item_entry(const uint8_t* base, const Item& it, int line, int e) {
  const int ci = line / it.lpc;
  return item_entry_cl(base, it, ci, line - ci * it.lpc, e);
}

// Panel in tree order: gt[inv(i)][n] = g[rhs0 + n][i] for the natural Omega indices i
// (inv(i) < 0: not in the tree), zero for rhs0 + n >= nrhs.  A CTA moves kPermPts
// consecutive natural indices for the 64 RHS of the panel: rows of g are read as
// 16-byte runs, and each point's 64 values are written as one 512-byte row of gt.  In
// shared memory an entry (n, i) sits in float4 (n / 2, i) at half n % 2, so that a warp
// reads one point's row without bank conflicts.
constexpr int kPermPts = 128;
constexpr int kPermStride = kPermPts + 1;   // float4 per pair of RHS rows
__global__ void __launch_bounds__(kLeafThreads) permute_in_kernel(const __grid_constant__ LeafArgs a) {
  extern __shared__ __align__(16) float4 ptile[];      // [kTcNR / 2][kPermStride]
  __shared__ int ptp[kPermPts];                        // tree positions of the tile's points
  const int64_t i0 = int64_t(blockIdx.x) * kPermPts;
  const int tid = threadIdx.x;
  if (tid < kPermPts) ptp[tid] = i0 + tid < a.len_vec ? __ldg(a.perm + i0 + tid) : -1;
  // rows of g start 16-byte aligned: 16-byte loads
  const bool vec = (a.len_vec & 1) == 0 && (reinterpret_cast<uintptr_t>(a.vec) & 15) == 0;
  constexpr int Q4 = kPermPts / 2;                     // float4 per row of the tile
  constexpr int NQ = kTcNR * Q4 / kLeafThreads;       // float4 per thread (all loads first)
  float4 v[NQ];
#pragma unroll
  for (int u = 0; u < NQ; ++u) {
    const int q = tid + u * kLeafThreads, n = q / Q4, i2 = q - n * Q4, rhs = a.rhs0 + n;
    const int64_t i = i0 + 2 * i2;
    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (rhs < a.nrhs) {
      const float2* row = a.vec + int64_t(rhs) * a.len_vec;
      if (vec && i + 1 < a.len_vec) {
        v[u] = __ldg(reinterpret_cast<const float4*>(row + i));
      } else {
        if (i < a.len_vec) {
          const float2 x = __ldg(row + i);
          v[u].x = x.x;
          v[u].y = x.y;
        }
        if (i + 1 < a.len_vec) {
          const float2 x = __ldg(row + i + 1);
          v[u].z = x.x;
          v[u].w = x.y;
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < NQ; ++u) {
    const int q = tid + u * kLeafThreads, n = q / Q4, i2 = q - n * Q4;
    float2* t0 = reinterpret_cast<float2*>(ptile + (n >> 1) * kPermStride + 2 * i2) + (n & 1);
    t0[0] = make_float2(v[u].x, v[u].y);
    t0[2] = make_float2(v[u].z, v[u].w);
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll 4
  for (int ii = warp; ii < kPermPts; ii += kLeafThreads / 32) {
    const int tp = ptp[ii];
    if (tp >= 0)
      reinterpret_cast<float4*>(a.outp + int64_t(tp) * kTcNR)[lane] = ptile[lane * kPermStride + ii];
  }
}

// Rows k0 .. k0 + 7 of column n of split block `leaf` from 8 accumulators: byte
// (hl, k, ri, n) as in apply.hpp, so 8 consecutive k are one 16-byte run per plane.
template <bool TF32>
__device__ __forceinline__ void store_split8(uint8_t* outs, int64_t leaf, int R8, int n, int k0, float2 (&acc)[8]) {
  float re[8], im[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    re[j] = acc[j].x;
    im[j] = acc[j].y;
    acc[j] = make_float2(0.f, 0.f);
  }
  // rows m = 2 n (real part) and 2 n + 1 (imaginary part) of the block: adjacent 16-byte
  // rows of one core matrix
  const int m = 2 * n;
  if constexpr (TF32) {   // TF32 block: byte (k / 4) 2048 + (m / 8) 128 + (m % 8) 16 + (k % 4) 4
    uint8_t* o = outs + leaf * split_block_bytes(R8) + (k0 >> 2) * 2048 + (m >> 3) * 128 + (m & 7) * 16;
    *reinterpret_cast<uint4*>(o) = tc::tf32x4(re);
    *reinterpret_cast<uint4*>(o + 2048) = tc::tf32x4(re + 4);
    *reinterpret_cast<uint4*>(o + 16) = tc::tf32x4(im);
    *reinterpret_cast<uint4*>(o + 2048 + 16) = tc::tf32x4(im + 4);
  } else {
    uint4 rh, rl, ih, il;
    tc::split8(re, rh, rl);
    tc::split8(im, ih, il);
    uint8_t* o = outs + leaf * split_block_bytes(R8) + (k0 >> 3) * 2048 + (m >> 3) * 128 + (m & 7) * 16;
    const int64_t half = int64_t(R8) * 256;
    *reinterpret_cast<uint4*>(o) = rh;               // Re hi
    *reinterpret_cast<uint4*>(o + 16) = ih;          // Im hi
    *reinterpret_cast<uint4*>(o + half) = rl;        // Re lo
    *reinterpret_cast<uint4*>(o + half + 16) = il;   // Im lo
  }
}

// (V^L)^* for a panel of 64 RHS, one CTA of 64 R8 / 8 threads per leaf j (of group
// g = j / c):
//   y_j[k][n] = sum over the points b of leaf j of conj(V^L_j[b][k]) gt[b][n],
// gt = the panel in tree order (permute_in_kernel), stored as split block j (rows k >= R
// are zero).  The group's item holds conj(V) with line = point (tree order from the
// group's first point), entry = k.  Up to a.pts_cap points at a time, the leaf's panel
// rows (contiguous, 512 bytes each) are copied into shared memory by 16-byte cp.async
// while its item entries are loaded, every load of the round in flight at once; then
// thread (n, kg) accumulates rows 8 kg .. 8 kg + 7 of column n from shared memory only.
// One CTA per leaf bounds a CTA's work by the largest leaf, not the largest group (a
// ragged tree puts several times the mean number of points into some groups).  The
// panel rows are read by this CTA alone and never again: their L2 lines are discarded
// rather than written back.  With `gather` the rows come straight from g in natural
// order through the leaf's table of natural indices instead (no panel, no permute
// kernel; the table, unlike the tree permutation, needs no offset load first): device
// buffers take this route; page-locked host buffers keep the panel, read row by row.
// Empty leaves give zero blocks.
__device__ __forceinline__ void leaf_v_point(float2 (&acc)[8], const float2* vrow, float2 x) {
  const float4* vp = reinterpret_cast<const float4*>(vrow);
#pragma unroll
  for (int j2 = 0; j2 < 4; ++j2) {
    const float4 v = vp[j2];
    acc[2 * j2].x = fmaf(v.x, x.x, fmaf(-v.y, x.y, acc[2 * j2].x));
    acc[2 * j2].y = fmaf(v.x, x.y, fmaf(v.y, x.x, acc[2 * j2].y));
    acc[2 * j2 + 1].x = fmaf(v.z, x.x, fmaf(-v.w, x.y, acc[2 * j2 + 1].x));
    acc[2 * j2 + 1].y = fmaf(v.z, x.y, fmaf(v.w, x.x, acc[2 * j2 + 1].y));
  }
}

// XPOSE (the adjoint's U^* leaf products): the group's item is a U^L item (line = k,
// entry = point of the group, U itself), read transposed and conjugated.
template <bool TF32, bool XPOSE>
__global__ void __launch_bounds__(kTcNR * kLeafMaxR8 / 8) leaf_v_kernel(const __grid_constant__ LeafArgs a) {
  using tc::sa;
  using tc::cp_async16;
  using tc::cp_async_wait_all;
  using tc::l2_discard;
  constexpr int NR = kTcNR;
  extern __shared__ __align__(16) float2 lsm[];
  __shared__ int nat[kLeafPts];            // gather: natural indices of the round's points
  const int j = blockIdx.x, c = a.c, g = j / c, R = a.R, R8 = a.R8, cap = a.pts_cap;
  const int tid = threadIdx.x, nth = int(blockDim.x), n = tid % NR, k0 = 8 * (tid / NR);
  // a gathered row is written one RHS per thread: padded to NR + 1 entries against bank conflicts
  const int xstride = a.gather ? NR + 1 : NR;
  float2* xs = lsm;                        // [cap][xstride]: the round's panel rows
  float2* vs = lsm + cap * xstride;        // [cap][R8]: conj V, zero for k >= R
  // first-level loads, all independent of one another: the leaf's offsets, its group's
  // item and (gather) the natural indices of its first round's points
  const int pg = __ldg(a.off + c * g), p0 = __ldg(a.off + j), p1 = __ldg(a.off + j + 1);
  const Item it = a.items[a.item_base + int64_t(g) * a.item_stride];
  const int32_t* natj = a.nat + int64_t(j) * a.nat_stride;
  const int nat0 = (a.gather && tid < cap) ? __ldg(natj + tid) : 0;
  const int np = p1 - p0;
  float2 acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = make_float2(0.f, 0.f);
  if (np > 0) {
    const uint8_t* ibase = a.arena + size_t(it.off128) * 128;
    const int kq = tid % R8, bq = tid / R8, bstep = nth / R8;   // entry k = kq of points bq + bstep u
    for (int b0 = 0; b0 < np; b0 += cap) {
      const int nb = min(cap, np - b0);
      if (b0 > 0) __syncthreads();         // previous round's shared reads done
      const float2* src = a.vec + int64_t(p0 + b0) * NR;
      if (a.gather) {
        // the round's points straight from g in natural order: thread q reads RHS
        // q / nb of point q % nb, so that a warp's loads fall on a few nearby rows
        for (int q = tid; q < nb; q += nth) nat[q] = b0 == 0 ? nat0 : __ldg(natj + b0 + q);
        __syncthreads();
        // (nn, b) = divmod(q, nb) for q = tid, tid + nth, ...: advanced by divmod(nth, nb)
        // with one carry (b + db < 2 nb), two divisions per thread and round
        const int total = nb * NR, dn = nth / nb, db = nth - dn * nb;
        int nn = tid / nb;
        int bb = tid - nn * nb;
        for (int q0 = tid; q0 < total; q0 += 4 * nth) {          // 4 loads in flight per thread
          float2 v[4];
          int bs[4], ns[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * nth, rhs = a.rhs0 + nn;
            ns[u] = nn;
            bs[u] = bb;
            v[u] = (q < total && rhs < a.nrhs)
                       ? __ldg((a.use_rows ? a.rows.in[rhs] : a.vec + int64_t(rhs) * a.len_vec) + nat[bb])
                       : make_float2(0.f, 0.f);
            nn += dn;
            bb += db;
            if (bb >= nb) {
              bb -= nb;
              ++nn;
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (q0 + u * nth < total) xs[bs[u] * xstride + ns[u]] = v[u];
        }
      } else {
        for (int q = tid; q < nb * (NR / 2); q += nth) cp_async16(sa(xs) + uint32_t(q) * 16u, src + 2 * q);
      }
      const int lpc = it.lpc;
      for (int b1 = bq; b1 < nb; b1 += 8 * bstep) {             // 8 loads in flight per thread
        float2 v[8];
        // forward: line pt of the item, as (chunk, line in chunk), advanced by bstep per u
        int ci = 0, li = 0;
        if (!XPOSE) {
          const int line = p0 - pg + b0 + b1;
          ci = line / lpc;
          li = line - ci * lpc;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int b = b1 + u * bstep, pt = p0 - pg + b0 + b;
          v[u] = make_float2(0.f, 0.f);
          if (b < nb && kq < R) {
            if (XPOSE) {
              const float2 e = item_entry(ibase, it, kq, pt);
              v[u] = make_float2(e.x, -e.y);
            } else {
              v[u] = item_entry_cl(ibase, it, ci, li, kq);
            }
          }
          if (!XPOSE) {
            li += bstep;
            while (li >= lpc) {
              li -= lpc;
              ++ci;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (b1 + u * bstep < nb) vs[(b1 + u * bstep) * R8 + kq] = v[u];
      }
      cp_async_wait_all();
      __syncthreads();
      if (!a.gather) {   // the panel rows are read by this CTA alone and never again
        const char* lines = reinterpret_cast<const char*>(src);
        for (int q = tid; q < nb * (NR * int(sizeof(float2)) / 128); q += nth) l2_discard(lines + 128 * q);
      }
#pragma unroll 4
      for (int b = 0; b < nb; ++b) leaf_v_point(acc, vs + b * R8 + k0, xs[b * xstride + n]);
    }
  }
  store_split8<TF32>(a.outs, j, R8, n, k0, acc);
}

// U^L for a panel, one CTA per group g (leaves i = c g + t) or, with leaf_split, one
// CTA per leaf:
//   u[rhs0 + n][x_perm(b)] (+)= sum_k U^L_i[b][k] w[i R + k][n]
// for the points b of leaf i.  The group's item is stored by columns (line = k, entry =
// point of the group); the coefficient rows of the CTA's leaves (R contiguous rows of
// 64 real then 64 imaginary parts per leaf) are staged whole in shared memory.  Thread
// (b, nq) computes point b of the round for the 16 RHS n = 16 nq + 0..15, so that a
// warp stores 32 consecutive points of one RHS row.  One CTA per leaf bounds a CTA's
// work by the largest leaf when a ragged tree puts several times the mean number of
// points into some groups.
// XPOSE (the adjoint's V^L leaf products): the group's item is a (V^L)^* item (line =
// point, entry = k, conj V), read transposed and conjugated.
template <bool XPOSE>
__global__ void __launch_bounds__(kLeafThreads) leaf_u_kernel(const __grid_constant__ LeafArgs a) {
  constexpr int NR = kTcNR, NQ = kLeafThreads / kLeafPts, MN = NR / NQ;
  extern __shared__ __align__(16) float2 lsm[];
  __shared__ int lend[kLeafMaxC + 1];
  const int c = a.c, R = a.R;
  const int g = a.leaf_split ? int(blockIdx.x) / c : int(blockIdx.x);
  const int t0 = a.leaf_split ? int(blockIdx.x) - g * c : 0, nl = a.leaf_split ? 1 : c;   // leaves t0 .. t0 + nl - 1
  const int tid = threadIdx.x;
  const int pg = a.off[c * g];
  const int pb = a.off[c * g + t0] - pg, np = a.off[c * g + t0 + nl] - pg - pb;   // points, group-relative
  if (np == 0) return;
  if (tid <= c) lend[tid] = a.off[c * g + tid] - pg;
  const Item it = a.items[a.item_base + int64_t(g) * a.item_stride];
  const uint8_t* ibase = a.arena + size_t(it.off128) * 128;
  float* ws = reinterpret_cast<float*>(lsm);                        // [nl R][2 NR]
  float2* us = reinterpret_cast<float2*>(ws + size_t(nl) * R * 2 * NR);   // [R][kLeafPts]
  const float* rows_g = a.wl + (int64_t(c) * g + t0) * R * 2 * NR;     // the CTA's leaves' rows
  {
    const float4* src = reinterpret_cast<const float4*>(rows_g);
    float4* dst = reinterpret_cast<float4*>(ws);
    const int nq4 = nl * R * (2 * NR / 4);
    for (int q0 = tid; q0 < nq4; q0 += 8 * kLeafThreads) {      // 8 loads in flight per thread
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (q0 + u * kLeafThreads < nq4) v[u] = __ldcg(src + q0 + u * kLeafThreads);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (q0 + u * kLeafThreads < nq4) dst[q0 + u * kLeafThreads] = v[u];
    }
  }
  const int bb = tid % kLeafPts, nq = tid / kLeafPts;
  __syncthreads();
  {   // the rows are read by this CTA alone and never again: drop them from L2
    using tc::l2_discard;
    const char* rows = reinterpret_cast<const char*>(rows_g);
    for (int q = tid; q < nl * R * (2 * NR * int(sizeof(float)) / 128); q += kLeafThreads) l2_discard(rows + 128 * q);
  }
  for (int b0 = 0; b0 < np; b0 += kLeafPts) {
    const int nb = min(kLeafPts, np - b0);
    if (b0 > 0) __syncthreads();
    for (int q0 = tid; q0 < R * nb; q0 += 8 * kLeafThreads) {   // 8 loads in flight per thread
      float2 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * kLeafThreads, k = q / nb, b = q - k * nb;
        if (q < R * nb) {
          if (XPOSE) {
            const float2 e = item_entry(ibase, it, pb + b0 + b, k);
            v[u] = make_float2(e.x, -e.y);
          } else {
            v[u] = item_entry(ibase, it, k, pb + b0 + b);
          }
        } else {
          v[u] = make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * kLeafThreads, k = q / nb, b = q - k * nb;
        if (q < R * nb) us[k * kLeafPts + b] = v[u];
      }
    }
    __syncthreads();
    if (bb < nb) {
      const int p = pb + b0 + bb;                 // group-relative point
      int t = t0;
      while (t + 1 < t0 + nl && p >= lend[t + 1]) ++t;
      const float* wr = ws + size_t(t - t0) * R * 2 * NR + MN * nq;
      float2 acc[MN];
#pragma unroll
      for (int j = 0; j < MN; ++j) acc[j] = make_float2(0.f, 0.f);
      for (int k = 0; k < R; ++k) {
        const float2 uv = us[k * kLeafPts + bb];
        const float* wk = wr + k * 2 * NR;
#pragma unroll
        for (int j4 = 0; j4 < MN / 4; ++j4) {
          const float4 wre = *reinterpret_cast<const float4*>(wk + 4 * j4);
          const float4 wim = *reinterpret_cast<const float4*>(wk + NR + 4 * j4);
          const float re[4] = {wre.x, wre.y, wre.z, wre.w}, im[4] = {wim.x, wim.y, wim.z, wim.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float2& o = acc[4 * j4 + j];
            o.x = fmaf(uv.x, re[j], fmaf(-uv.y, im[j], o.x));
            o.y = fmaf(uv.x, im[j], fmaf(uv.y, re[j], o.y));
          }
        }
      }
      const int nat = __ldg(a.perm + pg + p);
#pragma unroll
      for (int j = 0; j < MN; ++j) {
        const int rhs = a.rhs0 + MN * nq + j;
        if (rhs < a.nrhs) {
          float2* o = (a.use_rows ? a.rows.out[rhs] : a.outp + int64_t(rhs) * a.len_out) + nat;
          float2 v = acc[j];
          if (a.accumulate) {
            const float2 w = *o;
            v.x += w.x;
            v.y += w.y;
          }
          *o = v;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ host side

size_t tc_smem_bytes(int nsa, int nxb, int nsets, int mt_max, int kpad_max) {
  (void)nsets;
  return size_t(nsa) * 4 * size_t(mt_max) * 32 + size_t(nxb) * 2 * size_t(kpad_max) * 256 +
         (2 * size_t(nsa) + 20) * 8 + 64;
}

size_t leaf_smem_bytes(int R, int c, bool u_side, int pts_cap) {
  const int R8 = (R + 7) & ~7;
  return u_side ? size_t(c) * R * 2 * kTcNR * sizeof(float) + size_t(R) * kLeafPts * sizeof(float2)
                : sizeof(float2) * size_t(pts_cap) * (kTcNR + 1 + R8);
}

int leaf_pts_cap(int64_t max_leaf_points) {
  const int64_t r8 = (max_leaf_points + 7) & ~int64_t(7);
  return int(std::min<int64_t>(kLeafPts, std::max<int64_t>(8, r8)));
}

bool leaf_fits(int R8, int c) { return R8 <= kLeafMaxR8 && c <= kLeafMaxC; }

cudaError_t launch_apply_tc(const TCArgs& a, int grid, size_t smem, cudaStream_t stream, bool tf32) {
  if (a.nsa < kAProducers || a.nsa % kAProducers != 0) return cudaErrorInvalidValue;
  if (a.nxb < 1 || a.nxb > kMaxXBufs) return cudaErrorInvalidValue;
  cudaError_t err = cudaSuccess;   // (the caller clears the dependency counters)
  void (*kern)(TCArgs) = tf32 ? bf_apply_tc<true> : bf_apply_tc<false>;
  if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess)
    return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kTcThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// TF32 tiles from the split-BF16 tiles: T = hi + lo (FP32), rounded to TF32, in the
// TF32 chunk layout (planes Re, Im; byte ((m / 8) 4 + k / 4) 128 + (m % 8) 16 + (k % 4) 4).
// One CTA per K16 chunk of a tile, one thread per entry of the chunk's M_t x 16 block.
__global__ void __launch_bounds__(256) tf32_tiles_kernel(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst,
                                                        int64_t n_chunks, int M_t) {
  const int64_t chunk = blockIdx.x;
  if (chunk >= n_chunks) return;
  const int64_t cb = int64_t(M_t) * 128;   // bytes of one chunk (both layouts)
  const uint32_t pb = uint32_t(M_t) * 32, pbt = uint32_t(M_t) * 64;
  const uint8_t* s0 = src + chunk * cb;
  uint8_t* d0 = dst + chunk * cb;
  for (int q = threadIdx.x; q < M_t * 16; q += blockDim.x) {
    const int m = q >> 4, k = q & 15;
    const uint32_t sb = uint32_t(((m >> 3) * 2 + (k >> 3)) * 128 + (m & 7) * 16 + (k & 7) * 2);
    const auto bf = [&](uint32_t off) {
      return __uint_as_float(uint32_t(*reinterpret_cast<const uint16_t*>(s0 + off)) << 16);
    };
    const float re = bf(sb) + bf(2 * pb + sb), im = bf(pb + sb) + bf(3 * pb + sb);   // hi + lo
    const uint32_t db = uint32_t(((m >> 3) * 4 + (k >> 2)) * 128 + (m & 7) * 16 + (k & 3) * 4);
    *reinterpret_cast<float*>(d0 + db) = tc::to_tf32(re);
    *reinterpret_cast<float*>(d0 + pbt + db) = tc::to_tf32(im);
  }
}

// Adjoint tiles from the forward split-BF16 tiles of one stage: tile T (M_t x K_t,
// chunks along K) -> T^H (K_t x M_t, chunks along M_t): entry (i, k) of T^H is
// conj(T[k][i]); Im planes change sign (hi and lo).  One CTA per K16 chunk of the
// adjoint tile (n_groups x M_t / 16), one thread per entry.
__global__ void __launch_bounds__(256) adjoint_tiles_kernel(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst,
                                                           int64_t n_chunks, int M_t, int K_t) {
  const int64_t chunk = blockIdx.x;
  if (chunk >= n_chunks) return;
  const int nka = M_t / 16;                    // adjoint chunks per tile
  const int64_t g = chunk / nka;
  const int kka = int(chunk - g * nka);
  const int64_t tile = int64_t(M_t) * K_t * 8;
  const uint32_t pbf = uint32_t(M_t) * 32, pba = uint32_t(K_t) * 32;   // plane bytes of a chunk
  const uint8_t* t0 = src + g * tile;
  uint8_t* a0 = dst + g * tile + int64_t(kka) * 4 * pba;
  for (int q = threadIdx.x; q < K_t * 16; q += blockDim.x) {
    const int i = q >> 4, kc = q & 15;          // adjoint row i (= forward column), K kc
    const int m = 16 * kka + kc, k = i;         // forward row m, column k
    const uint8_t* fc = t0 + int64_t(k >> 4) * 4 * pbf;
    const uint32_t fo = uint32_t(((m >> 3) * 2 + ((k & 15) >> 3)) * 128 + (m & 7) * 16 + (k & 7) * 2);
    const uint32_t ao = uint32_t(((i >> 3) * 2 + (kc >> 3)) * 128 + (i & 7) * 16 + (kc & 7) * 2);
#pragma unroll
    for (int pl = 0; pl < 4; ++pl) {            // planes Re hi, Im hi, Re lo, Im lo
      uint16_t v = *reinterpret_cast<const uint16_t*>(fc + pl * pbf + fo);
      if (pl & 1) v ^= 0x8000u;                 // conj
      *reinterpret_cast<uint16_t*>(a0 + pl * pba + ao) = v;
    }
  }
}

cudaError_t launch_adjoint_tiles(const uint8_t* src, uint8_t* dst, int n_groups, int M_t, int K_t, cudaStream_t stream) {
  const int64_t n_chunks = int64_t(n_groups) * (M_t / 16);
  if (n_chunks <= 0) return cudaSuccess;
  adjoint_tiles_kernel<<<unsigned(n_chunks), 256, 0, stream>>>(src, dst, n_chunks, M_t, K_t);
  return cudaGetLastError();
}

cudaError_t launch_tf32_tiles(const uint8_t* src, uint8_t* dst, int64_t n_chunks, int M_t, cudaStream_t stream) {
  if (n_chunks <= 0) return cudaSuccess;
  tf32_tiles_kernel<<<unsigned(n_chunks), 256, 0, stream>>>(src, dst, n_chunks, M_t);
  return cudaGetLastError();
}

size_t tc_counter_bytes(const TCPlan& plan) {
  size_t n = 0;
  for (int e = 0; e < plan.n_stages; ++e) n += size_t(plan.st[e].n_groups);
  return (n * sizeof(unsigned) + 255) & ~size_t(255);
}

cudaError_t launch_permute_in(const LeafArgs& a, cudaStream_t stream) {
  const size_t smem = sizeof(float4) * (kTcNR / 2) * kPermStride;
  cudaError_t err = cudaFuncSetAttribute(permute_in_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (err != cudaSuccess) return err;
  permute_in_kernel<<<unsigned((a.len_vec + kPermPts - 1) / kPermPts), kLeafThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_leaf(const LeafArgs& a, bool u_side, int n_groups, cudaStream_t stream, bool tf32, bool xpose) {
  const size_t smem = u_side ? leaf_smem_bytes(a.R, a.leaf_split ? 1 : a.c, true)
                             : sizeof(float2) * size_t(a.pts_cap) * (kTcNR + (a.gather ? 1 : 0) + a.R8);
  void (*kern)(LeafArgs) =
      u_side ? (xpose ? leaf_u_kernel<true> : leaf_u_kernel<false>)
             : (tf32 ? (xpose ? leaf_v_kernel<true, true> : leaf_v_kernel<true, false>)
                     : (xpose ? leaf_v_kernel<false, true> : leaf_v_kernel<false, false>));
  // U^L: a CTA per group; (V^L)^*: a CTA per leaf, one thread per RHS column and group of 8 rows
  const int threads = u_side ? kLeafThreads : kTcNR * (a.R8 / 8);
  const int64_t blocks = (u_side && !a.leaf_split) ? int64_t(n_groups) : int64_t(n_groups) * a.c;
  if (!u_side && (a.pts_cap < 8 || a.pts_cap > kLeafPts || a.pts_cap % 8 != 0)) return cudaErrorInvalidValue;
  if (blocks <= 0) return cudaSuccess;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (err != cudaSuccess) return err;
  kern<<<unsigned(blocks), threads, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace mbf
