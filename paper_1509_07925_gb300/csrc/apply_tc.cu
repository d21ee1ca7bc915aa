// Tensor-core apply of a butterfly factorization for panels of many right-hand
// sides (sm_103a: tcgen05 MMAs, TMEM accumulators, cp.async.bulk staging).
//
// Every group product of a G^l / (H^l)^* level, Y = T X with T complex (M_t x K_t) and X
// complex (K_t x NR), becomes real MMAs on split-BF16 planes (T = T_hi + T_lo, X = X_hi +
// X_lo, products hi*hi + hi*lo + lo*hi accumulated in FP32):
//     Y_re = T_re X_re - T_im X_im,     Y_im = T_im X_re + T_re X_im.
// T is the MMA's A operand (M = 128 rows per block), the panel X the B operand
// (N = NR), both K-major without swizzle; K advances 16 per MMA.
//
// Warp roles in a CTA (one per SM, persistent, cooperative):
//   warp 0     one lane streams each group's tile, chunk by chunk (K = 16 columns,
//              4 planes), into a ring of shared-memory slots (full/empty mbarriers);
//   warp 1     allocates TMEM; one lane issues the MMAs into one of two accumulator
//              buffers and commits completions to the mbarriers;
//   warps 4-7, 8-11   two epilogue sets, alternating groups: wait for the group's
//              inputs (dependency counters), gather and split the RHS panel into the
//              B buffer, wait for the MMAs, read the accumulators (tcgen05.ld) and
//              store the group's outputs, then count them in for the consumers.
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

// 32 consecutive TMEM columns of this thread's lane (one row of the accumulator).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ int64_t pat_off(int pat, int g, int t, const TCStage& s, int R, int c) {
  const int a = g / s.B, b = g - (g / s.B) * s.B;
  if (pat == PAT_SPLIT) return (int64_t(c * a + t) * s.B + b) * R;
  if (pat == PAT_CONTIG) return (int64_t(c) * g + t) * R;
  return (int64_t(c * b + t) * s.ch + a) * R;  // PAT_CORNER
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

constexpr int kTcThreads = 384;

__global__ void __launch_bounds__(kTcThreads, 1) bf_apply_tc(const __grid_constant__ TCArgs a) {
  using namespace tc;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int NR = a.NR, nsa = a.nsa;
  const uint32_t a_plane = uint32_t(a.mpad) * 32u;          // bytes of one A plane (mpad rows x 16 cols)
  const uint32_t a_slot = 4u * a_plane;
  const uint32_t b_buf = 4u * uint32_t(NR) * uint32_t(a.kpad_max) * 2u;
  uint8_t* aring = smem;
  uint8_t* bbuf = smem + size_t(nsa) * a_slot;
  uint64_t* afull = reinterpret_cast<uint64_t*>(bbuf + 2 * size_t(b_buf));
  uint64_t* aempty = afull + nsa;
  uint64_t* bfull = aempty + nsa;
  uint64_t* bempty = bfull + 2;
  uint64_t* dfull = bempty + 2;
  uint64_t* dempty = dfull + 2;
  uint64_t* done = dempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < nsa; ++i) {
      mbar_init(&afull[i], 1);
      mbar_init(&aempty[i], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bfull[s], 128);
      mbar_init(&bempty[s], 1);
      mbar_init(&dfull[s], 1);
      mbar_init(&dempty[s], 128);
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
  // accumulator set s (2 x MB blocks of NR columns) starts at column s * set_cols
  int mb_max = 1;
  for (int e = 0; e < S; ++e) mb_max = max(mb_max, plan.st[e].MB);
  const uint32_t set_cols = uint32_t(mb_max * 2 * NR);

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- producer
    uint32_t ca = 0;
    bool ok = true;
    for (int e = 0; e < S && ok; ++e) {
      const TCStage& st = plan.st[e];
      const int nk = st.K_pad / 16;
      for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x) {
        const uint8_t* src = a.arena + st.base + int64_t(g) * st.tile_bytes;
        for (int kk = 0; kk < nk; ++kk, ++ca) {
          const uint32_t slot = ca % uint32_t(nsa), ph = (ca / uint32_t(nsa)) & 1u;
          if (!wait_bar(&aempty[slot], ph ^ 1u, abort)) {
            if (!*abort) {
              atomicCAS(a.status, 0, ST_EMPTY_TIMEOUT);
              *abort = 1;
            }
            ok = false;
            break;
          }
          mbar_expect_tx(&afull[slot], 4u * uint32_t(st.plane_bytes));
          for (int p = 0; p < 4; ++p)
            bulk_g2s(aring + size_t(slot) * a_slot + size_t(p) * a_plane,
                     src + (int64_t(kk) * 4 + p) * st.plane_bytes, uint32_t(st.plane_bytes), &afull[slot]);
        }
      }
    }
    // wait (bounded) for every copy still in flight
    for (uint32_t q = (ca > uint32_t(nsa) ? ca - uint32_t(nsa) : 0u); q < ca; ++q) {
      const uint32_t slot = q % uint32_t(nsa), ph = (q / uint32_t(nsa)) & 1u;
      const uint64_t t1 = gtimer();
      while (!mbar_try(&afull[slot], ph) && gtimer() - t1 < kTimeoutNs) {
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    uint32_t ca = 0;
    int j = 0;
    bool ok = true;
    const uint32_t abase = sa(aring), bbase0 = sa(bbuf);
    for (int e = 0; e < S && ok; ++e) {
      const TCStage& st = plan.st[e];
      const int nk = st.K_pad / 16;
      const uint32_t bplane = uint32_t(NR) * uint32_t(st.K_pad) * 2u;
      const uint32_t sbo_b = uint32_t(st.K_pad) * 16u;
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(NR >> 3) << 17) | (uint32_t(128 >> 4) << 24);
      for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x, ++j) {
        const int s = j & 1;
        const uint32_t u = uint32_t(j >> 1);
        if (!wait_bar(&bfull[s], u & 1u, abort) || !wait_bar(&dempty[s], (u & 1u) ^ 1u, abort)) {
          if (!*abort) {
            atomicCAS(a.status, 0, ST_FULL_TIMEOUT);
            *abort = 1;
          }
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dcol = taddr + uint32_t(s) * set_cols;
        const uint32_t bb = bbase0 + uint32_t(s) * b_buf;
        for (int kk = 0; kk < nk; ++kk, ++ca) {
          const uint32_t slot = ca % uint32_t(nsa), ph = (ca / uint32_t(nsa)) & 1u;
          if (!wait_bar(&afull[slot], ph, abort)) {
            if (!*abort) {
              atomicCAS(a.status, 0, ST_FULL_TIMEOUT);
              *abort = 1;
            }
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t as = abase + slot * a_slot;
          for (int mb = 0; mb < st.MB; ++mb) {
            // A planes: 0 Re hi, 1 Re lo, 2 Im hi, 3 Im lo; B planes: 0 Xre hi, 1 Xre lo, 2 Xim hi, 3 Xim lo
            auto A = [&](int p) { return sdesc(as + uint32_t(p) * a_plane + uint32_t(mb) * 4096u, 128u, 256u); };
            auto Bd = [&](int p) { return sdesc(bb + uint32_t(p) * bplane + uint32_t(kk) * 256u, 128u, sbo_b); };
            const uint32_t dre = dcol + uint32_t((mb * 2 + 0) * NR), dim = dcol + uint32_t((mb * 2 + 1) * NR);
            const uint32_t acc0 = kk > 0 ? 1u : 0u;
            const uint32_t neg = idesc | (1u << 13);
            // Re: T_re X_re - T_im X_im
            mma_bf16(dre, A(0), Bd(0), idesc, acc0);
            mma_bf16(dre, A(0), Bd(1), idesc, 1u);
            mma_bf16(dre, A(1), Bd(0), idesc, 1u);
            mma_bf16(dre, A(2), Bd(2), neg, 1u);
            mma_bf16(dre, A(2), Bd(3), neg, 1u);
            mma_bf16(dre, A(3), Bd(2), neg, 1u);
            // Im: T_im X_re + T_re X_im
            mma_bf16(dim, A(2), Bd(0), idesc, acc0);
            mma_bf16(dim, A(2), Bd(1), idesc, 1u);
            mma_bf16(dim, A(3), Bd(0), idesc, 1u);
            mma_bf16(dim, A(0), Bd(2), idesc, 1u);
            mma_bf16(dim, A(0), Bd(3), idesc, 1u);
            mma_bf16(dim, A(1), Bd(2), idesc, 1u);
          }
          mma_commit(&aempty[slot]);
        }
        if (!ok) break;
        mma_commit(&dfull[s]);
        mma_commit(&bempty[s]);
      }
    }
    // every MMA this thread issued has completed before TMEM is freed
    mma_commit(done);
    const uint64_t t1 = gtimer();
    while (!mbar_try(done, 0) && gtimer() - t1 < kTimeoutNs) {
    }
  } else if (warp >= 4) {
    // ---------------------------------------------------------------- epilogue sets
    const int set = (warp - 4) >> 2;            // 0: warps 4-7, 1: warps 8-11
    const int et = (warp - 4 - 4 * set) * 32 + lane;   // 0..127
    const int quarter = warp & 3;                // TMEM lane quarter this warp may access
    const int bar_id = 1 + set;
    const uint32_t lane_base = uint32_t(32 * quarter) << 16;
    int j = 0;
    bool ok = true;
    for (int e = 0; e < S && ok; ++e) {
      const TCStage& st = plan.st[e];
      const float2* src = e == 0 ? a.x_in : a.bufs + int64_t(e - 1) * a.buf_stride;
      float2* dst = a.bufs + int64_t(e) * a.buf_stride;
      const bool notify = e + 1 < S;
      const TCStage& nst = plan.st[e + 1 < S ? e + 1 : e];
      unsigned* cnt_in = a.counters + int64_t(e) * st.n_groups;
      unsigned* cnt_out = a.counters + int64_t(e + 1) * nst.n_groups;
      const uint32_t bplane = uint32_t(NR) * uint32_t(st.K_pad) * 2u;
      const uint32_t sbo_b = uint32_t(st.K_pad) * 16u;
      for (int g = blockIdx.x; g < st.n_groups && ok; g += gridDim.x, ++j) {
        if ((j & 1) != set) continue;
        const uint32_t u = uint32_t(j >> 1);
        uint8_t* bb = bbuf + size_t(set) * b_buf;
        // (1) the B buffer is free once the MMAs of this set's previous group are done
        int fail = 0;
        if (et == 0) {
          if (!wait_bar(&bempty[set], (u & 1u) ^ 1u, abort)) fail = 1;
          // (2) all c input segments written by the previous stage
          if (!fail && e > 0) {
            const unsigned* cp = cnt_in + g;
            const uint64_t t0 = gtimer();
            while (ld_acquire(cp) < unsigned(c)) {
              if (*abort || *reinterpret_cast<volatile int*>(a.status) != 0) { fail = 1; break; }
              if (gtimer() - t0 > kTimeoutNs) {
                atomicCAS(a.status, 0, ST_DEP_TIMEOUT);
                fail = 1;
                break;
              }
              __nanosleep(32);
            }
          }
          if (fail) *abort = 1;
        }
        if (named_sync_or(bar_id, 128, *abort != 0)) {
          ok = false;
          break;
        }
        // (3) gather the panel and split it into bf16 hi/lo planes (K-major core matrices)
        {
          const int nkb = st.K_pad / 8;
          for (int item = et; item < nkb * NR; item += 128) {
            const int kb = item / NR, n = item - (item / NR) * NR;
            uint32_t w[4][4];
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
              float2 v[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int k = kb * 8 + i + h;
                if (k < st.K_t) {
                  const int t = k / st.R_in, kk = k - t * st.R_in;
                  const int64_t pos = pat_off(st.in_pat, g, t, st, st.R_in, c) + kk;
                  v[h] = __ldcg(src + pos * NR + n);
                } else {
                  v[h] = make_float2(0.f, 0.f);
                }
              }
              uint16_t hr[2], lr[2], hi[2], li[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                hr[h] = bf16_bits(v[h].x);
                lr[h] = bf16_bits(v[h].x - __bfloat162float(__ushort_as_bfloat16(hr[h])));
                hi[h] = bf16_bits(v[h].y);
                li[h] = bf16_bits(v[h].y - __bfloat162float(__ushort_as_bfloat16(hi[h])));
              }
              w[0][i / 2] = uint32_t(hr[0]) | (uint32_t(hr[1]) << 16);
              w[1][i / 2] = uint32_t(lr[0]) | (uint32_t(lr[1]) << 16);
              w[2][i / 2] = uint32_t(hi[0]) | (uint32_t(hi[1]) << 16);
              w[3][i / 2] = uint32_t(li[0]) | (uint32_t(li[1]) << 16);
            }
            const uint32_t off = uint32_t(n >> 3) * sbo_b + uint32_t(kb) * 128u + uint32_t(n & 7) * 16u;
#pragma unroll
            for (int p = 0; p < 4; ++p)
              *reinterpret_cast<uint4*>(bb + size_t(p) * bplane + off) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&bfull[set]);
        // (4) wait for the MMAs of this group
        int got = 1;
        if (et == 0 && !wait_bar(&dfull[set], u & 1u, abort)) {
          got = 0;
          if (!*abort) {
            atomicCAS(a.status, 0, ST_FULL_TIMEOUT);
            *abort = 1;
          }
        }
        if (named_sync_or(bar_id, 128, !got || *abort != 0)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // (5) accumulators -> outputs; row = one output entry (t, k) of the group
        const uint32_t dcol = taddr + uint32_t(set) * set_cols;
        for (int mb = 0; mb < st.MB; ++mb) {
          const int row = mb * 128 + quarter * 32 + lane;
          const bool live = row < st.M_t;
          int64_t pos = 0;
          if (live) {
            const int t = row / st.R_out, kk = row - t * st.R_out;
            pos = pat_off(st.out_pat, g, t, st, st.R_out, c) + kk;
          }
          for (int c0 = 0; c0 < NR; c0 += 32) {
            float re[32], im[32];
            tmem_ld32(dcol + lane_base + uint32_t((mb * 2 + 0) * NR + c0), re);
            tmem_ld32(dcol + lane_base + uint32_t((mb * 2 + 1) * NR + c0), im);
            if (live) {
              float4* o = reinterpret_cast<float4*>(dst + pos * NR + c0);
#pragma unroll
              for (int q = 0; q < 16; ++q) o[q] = make_float4(re[2 * q], im[2 * q], re[2 * q + 1], im[2 * q + 1]);
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&dempty[set]);
        // (6) count the written segments in for the consumers of the next stage
        if (notify) {
          __threadfence();
          named_sync(bar_id, 128);
          if (et < c) {
            const int64_t P = pat_off(st.out_pat, g, et, st, st.R_out, c) / st.R_out;
            atomicAdd(cnt_out + pat_group(nst.in_pat, P, nst, c), 1u);
          }
        }
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
// (V^L_j)^* for a panel of NR RHS: one CTA per group of c Omega leaves.  The group's
// leaf item (lines = points, len = R_L, split planes per chunk) and the panel's input
// values are staged in shared memory; y[(c g + t) R + k][r] = sum over the points b of
// leaf t of conj(V^L_t[b][k]) g[r][perm(b)].
constexpr int kLeafThreads = 256;
constexpr int kLeafRhs = 16;   // RHS per sub-panel

__device__ __forceinline__ void stage_item(const LeafArgs& a, const Item& it, float* re_s, float* im_s) {
  // unpack the item's chunks into dense [line][len] real / imaginary arrays
  const uint8_t* base = a.arena + size_t(it.off128) * 128;
  for (int l0 = 0; l0 < it.nlines; l0 += it.lpc) {
    const int nl = min(int(it.lpc), int(it.nlines) - l0);
    const float* re = reinterpret_cast<const float*>(base);
    const float* im = re + pad4(int64_t(nl) * it.len);
    for (int q = threadIdx.x; q < nl * it.len; q += blockDim.x) {
      re_s[l0 * it.len + q] = __ldg(re + q);
      im_s[l0 * it.len + q] = __ldg(im + q);
    }
    base += chunk_bytes(nl, it.len);
  }
}

__global__ void __launch_bounds__(kLeafThreads) leaf_v_kernel(const __grid_constant__ LeafArgs a) {
  extern __shared__ __align__(16) float lsm[];
  const int g = blockIdx.x, c = a.c, R = a.R;
  const Item it = a.items[a.item_base + int64_t(g) * a.item_stride];
  const int p0 = a.off[c * g], npts = a.off[c * g + c] - p0;   // == it.nlines
  float* re_s = lsm;
  float* im_s = re_s + kMaxGroupPoints * R;
  float2* xs = reinterpret_cast<float2*>(im_s + kMaxGroupPoints * R);   // [point][kLeafRhs]
  int* bnd = reinterpret_cast<int*>(xs + kMaxGroupPoints * kLeafRhs);
  if (threadIdx.x <= c) bnd[threadIdx.x] = a.off[c * g + threadIdx.x] - p0;
  stage_item(a, it, re_s, im_s);
  for (int r0 = 0; r0 < a.NR; r0 += kLeafRhs) {
    __syncthreads();
    for (int q = threadIdx.x; q < npts * kLeafRhs; q += blockDim.x) {
      const int b = q / kLeafRhs, r = q - b * kLeafRhs;
      const int rhs = a.rhs0 + r0 + r;
      xs[q] = rhs < a.nrhs ? __ldg(a.vec + int64_t(rhs) * a.len_vec + a.perm[p0 + b]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < c * R * kLeafRhs; q += blockDim.x) {
      const int r = q % kLeafRhs, k = (q / kLeafRhs) % R, t = q / (kLeafRhs * R);
      float2 s = make_float2(0.f, 0.f);
      for (int b = bnd[t]; b < bnd[t + 1]; ++b) {
        const float ar = re_s[b * R + k], ai = im_s[b * R + k];   // stored conj(V)
        const float2 x = xs[b * kLeafRhs + r];
        s.x = fmaf(ar, x.x, fmaf(-ai, x.y, s.x));
        s.y = fmaf(ar, x.y, fmaf(ai, x.x, s.y));
      }
      a.outp[(int64_t(c * g + t) * R + k) * a.NR + r0 + r] = s;
    }
  }
}

// U^L for a panel: u[r][perm(a)] = sum_k U^L_t[a][k] w[(c g + t) R + k][r] for the points a
// of leaf t of group g (item stored by columns: line = k, entry = point).
__global__ void __launch_bounds__(kLeafThreads) leaf_u_kernel(const __grid_constant__ LeafArgs a) {
  extern __shared__ __align__(16) float lsm[];
  const int g = blockIdx.x, c = a.c, R = a.R;
  const Item it = a.items[a.item_base + int64_t(g) * a.item_stride];
  const int p0 = a.off[c * g], npts = a.off[c * g + c] - p0;
  float* re_s = lsm;                                         // [k][point]
  float* im_s = re_s + kMaxGroupPoints * R;
  float2* ws = reinterpret_cast<float2*>(im_s + kMaxGroupPoints * R);   // [c R][kLeafRhs]
  int* bnd = reinterpret_cast<int*>(ws + c * R * kLeafRhs);
  if (threadIdx.x <= c) bnd[threadIdx.x] = a.off[c * g + threadIdx.x] - p0;
  stage_item(a, it, re_s, im_s);
  const int len = it.len;   // = npts (at least 1)
  for (int r0 = 0; r0 < a.NR; r0 += kLeafRhs) {
    __syncthreads();
    for (int q = threadIdx.x; q < c * R * kLeafRhs; q += blockDim.x) {
      const int r = q % kLeafRhs, m = q / kLeafRhs;
      ws[q] = __ldcg(a.vec + (int64_t(c * g) * R + m) * a.NR + r0 + r);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < npts * kLeafRhs; q += blockDim.x) {
      const int r = q % kLeafRhs, pt = q / kLeafRhs;
      int t = 0;
      while (t + 1 < c && pt >= bnd[t + 1]) ++t;
      float2 s = make_float2(0.f, 0.f);
      for (int k = 0; k < R; ++k) {
        const float ar = re_s[k * len + pt], ai = im_s[k * len + pt];
        const float2 w = ws[(t * R + k) * kLeafRhs + r];
        s.x = fmaf(ar, w.x, fmaf(-ai, w.y, s.x));
        s.y = fmaf(ar, w.y, fmaf(ai, w.x, s.y));
      }
      const int rhs = a.rhs0 + r0 + r;
      if (rhs < a.nrhs) a.outp[int64_t(rhs) * a.len_out + a.perm[p0 + pt]] = s;
    }
  }
}

// ------------------------------------------------------------------ host side

size_t tc_smem_bytes(int nsa, int mpad, int NR, int kpad_max) {
  return size_t(nsa) * 4 * size_t(mpad) * 32 + 2 * 4 * size_t(NR) * size_t(kpad_max) * 2 + (2 * size_t(nsa) + 16) * 8 + 64;
}

size_t leaf_smem_bytes(int R, int c) {
  return size_t(2) * kMaxGroupPoints * R * sizeof(float) +
         sizeof(float2) * size_t(std::max(kMaxGroupPoints, c * R)) * kLeafRhs + 64 * sizeof(int);
}

cudaError_t launch_apply_tc(const TCArgs& a, int grid, size_t smem, cudaStream_t stream) {
  cudaError_t err = cudaMemsetAsync(a.counters, 0, tc_counter_bytes(a.plan), stream);
  if (err != cudaSuccess) return err;
  if ((err = cudaFuncSetAttribute(bf_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess)
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
  return cudaLaunchKernelEx(&cfg, bf_apply_tc, a);
}

size_t tc_counter_bytes(const TCPlan& plan) {
  size_t n = 0;
  for (int e = 0; e < plan.n_stages; ++e) n += size_t(plan.st[e].n_groups);
  return (n * sizeof(unsigned) + 255) & ~size_t(255);
}

cudaError_t launch_leaf(const LeafArgs& a, bool u_side, int n_groups, cudaStream_t stream) {
  const size_t smem = leaf_smem_bytes(a.R, a.c);
  auto kern = u_side ? leaf_u_kernel : leaf_v_kernel;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (err != cudaSuccess) return err;
  kern<<<n_groups, kLeafThreads, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace mbf
