// Persistent SIMT apply of a butterfly factorization on sm_103a (FP32 arithmetic on
// complex64 factors; 1, 2 or 4 right-hand sides per pass).
//
// One CTA per SM walks every stage of eq. (gbf) -- (V^L)^*, (H^l)^*, M^h, G^l, U^L --
// in order (or in reverse, conjugated, for K^*).  Every warp works alone on whole
// groups: it owns a private ring of D shared-memory slots, issues its own
// cp.async.bulk copies of its factor chunks D chunks ahead of the chunk it is
// multiplying (completion tracked by one mbarrier per slot), gathers the group's
// input segments, multiplies, and scatters the result.  Factor data does not depend
// on the vectors, so each warp's copies run ahead across group, stage and pass
// boundaries -- in particular across the grid-wide barrier that separates stages.
// Every wait gives up after kTimeoutNs and sets the status word; all warps then
// leave together at the next barrier, each after waiting for its own copies.
#include <cuda_runtime.h>

#include <cstdint>

#include "apply.hpp"

namespace mbf {

// Warps per CTA and slots per warp for NRB right-hand sides per pass, chosen so that
// W * (D * kSlotBytes + 2 * kMaxLen * NRB * 8) fits the 227 KB opt-in shared memory.
template <int NRB>
struct Cfg;
template <>
struct Cfg<1> {
  static constexpr int W = 8, D = 3;
};
template <>
struct Cfg<2> {
  static constexpr int W = 7, D = 3;
};
template <>
struct Cfg<4> {
  static constexpr int W = 5, D = 3;
};

template <int NRB>
constexpr size_t smem_bytes_for() {
  return size_t(Cfg<NRB>::W) * (size_t(Cfg<NRB>::D) * kSlotBytes + 2 * kMaxLen * NRB * sizeof(float2)) +
         size_t(Cfg<NRB>::W) * Cfg<NRB>::D * 8 + size_t(Cfg<NRB>::W) * 16 * sizeof(int) + 16;
}

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
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Row of RHS `rhs` of the input / output: contiguous [nrhs][len], or the row table.
__device__ __forceinline__ const float2* in_row(const ApplyArgs& a, int rhs) {
  return a.use_rows ? a.rows.in[rhs] : a.in + int64_t(rhs) * a.in_len;
}
__device__ __forceinline__ float2* out_row(const ApplyArgs& a, int rhs) {
  return a.use_rows ? a.rows.out[rhs] : a.out + int64_t(rhs) * a.out_len;
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

// The group of stage `s` whose input pattern `pat` reads segment P (position P * R).
__device__ __forceinline__ int pat_group(int pat, int64_t P, const Stage& s, int c) {
  if (pat == PAT_CONTIG) return int(P / c);
  if (pat == PAT_SPLIT) {
    const int64_t q = P / s.B;
    return int((q / c) * s.B + (P - q * s.B));
  }
  const int64_t q = P / s.ch;   // PAT_CORNER: P = (c b + t) ch + a, g = a B + b
  return int((P - q * s.ch) * s.B + q / c);
}

__device__ __forceinline__ bool item_ok(const Item& it) {
  return it.len >= 1 && it.len <= kMaxLen && it.lpc >= 1 && it.lpc <= kMaxChunkLines &&
         it.nlines <= (it.kind == ITEM_MAIN ? kMaxLen : kMaxLeaf) &&
         chunk_bytes(it.lpc, it.len) <= kSlotBytes;
}

// Position of an item in one warp's sequence: pass, execution stage, the warp's
// k-th group of that stage, and item index in execution order.
struct Pos {
  int pass, e, k, mi;
};

// Normalise p to the first position at or after it whose group exists; false at
// the end of the sequence.  Needs only the plan (no memory loads).
template <bool ADJ>
__device__ __forceinline__ bool pos_fix(const ApplyArgs& a, Pos& p, int wslot, int nslots) {
  const int S = a.plan.n_stages;
  for (;;) {
    if (p.pass >= a.n_pass) return false;
    const Stage& st = a.plan.st[ADJ ? S - 1 - p.e : p.e];
    if (wslot + nslots * p.k >= st.n_groups) {
      p.k = p.mi = 0;
      if (++p.e >= S) {
        p.e = 0;
        ++p.pass;
      }
      continue;
    }
    if (p.mi >= st.n_items) {
      p.mi = 0;
      ++p.k;
      continue;
    }
    return true;
  }
}

template <bool ADJ>
__device__ __forceinline__ Item load_item(const ApplyArgs& a, const Pos& p, int wslot, int nslots) {
  const int S = a.plan.n_stages;
  const Stage& st = a.plan.st[ADJ ? S - 1 - p.e : p.e];
  const int g = wslot + nslots * p.k;
  const int idx = ADJ ? st.n_items - 1 - p.mi : p.mi;
  return a.items[st.item_base + int64_t(g) * st.n_items + idx];
}

__device__ __forceinline__ Item shfl_item(const Item& it, int src) {
  Item o;
  o.off128 = __shfl_sync(0xffffffffu, it.off128, src);
  o.base = __shfl_sync(0xffffffffu, it.base, src);
  const uint32_t w2 = __shfl_sync(0xffffffffu, uint32_t(it.nlines) | (uint32_t(it.len) << 16), src);
  const uint32_t w3 = __shfl_sync(0xffffffffu, uint32_t(it.lpc) | (uint32_t(it.kind) << 16) |
                                                   (uint32_t(it.t) << 24), src);
  o.nlines = uint16_t(w2 & 0xffffu);
  o.len = uint16_t(w2 >> 16);
  o.lpc = uint16_t(w3 & 0xffffu);
  o.kind = uint8_t((w3 >> 16) & 0xffu);
  o.t = uint8_t(w3 >> 24);
  return o;
}

template <int NRB>
struct Acc {
  float2 v[8][NRB];
};

// ---------------------------------------------------------------- chunk routines
// Each lane owns entries e = lane + 32 j (j < JE) of the output (axpy forms); JE =
// ceil(len / 32) is a template argument so the inner loops carry no dead branches.

// y[e] += sum_l T[l][e] x[l]: lines are inputs (forward G^l / (H^l)^* blocks).
template <int NRB, int JE>
__device__ __forceinline__ void chunk_axpy(const float* __restrict__ re, const float* __restrict__ im, int nl,
                                           int len, int lane, const float2* __restrict__ x,
                                           float2 (&acc)[8][NRB]) {
#pragma unroll 4
  for (int l = 0; l < nl; ++l) {
    float2 xv[NRB];
#pragma unroll
    for (int r = 0; r < NRB; ++r) xv[r] = x[l * NRB + r];
#pragma unroll
    for (int j = 0; j < JE; ++j) {
      const int ee = lane + 32 * j;
      if (j < JE - 1 || ee < len) {
        const float ar = re[l * len + ee], ai = im[l * len + ee];
#pragma unroll
        for (int r = 0; r < NRB; ++r) {
          acc[j][r].x = fmaf(ar, xv[r].x, fmaf(-ai, xv[r].y, acc[j][r].x));
          acc[j][r].y = fmaf(ar, xv[r].y, fmaf(ai, xv[r].x, acc[j][r].y));
        }
      }
    }
  }
}

// Same, lines are the group's points; when a line enters a new leaf the sums of the
// previous leaf are written to its segment of `seg` and cleared.
template <int NRB, int JE>
__device__ __forceinline__ void chunk_axpy_leaves(const float* __restrict__ re, const float* __restrict__ im,
                                                  int nl, int len, int lane, int l0, const float2* __restrict__ x,
                                                  float2 (&acc)[8][NRB], int& ct, int& nb, const int* lbnd, int c,
                                                  float2* seg) {
  for (int l = 0; l < nl; ++l) {
    while (l0 + l >= nb) {
      if (ct >= 0) {
#pragma unroll
        for (int j = 0; j < JE; ++j) {
          const int ee = lane + 32 * j;
          if (j < JE - 1 || ee < len)
#pragma unroll
            for (int r = 0; r < NRB; ++r) {
              seg[(ct * len + ee) * NRB + r] = acc[j][r];
              acc[j][r] = make_float2(0.f, 0.f);
            }
        }
      }
      ++ct;
      nb = ct + 1 <= c ? lbnd[ct + 1] : 0x7fffffff;
    }
    float2 xv[NRB];
#pragma unroll
    for (int r = 0; r < NRB; ++r) xv[r] = x[l * NRB + r];
#pragma unroll
    for (int j = 0; j < JE; ++j) {
      const int ee = lane + 32 * j;
      if (j < JE - 1 || ee < len) {
        const float ar = re[l * len + ee], ai = im[l * len + ee];
#pragma unroll
        for (int r = 0; r < NRB; ++r) {
          acc[j][r].x = fmaf(ar, xv[r].x, fmaf(-ai, xv[r].y, acc[j][r].x));
          acc[j][r].y = fmaf(ar, xv[r].y, fmaf(ai, xv[r].x, acc[j][r].y));
        }
      }
    }
  }
}

// U^L: lines are columns k (l0 + l), entries are the group's points; point e uses
// coefficient k of its own leaf ta[j]'s segment of `x` (segments of length R = rows).
template <int NRB, int JE>
__device__ __forceinline__ void chunk_axpy_ul(const float* __restrict__ re, const float* __restrict__ im, int nl,
                                              int len, int lane, int l0, int rows, const float2* __restrict__ x,
                                              const int (&ta)[8], float2 (&acc)[8][NRB]) {
#pragma unroll 2
  for (int l = 0; l < nl; ++l) {
#pragma unroll
    for (int j = 0; j < JE; ++j) {
      const int ee = lane + 32 * j;
      if (j < JE - 1 || ee < len) {
        const float ar = re[l * len + ee], ai = im[l * len + ee];
        const float2* xv = x + size_t(ta[j] * rows + l0 + l) * NRB;
#pragma unroll
        for (int r = 0; r < NRB; ++r) {
          const float2 v = xv[r];
          acc[j][r].x = fmaf(ar, v.x, fmaf(-ai, v.y, acc[j][r].x));
          acc[j][r].y = fmaf(ar, v.y, fmaf(ai, v.x, acc[j][r].y));
        }
      }
    }
  }
}

#define MBF_DISPATCH_JE(je, CALL) \
  switch (je) {                   \
    case 1: CALL(1); break;       \
    case 2: CALL(2); break;       \
    case 3: CALL(3); break;       \
    case 4: CALL(4); break;       \
    case 5: CALL(5); break;       \
    case 6: CALL(6); break;       \
    case 7: CALL(7); break;       \
    default: CALL(8); break;      \
  }

// ---------------------------------------------------------------- kernel

template <int NRB, bool ADJ>
__global__ void __launch_bounds__(Cfg<NRB>::W * 32, 1) bf_apply_simt(const __grid_constant__ ApplyArgs a) {
  const uint64_t wait_lim = a.wait_ns ? a.wait_ns : kTimeoutNs;
  constexpr int W = Cfg<NRB>::W, D = Cfg<NRB>::D;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* ring = smem + size_t(warp) * D * kSlotBytes;
  float2* xin = reinterpret_cast<float2*>(smem + size_t(W) * D * kSlotBytes) + size_t(warp) * 2 * kMaxLen * NRB;
  float2* yout = xin + kMaxLen * NRB;      // group output; also the leaf-gather buffer
  uint64_t* bars = reinterpret_cast<uint64_t*>(
      smem + size_t(W) * (size_t(D) * kSlotBytes + 2 * kMaxLen * NRB * sizeof(float2)));
  uint64_t* full = bars + warp * D;
  int* lbnd = reinterpret_cast<int*>(bars + W * D) + warp * 16;   // leaf starts of the group
  volatile int* abort = reinterpret_cast<volatile int*>(reinterpret_cast<int*>(bars + W * D) + W * 16);

  if (lane == 0)
    for (int s = 0; s < D; ++s) mbar_init(&full[s], 1);
  if (threadIdx.x == 0) *abort = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  const Plan& plan = a.plan;
  const int S = plan.n_stages, c = plan.c;
  const int wslot = blockIdx.x + gridDim.x * warp;   // this warp's index among all warps
  const int nslots = gridDim.x * W;

  // ---- issue cursor (lane 0 only): D chunks ahead of the chunk being consumed.
  // It holds the current item and keeps the descriptor of the following item in
  // flight, so crossing into the next item does not wait for a memory load.
  Pos ip{0, 0, 0, 0}, np{0, 0, 0, 0};
  Item icur{}, inext{};
  bool ivalid = false, nvalid = false;
  int il0 = 0;
  uint32_t issued = 0;
  if (lane == 0) {
    ivalid = pos_fix<ADJ>(a, ip, wslot, nslots);
    if (ivalid) icur = load_item<ADJ>(a, ip, wslot, nslots);
    np = ip;
    ++np.mi;
    nvalid = ivalid && pos_fix<ADJ>(a, np, wslot, nslots);
    if (nvalid) inext = load_item<ADJ>(a, np, wslot, nslots);
  }
  auto issue_next = [&](uint32_t slot) {
    while (ivalid && il0 >= int(icur.nlines)) {
      ip = np;
      icur = inext;
      ivalid = nvalid;
      il0 = 0;
      if (nvalid) {
        ++np.mi;
        nvalid = pos_fix<ADJ>(a, np, wslot, nslots);
        if (nvalid) inext = load_item<ADJ>(a, np, wslot, nslots);
      }
    }
    if (!ivalid) return;
    if (!item_ok(icur)) {
      set_status(a.status, abort, ST_BAD_ITEM);
      ivalid = false;
      return;
    }
    const int nl = min(int(icur.lpc), int(icur.nlines) - il0);
    const uint64_t off =
        uint64_t(icur.off128) * 128u + uint64_t(il0 / icur.lpc) * uint64_t(chunk_bytes(icur.lpc, icur.len));
    const uint32_t bytes = uint32_t(chunk_bytes(nl, icur.len));
    fence_proxy_async();
    mbar_expect_tx(&full[slot], bytes);
    bulk_g2s(ring + size_t(slot) * kSlotBytes, a.arena + off, bytes, &full[slot]);
    ++issued;
    il0 += icur.lpc;
  };
  if (lane == 0)
    for (int s = 0; s < D; ++s) issue_next(uint32_t(s));
  __syncwarp();

  uint32_t consumed = 0;
  unsigned nbar = 0;

  // Wait for chunk `consumed`.  Lane 0 polls with a time limit, then every lane
  // observes the completed phase itself.  A chunk that was never issued (after an
  // abort) or a wait that gives up leaves the warp computing on garbage, with
  // uniform control flow; the results are discarded.
  auto wait_chunk = [&](uint32_t slot, uint32_t ph) {
    int got = 0;
    if (lane == 0 && consumed < issued) {
      got = 1;
      if (!mbar_try(&full[slot], ph)) {
        const uint64_t t0 = gtimer();
        while (!mbar_try(&full[slot], ph)) {
          if (gtimer() - t0 > wait_lim) {
            got = 0;
            if (!*abort) set_status(a.status, abort, ST_FULL_TIMEOUT);
            break;
          }
        }
      }
    }
    got = __shfl_sync(0xffffffffu, got, 0);
    if (got)
      while (!mbar_try(&full[slot], ph)) {
      }
  };
  // After the whole warp is done with `slot`, lane 0 refills it with the next chunk.
  auto release = [&](uint32_t slot) {
    __syncwarp();
    if (lane == 0 && !*abort) issue_next(slot);
    __syncwarp();
    ++consumed;
  };

  bool stop = false;
  for (int pass = 0; pass < a.n_pass && !stop; ++pass) {
    const int rhs0 = pass * NRB;
    for (int e = 0; e < S; ++e) {
      const Stage& st = plan.st[ADJ ? S - 1 - e : e];
      if (pass > 0 && e == 0) {
        // grid-wide barrier between passes: the next pass reuses every stage buffer
        // (the last thread of the CTA issues no bulk copies)
        ++nbar;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
          __threadfence();
          atomicAdd(a.barrier, 1u);
          const unsigned target = nbar * gridDim.x;
          const uint64_t t0 = gtimer();
          while (*reinterpret_cast<volatile unsigned*>(a.barrier) < target) {
            if (*reinterpret_cast<volatile int*>(a.status) != 0) { *abort = 1; break; }
            if (gtimer() - t0 > wait_lim) { set_status(a.status, abort, ST_BARRIER_TIMEOUT); break; }
            __nanosleep(20);
          }
          __threadfence();
        }
        if (__syncthreads_or(*abort)) {
          stop = true;
          break;
        }
      }
      const float2* src = a.bufs + (e > 0 ? e - 1 : 0) * a.buf_stride;   // previous stage's output
      float2* dst = a.bufs + int64_t(e) * a.buf_stride;
      unsigned* cnt_in = a.counters + int64_t(e) * st.n_groups;
      const bool notify = e + 1 < S;
      const Stage& nst = plan.st[ADJ ? (S - 2 - e >= 0 ? S - 2 - e : 0) : (e + 1 < S ? e + 1 : e)];
      const int next_in_pat = ADJ ? nst.out_pat : nst.in_pat;
      unsigned* cnt_out = a.counters + int64_t(e + 1) * nst.n_groups;
      const unsigned need = unsigned(c) * unsigned(pass + 1);
      const int in_pat = ADJ ? st.out_pat : st.in_pat;
      const int out_pat = ADJ ? st.in_pat : st.out_pat;
      const int Rin = ADJ ? st.R_out : st.R_in;    // execution-sense segment lengths
      const int Rout = ADJ ? st.R_in : st.R_out;
      // after a group's outputs are stored: make them visible, then count one written
      // segment for the consumer group of each of the c output segments
      auto notify_consumers = [&](int g) {
        if (!notify) return;
        __threadfence();
        __syncwarp();
        if (lane < c) {
          const int64_t P = pat_off(out_pat, g, lane, st, Rout, c) / Rout;
          atomicAdd(cnt_out + pat_group(next_in_pat, P, nst, c), 1u);
        }
      };
      // leaves of this stage: Omega side (V^L) next to H^{L-1}, X side (U^L) next to G^{L-1}
      const bool leaf_w = st.in_pat == PAT_LEAF, leaf_x = st.out_pat == PAT_LEAF;
      const int32_t* lperm = leaf_w ? a.w_perm : a.x_perm;
      const int32_t* loff = leaf_w ? a.w_off : a.x_off;
      const bool leaf_in = in_pat == PAT_LEAF;      // leaves read the input vector
      const bool leaf_out = out_pat == PAT_LEAF;    // leaves write the output vector

      for (int k = 0;; ++k) {
        const int g = wslot + nslots * k;
        if (g >= st.n_groups || *abort) break;
        // all item descriptors of the group, one per lane (execution order)
        Item myit{};
        if (lane < st.n_items) {
          const int idx = ADJ ? st.n_items - 1 - lane : lane;
          myit = a.items[st.item_base + int64_t(g) * st.n_items + idx];
        }
        int p0 = 0, npts = 0, myb = 0;
        if (leaf_w || leaf_x) {
          // the group's c leaves hold the contiguous tree-order points [p0, p0 + npts);
          // lane t <= c keeps the start of leaf t relative to p0
          int v = 0;
          if (lane <= c) v = loff[c * g + lane];
          p0 = __shfl_sync(0xffffffffu, v, 0);
          npts = min(__shfl_sync(0xffffffffu, v, c) - p0, kMaxGroupPoints);
          myb = v - p0;
          if (lane <= c) lbnd[lane] = myb;
          if (leaf_in) {
            if (!st.leaf_only)
              for (int q = lane; q < c * Rin * NRB; q += 32) xin[q] = make_float2(0.f, 0.f);
            // values of the group's points: all indices first, then all values, so the
            // loads of one lane are independent of each other
            for (int pb = 0; pb < npts; pb += 32 * 8) {
              int idx[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int pt = pb + lane + 32 * u;
                idx[u] = pt < npts ? lperm[p0 + pt] : 0;
              }
              float2 v[8][NRB];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int pt = pb + lane + 32 * u;
#pragma unroll
                for (int r = 0; r < NRB; ++r)
                  v[u][r] = (pt < npts && rhs0 + r < a.nrhs)
                                ? __ldg(in_row(a, rhs0 + r) + idx[u])
                                : make_float2(0.f, 0.f);
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int pt = pb + lane + 32 * u;
                if (pt < npts)
#pragma unroll
                  for (int r = 0; r < NRB; ++r) yout[pt * NRB + r] = v[u][r];
              }
            }
          }
        }
        if (in_pat != PAT_LEAF) {
          // wait until all c input segments of this group have been written by the
          // producing groups of the previous stage (each adds 1 per segment)
          if (lane == 0) {
            const unsigned* cp = cnt_in + g;
            const unsigned need_g = need + (e + 1 == a.stall_stage1 && g == 0 ? 1u : 0u);
            if (ld_acquire(cp) < need_g) {
              const uint64_t t0 = gtimer();
              while (ld_acquire(cp) < need_g) {
                if (*abort || *reinterpret_cast<volatile int*>(a.status) != 0) { *abort = 1; break; }
                if (gtimer() - t0 > wait_lim) { set_status(a.status, abort, ST_DEP_TIMEOUT); break; }
                __nanosleep(32);
              }
            }
          }
          __syncwarp();
          // the group's input segments from the previous stage's vector (L2), in
          // batches of 8 independent loads per lane; a compact stage's main item holds
          // only the first r_t lines of segment t (c = 4), so only those are read, packed
          // in line order: segment t starts at line p_t = r_0 + ... + r_(t-1)
          const bool cmp = st.compact && !ADJ;
          int p1 = Rin, p2 = 2 * Rin, p3 = 3 * Rin, nlin = c * Rin;
          if (cmp) {
            const int32_t rk = __shfl_sync(0xffffffffu, myit.base, st.main_idx);
            p1 = seg_lines(rk, 0);
            p2 = p1 + seg_lines(rk, 1);
            p3 = p2 + seg_lines(rk, 2);
            nlin = p3 + seg_lines(rk, 3);
          }
          const int nq = nlin * NRB;
          for (int qb = 0; qb < nq; qb += 32 * 8) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int q = qb + lane + 32 * u;
              if (q < nq) {
                const int r = q % NRB;
                int t, kk;
                if (cmp) {
                  const int line = q / NRB;
                  t = (line >= p1 ? 1 : 0) + (line >= p2 ? 1 : 0) + (line >= p3 ? 1 : 0);
                  kk = line - (t == 0 ? 0 : t == 1 ? p1 : t == 2 ? p2 : p3);
                } else {
                  kk = (q / NRB) % Rin;
                  t = q / (NRB * Rin);
                }
                const int64_t pos = pat_off(in_pat, g, t, st, Rin, c) + kk;
                v[u] = __ldcg(src + pos * NRB + r);
              }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int q = qb + lane + 32 * u;
              if (q < nq) xin[q] = v[u];
            }
          }
        }
        __syncwarp();
        for (int mi = 0; mi < st.n_items; ++mi) {
          const Item it = shfl_item(myit, mi);
          if (!item_ok(it)) {
            if (lane == 0) set_status(a.status, abort, ST_BAD_ITEM);
            break;
          }
          const int len = it.len, nlines = it.nlines;
          const int je = (len + 31) >> 5;
          const int kind = it.kind;
          Acc<NRB> acc;
#pragma unroll
          for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int r = 0; r < NRB; ++r) acc.v[j][r] = make_float2(0.f, 0.f);
          // leaf of each of this lane's entries (entries are group points for U^L items)
          int ta[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) ta[j] = 0;
          if (kind == ITEM_LEAF_X) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int pt = lane + 32 * j;
              int t = 0;
              for (int q = 1; q < c; ++q) t += (pt >= lbnd[q]) ? 1 : 0;
              ta[j] = t;
            }
          }
          // points-as-lines items: ct = leaf of the current line, nb = start of leaf ct+1
          int ct = -1, nb = 0;
          // leaf sums go to segment t of xin (fused) or, in the leaf stage, straight to
          // the level-L coefficient vector at leaf c g + t
          float2* seg = st.leaf_only ? dst + size_t(c) * g * len * NRB : xin;
          auto flush_leaf = [&](int t) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int ee = lane + 32 * j;
              if (j < je && ee < len)
#pragma unroll
                for (int r = 0; r < NRB; ++r) {
                  seg[(t * len + ee) * NRB + r] = acc.v[j][r];
                  acc.v[j][r] = make_float2(0.f, 0.f);
                }
            }
          };

          for (int l0 = 0; l0 < nlines; l0 += it.lpc) {
            const int nl = min(int(it.lpc), nlines - l0);
            const uint32_t slot = consumed % D, ph = (consumed / D) & 1u;
            wait_chunk(slot, ph);
            __syncwarp();
            const float* re = reinterpret_cast<const float*>(ring + size_t(slot) * kSlotBytes);
            const float* im = re + pad4(int64_t(nl) * len);
            if (kind == ITEM_MAIN && !ADJ) {
              // G^l / (H^l)^* block: lines are inputs (x = xin), one lane per output row
#define MBF_CALL(JE) chunk_axpy<NRB, JE>(re, im, nl, len, lane, xin + size_t(l0) * NRB, acc.v)
              MBF_DISPATCH_JE(je, MBF_CALL)
#undef MBF_CALL
            } else if (kind == ITEM_LEAF_W && !ADJ) {
              // (V^L_j)^*: lines are the group's points (values gathered in yout); the sum
              // of leaf t goes to segment t of xin once its last point is passed
#define MBF_CALL(JE) \
  chunk_axpy_leaves<NRB, JE>(re, im, nl, len, lane, l0, yout + size_t(l0) * NRB, acc.v, ct, nb, lbnd, c, seg)
              MBF_DISPATCH_JE(je, MBF_CALL)
#undef MBF_CALL
            } else if (kind == ITEM_LEAF_X && !ADJ) {
              // U^L: lines are the columns k, one lane per group point; each point takes
              // coefficient k of its own leaf's segment of the main output (yout)
#define MBF_CALL(JE) chunk_axpy_ul<NRB, JE>(re, im, nl, len, lane, l0, nlines, yout, ta, acc.v)
              MBF_DISPATCH_JE(je, MBF_CALL)
#undef MBF_CALL
            } else if (kind == ITEM_LEAF_X) {
              // adjoint of U^L: for each column k and each leaf t, the conjugate dot
              // product over the leaf's points (values gathered in yout) -> xin[t][k]
              for (int l = 0; l < nl; ++l) {
                const int kk = l0 + l;
                float2 pr[8][NRB];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const int ee = lane + 32 * j;
                  const bool on = j < je && ee < len;
                  const float ar = on ? re[l * len + ee] : 0.f, ai = on ? -im[l * len + ee] : 0.f;
#pragma unroll
                  for (int r = 0; r < NRB; ++r) {
                    const float2 v = on ? yout[ee * NRB + r] : make_float2(0.f, 0.f);
                    pr[j][r] = make_float2(ar * v.x - ai * v.y, ar * v.y + ai * v.x);
                  }
                }
                for (int t = 0; t < c; ++t) {
                  float2 sm[NRB];
#pragma unroll
                  for (int r = 0; r < NRB; ++r) {
                    sm[r] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                      if (ta[j] == t) { sm[r].x += pr[j][r].x; sm[r].y += pr[j][r].y; }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                      sm[r].x += __shfl_xor_sync(0xffffffffu, sm[r].x, off);
                      sm[r].y += __shfl_xor_sync(0xffffffffu, sm[r].y, off);
                    }
                  }
                  if (lane == 0)
#pragma unroll
                    for (int r = 0; r < NRB; ++r) xin[(t * nlines + kk) * NRB + r] = sm[r];
                }
              }
            } else {
              // dot: one output per line, lanes across the line.  Adjoint main block
              // (x = xin, out -> yout) or adjoint of (V^L)^* (a line is a point of leaf
              // ct, x = that leaf's segment of yout, out -> xin at the point)
              const bool main = kind == ITEM_MAIN;
              const float2* x = xin;
              // leaf lines: x = the leaf's segment of the main output (yout), or of the
              // gathered input (xin) in the leaf stage; out = the other buffer
              const float2* lx = st.leaf_only ? xin : yout;
              float2* o = main ? yout : (st.leaf_only ? yout : xin);
              for (int l = 0; l < nl; ++l) {
                if (!main) {
                  while (l0 + l >= nb) {
                    ++ct;
                    nb = ct + 1 <= c ? lbnd[ct + 1] : 0x7fffffff;
                  }
                  x = lx + size_t(ct) * len * NRB;
                }
                float2 sm[NRB];
#pragma unroll
                for (int r = 0; r < NRB; ++r) sm[r] = make_float2(0.f, 0.f);
                for (int ee = lane; ee < len; ee += 32) {
                  const float ar = re[l * len + ee], ai = -im[l * len + ee];
#pragma unroll
                  for (int r = 0; r < NRB; ++r) {
                    const float2 xv = x[ee * NRB + r];
                    sm[r].x = fmaf(ar, xv.x, fmaf(-ai, xv.y, sm[r].x));
                    sm[r].y = fmaf(ar, xv.y, fmaf(ai, xv.x, sm[r].y));
                  }
                }
#pragma unroll
                for (int r = 0; r < NRB; ++r)
#pragma unroll
                  for (int off = 16; off > 0; off >>= 1) {
                    sm[r].x += __shfl_xor_sync(0xffffffffu, sm[r].x, off);
                    sm[r].y += __shfl_xor_sync(0xffffffffu, sm[r].y, off);
                  }
                if (lane == 0)
#pragma unroll
                  for (int r = 0; r < NRB; ++r) o[(l0 + l) * NRB + r] = sm[r];
              }
            }
            release(slot);
          }
          // ---- results held in registers
          if (kind == ITEM_MAIN && !ADJ) {
            if (out_pat == PAT_LEAF) {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int ee = lane + 32 * j;
                if (j < je && ee < len)
#pragma unroll
                  for (int r = 0; r < NRB; ++r) yout[ee * NRB + r] = acc.v[j][r];
              }
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int ee = lane + 32 * j;
                if (j < je && ee < len) {
                  const int t = ee / Rout, kk = ee - (ee / Rout) * Rout;
                  const int64_t pos = pat_off(out_pat, g, t, st, Rout, c) + kk;
#pragma unroll
                  for (int r = 0; r < NRB; ++r) dst[pos * NRB + r] = acc.v[j][r];
                }
              }
              notify_consumers(g);
            }
          } else if (kind == ITEM_LEAF_W && !ADJ) {
            // the last leaf with points; in the leaf stage also every later (empty) leaf,
            // whose vector must read zero
            for (;;) {
              if (ct >= 0) flush_leaf(ct);
              if (!st.leaf_only || ct >= c - 1) break;
              ++ct;
            }
            if (st.leaf_only) notify_consumers(g);
          } else if (kind == ITEM_LEAF_X && !ADJ) {
            // outputs of the group's points, tree order, for the scatter below
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int ee = lane + 32 * j;
              if (j < je && ee < npts)
#pragma unroll
                for (int r = 0; r < NRB; ++r) xin[ee * NRB + r] = acc.v[j][r];
            }
          } else if (kind == ITEM_MAIN && ADJ && out_pat != PAT_LEAF) {
            // adjoint main block: scatter yout (forward-input layout) to the next buffer;
            // in a compact stage yout holds the item's lines (the first r_t entries of
            // each segment t, in order) and the entries beyond r_t are zero
            __syncwarp();
            for (int q = lane; q < c * Rout * NRB; q += 32) {
              const int r = q % NRB, kk = (q / NRB) % Rout, t = q / (NRB * Rout);
              const int64_t pos = pat_off(out_pat, g, t, st, Rout, c) + kk;
              float2 v;
              if (st.compact) {
                int pre = 0;
                for (int u = 0; u < t; ++u) pre += seg_lines(it.base, u);
                v = kk < seg_lines(it.base, t) ? yout[(pre + kk) * NRB + r] : make_float2(0.f, 0.f);
              } else {
                v = yout[q];
              }
              dst[pos * NRB + r] = v;
            }
            notify_consumers(g);
          }
          __syncwarp();
        }
        if (leaf_out) {
          // the group's leaf outputs (tree order; in yout for the leaf stage, else in
          // xin) to natural order
          __syncwarp();
          const float2* res = st.leaf_only ? yout : xin;
          for (int pb = 0; pb < npts; pb += 32 * 8) {
            int idx[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int pt = pb + lane + 32 * u;
              idx[u] = pt < npts ? lperm[p0 + pt] : 0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int pt = pb + lane + 32 * u;
              if (pt < npts)
#pragma unroll
                for (int r = 0; r < NRB; ++r)
                  if (rhs0 + r < a.nrhs) {
                    float2* o = out_row(a, rhs0 + r) + idx[u];
                    float2 v = res[pt * NRB + r];
                    if (a.accumulate) {
                      const float2 w = *o;
                      v.x += w.x;
                      v.y += w.y;
                    }
                    *o = v;
                  }
            }
          }
          __syncwarp();
        }
      }
    }
  }

  // Drain: after an abort, wait (bounded) for this warp's copies still in flight so
  // that no bulk copy writes shared memory after the CTA exits.
  if (lane == 0) {
    for (uint32_t q = consumed; q < issued; ++q) {
      const uint32_t slot = q % D, ph = (q / D) & 1u;
      const uint64_t t1 = gtimer();
      while (!mbar_try(&full[slot], ph) && gtimer() - t1 < kTimeoutNs) {
      }
    }
  }
}

// ---------------------------------------------------------------- host side

size_t simt_smem_bytes(int nrb, int) {
  switch (nrb) {
    case 1: return smem_bytes_for<1>();
    case 2: return smem_bytes_for<2>();
    default: return smem_bytes_for<4>();
  }
}

int simt_threads(int nrb) {
  switch (nrb) {
    case 1: return Cfg<1>::W * 32;
    case 2: return Cfg<2>::W * 32;
    default: return Cfg<4>::W * 32;
  }
}

template <int NRB, bool ADJ>
static cudaError_t launch_t(const ApplyArgs& a, int grid, size_t smem, cudaStream_t stream) {
  auto kern = bf_apply_simt<NRB, ADJ>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(Cfg<NRB>::W * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// Shared-memory footprint and co-resident grid (one CTA per SM).
cudaError_t simt_config(int nrb, int* grid, int* ns, size_t* smem) {
  int dev = 0, sms = 0, optin = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return err;
  *smem = simt_smem_bytes(nrb, 0);
  if (*smem > size_t(optin)) return cudaErrorInvalidConfiguration;
  *ns = 0;
  *grid = sms;
  return cudaSuccess;
}

size_t counter_bytes(const Plan& plan) {
  size_t n = 0;
  for (int e = 0; e < plan.n_stages; ++e) n += size_t(plan.st[e].n_groups);
  return (n * sizeof(unsigned) + 255) & ~size_t(255);
}

// The barrier word is followed (256 bytes later) by the counters; both are cleared.
cudaError_t launch_apply_simt(const ApplyArgs& a, int nrb, bool adj, int grid, size_t smem,
                              cudaStream_t stream) {
  cudaError_t err = cudaMemsetAsync(a.barrier, 0, 256 + counter_bytes(a.plan), stream);
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
