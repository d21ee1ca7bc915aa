// Dense centre term of the multiscale butterfly factorization (§4.2, eq. f1):
//   forward  u[r][x]      (= or +=) sum_c K_C[c][x] g[r][idx[c]]
//   adjoint  g[r][idx[c]]   +=      sum_x conj(K_C[c][x]) u[r][x]
// K_C is stored centre-point-major ([c][x], complex64), so a warp reads consecutive x.
#include <cuda_runtime.h>

#include <cstdint>

#include "msbf.hpp"

namespace mbf {

namespace {

constexpr int kCThreads = 256;
constexpr int kCRhs = 8;      // RHS per CTA
constexpr int kCTile = 512;   // centre points staged per round

__global__ void __launch_bounds__(kCThreads) center_fwd_kernel(const float2* __restrict__ Kc,
                                                               const int32_t* __restrict__ idx, int n_c,
                                                               const float2* __restrict__ g, int64_t len_in,
                                                               float2* __restrict__ u, int64_t n_out, int nrhs,
                                                               int accumulate) {
  __shared__ float2 gs[kCTile][kCRhs];
  const int64_t x = int64_t(blockIdx.x) * kCThreads + threadIdx.x;
  const int r0 = blockIdx.y * kCRhs;
  float2 acc[kCRhs];
#pragma unroll
  for (int r = 0; r < kCRhs; ++r) acc[r] = make_float2(0.f, 0.f);
  for (int c0 = 0; c0 < n_c; c0 += kCTile) {
    const int nc = min(kCTile, n_c - c0);
    __syncthreads();
    for (int q = threadIdx.x; q < nc * kCRhs; q += kCThreads) {
      const int cc = q / kCRhs, r = q - cc * kCRhs;
      gs[cc][r] = r0 + r < nrhs ? __ldg(g + int64_t(r0 + r) * len_in + idx[c0 + cc]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (x < n_out)
      for (int cc = 0; cc < nc; ++cc) {
        const float2 k = __ldg(Kc + int64_t(c0 + cc) * n_out + x);
#pragma unroll
        for (int r = 0; r < kCRhs; ++r) {
          const float2 v = gs[cc][r];
          acc[r].x = fmaf(k.x, v.x, fmaf(-k.y, v.y, acc[r].x));
          acc[r].y = fmaf(k.x, v.y, fmaf(k.y, v.x, acc[r].y));
        }
      }
  }
  if (x >= n_out) return;
#pragma unroll
  for (int r = 0; r < kCRhs; ++r) {
    if (r0 + r >= nrhs) break;
    float2* o = u + int64_t(r0 + r) * n_out + x;
    float2 v = acc[r];
    if (accumulate) {
      const float2 w = *o;
      v.x += w.x;
      v.y += w.y;
    }
    *o = v;
  }
}

// One CTA per (centre point, 8 RHS): a block reduction over x.
__global__ void __launch_bounds__(kCThreads) center_adj_kernel(const float2* __restrict__ Kc,
                                                               const int32_t* __restrict__ idx,
                                                               const float2* __restrict__ u, int64_t n_out,
                                                               float2* __restrict__ g, int64_t len_in, int nrhs) {
  __shared__ float2 red[kCThreads / 32][kCRhs];
  const int c = blockIdx.x, r0 = blockIdx.y * kCRhs;
  float2 acc[kCRhs];
#pragma unroll
  for (int r = 0; r < kCRhs; ++r) acc[r] = make_float2(0.f, 0.f);
  for (int64_t x = threadIdx.x; x < n_out; x += kCThreads) {
    const float2 k = __ldg(Kc + int64_t(c) * n_out + x);   // use conj(k)
#pragma unroll
    for (int r = 0; r < kCRhs; ++r) {
      if (r0 + r < nrhs) {
        const float2 v = __ldg(u + int64_t(r0 + r) * n_out + x);
        acc[r].x = fmaf(k.x, v.x, fmaf(k.y, v.y, acc[r].x));
        acc[r].y = fmaf(k.x, v.y, fmaf(-k.y, v.x, acc[r].y));
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < kCRhs; ++r) {
    float sx = acc[r].x, sy = acc[r].y;
    for (int off = 16; off > 0; off >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, off);
      sy += __shfl_xor_sync(0xffffffffu, sy, off);
    }
    if (lane == 0) red[warp][r] = make_float2(sx, sy);
  }
  __syncthreads();
  if (threadIdx.x < kCRhs && r0 + int(threadIdx.x) < nrhs) {
    float2 s = make_float2(0.f, 0.f);
    for (int w = 0; w < kCThreads / 32; ++w) {
      s.x += red[w][threadIdx.x].x;
      s.y += red[w][threadIdx.x].y;
    }
    float2* o = g + int64_t(r0 + threadIdx.x) * len_in + idx[c];
    const float2 w = *o;
    *o = make_float2(w.x + s.x, w.y + s.y);
  }
}

}  // namespace

cudaError_t launch_center_fwd(const float2* Kc, const int32_t* idx, int n_c, const float2* g, int64_t len_in,
                              float2* u, int64_t n_out, int nrhs, bool accumulate, cudaStream_t st) {
  if (n_c == 0) {
    if (accumulate) return cudaSuccess;
    return cudaMemsetAsync(u, 0, size_t(nrhs) * size_t(n_out) * sizeof(float2), st);
  }
  const dim3 grid(unsigned((n_out + kCThreads - 1) / kCThreads), unsigned((nrhs + kCRhs - 1) / kCRhs));
  center_fwd_kernel<<<grid, kCThreads, 0, st>>>(Kc, idx, n_c, g, len_in, u, n_out, nrhs, accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_center_adj(const float2* Kc, const int32_t* idx, int n_c, const float2* u, int64_t n_out,
                              float2* g, int64_t len_in, int nrhs, cudaStream_t st) {
  if (n_c == 0) return cudaSuccess;
  const dim3 grid(unsigned(n_c), unsigned((nrhs + kCRhs - 1) / kCRhs));
  center_adj_kernel<<<grid, kCThreads, 0, st>>>(Kc, idx, u, n_out, g, len_in, nrhs);
  return cudaGetLastError();
}

}  // namespace mbf
