// Launchers of the dense centre term of the multiscale butterfly factorization.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mbf {

// u[r][x] (= or +=) sum_c Kc[c][x] g[r][idx[c]]; with n_c = 0 it zeroes u (unless accumulating).
cudaError_t launch_center_fwd(const float2* Kc, const int32_t* idx, int n_c, const float2* g, int64_t len_in,
                              float2* u, int64_t n_out, int nrhs, bool accumulate, cudaStream_t st);
// g[r][idx[c]] += sum_x conj(Kc[c][x]) u[r][x].
cudaError_t launch_center_adj(const float2* Kc, const int32_t* idx, int n_c, const float2* u, int64_t n_out,
                              float2* g, int64_t len_in, int nrhs, cudaStream_t st);

}  // namespace mbf
