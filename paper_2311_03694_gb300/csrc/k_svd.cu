// SVD-ROM (Sec. 4.4.2): middle weights of the streaming contraction.
//
// With the truncated SVD of the tensor's matricization over the advecting
// index, C_ijk ~ sum_r U_jr sigma_r V[i][r][k], the advection term is
//   c_i = sum_r beta_r sum_k V[i][r][k] u_k,   beta = sigma o (U^T u),
// i.e. the streaming contraction over the slices of V with the middle index
// weighted by beta.  This kernel forms beta (FP64) for every trajectory.
#include "grom_internal.h"

namespace grom {

// One warp per (r, b): the lanes stride over j along row r of U^T (stored
// transposed, rank x n, so the warp reads contiguous memory) and reduce with
// a fixed shuffle tree.
__global__ void k_svd_project(const double* __restrict__ ut, const double* __restrict__ sigma, int64_t n,
                              int64_t rank, const double* u, int64_t u_stride, const double* hist,
                              const int64_t* taken, int64_t hist_stride, const int32_t* active, double* beta) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int b = blockIdx.y;
  if (r >= rank) return;
  double* out = beta + (int64_t)b * rank + r;
  if (active && !active[b]) {
    if (lane == 0) *out = 0.0;
    return;
  }
  const double* ub = taken ? hist + b * hist_stride + (taken[b] % 3) * n : u + b * u_stride;
  const double* row = ut + r * n;
  double s = 0.0;
  for (int64_t j = lane; j < n; j += 32) s = fma(row[j], ub[j], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) *out = sigma[r] * s;
}

cudaError_t svd_project_launch(const double* ut, const double* sigma, int64_t n, int64_t rank, int batch,
                               const double* u, int64_t u_stride, const double* hist, const int64_t* taken,
                               int64_t hist_stride, const int32_t* active, double* beta, cudaStream_t s) {
  constexpr int WARPS = 8;
  dim3 grid((unsigned)((rank + WARPS - 1) / WARPS), (unsigned)batch);
  k_svd_project<<<grid, WARPS * 32, 0, s>>>(ut, sigma, n, rank, u, u_stride, hist, taken, hist_stride, active, beta);
  return cudaGetLastError();
}

}  // namespace grom
