// CP fitting by alternating least squares (Sec. 2.3, eq. cp_als) and its
// skew-preserving variant ALS-skew (Sec. 3.3, eq. skew_abc_struct,
// eq. cp_als_quad), with the MTTKRP of every subproblem on the tensor cores.
//
// Each least-squares subproblem is solved through its normal equations,
//   A_m = MTTKRP_m * (Hadamard product of the other two Gram matrices)^-1,
// where MTTKRP_m = X_(m) (P kr Q) is the K2 contraction with the Khatri-Rao
// operand built from the two other factors.  The tensor is kept in three
// BF16 layouts, one per matricization, each in the K2 row format (rows of
// round_up(n, 64) values):
//   X1[i][j][k]  (rows i: P = A2 over j, Q = A3 over k)
//   X2[j][i][k]  (rows j: P = A1 over i, Q = A3 over k)
//   X3[k][i][j]  (rows k: P = A1 over i, Q = A2 over j)
// Everything after the upload stays on the device: the factors, their FP64
// Gram matrices, and the rank x rank SPD solves (a blocked FP64 Cholesky of
// the normal matrix, then one warp per row for the two triangular solves;
// rank^3/3 + 2 n rank^2 flops per update).  Only the Cholesky breakdown flag,
// the residual's two sums and the final factors come back to the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "grom_internal.h"

using namespace grom;

constexpr int ALS_PARTS = 256;  // blocks of the residual's reductions

struct grom_als {
  int64_t n = 0, np = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  uint8_t* x[3] = {nullptr, nullptr, nullptr};  // BF16 layouts X1, X2, X3
  CUtensorMap tmap[3];
  double xnorm2 = 0.0;  // ||X||_F^2 of the BF16 tensor the fit sees
  int* err = nullptr;
  // per-fit buffers (grown on demand), FP64 on the device
  int64_t rcap = 0;
  double* f[3] = {nullptr, nullptr, nullptr};     // factors, n x rank
  double* anew = nullptr;                         // a least-squares update, n x rank
  double* b1 = nullptr;                           // ALS-skew's shared factor, n x rank/2
  double* mt = nullptr;                           // MTTKRP output, rank x n
  double* gram[3] = {nullptr, nullptr, nullptr};  // Gram matrices of the factors, rank x rank
  double* h = nullptr;                            // normal matrix, then its Cholesky factor L
  double* lt = nullptr;                           // L^T
  double* rdiag = nullptr;                        // reciprocals of L's diagonal
  double* part = nullptr;                         // 2 x ALS_PARTS reduction partials
  int* flag = nullptr;                            // Cholesky breakdown
  void* k2s = nullptr;
  size_t k2s_bytes = 0;
  // timing since the last grom_als_stats: MTTKRP device time (CUDA events
  // around each tensor-core launch) and wall time of the SPD solves
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double mttkrp_ms = 0.0, solve_ms = 0.0;
  int64_t mttkrp_calls = 0;
};

namespace {

// X1 and X2 rows of a slab of test indices [i0, i0 + cnt) (FP64 input rows
// (i, j) of n values), rounded once to BF16.
__global__ void k_als_x12(const double* __restrict__ src, int64_t cnt, int64_t n, int64_t np, int64_t i0,
                          __nv_bfloat16* __restrict__ x1, __nv_bfloat16* __restrict__ x2) {
  const int64_t total = cnt * n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t il = t / (n * n), rem = t - il * n * n, j = rem / n, k = rem - j * n;
    const int64_t i = i0 + il;
    const __nv_bfloat16 v = __double2bfloat16(src[t]);
    x1[(i * n + j) * np + k] = v;
    x2[(j * n + i) * np + k] = v;
  }
}

// X3[k][i][j] = X[i][j][k]: a 32 x 32 tile of (j, k) per block through shared
// memory, coalesced on both sides.
__global__ void k_als_x3(const double* __restrict__ src, int64_t n, int64_t np, int64_t i0,
                         __nv_bfloat16* __restrict__ x3) {
  __shared__ double tile[32][33];
  const int64_t il = blockIdx.z;
  const int64_t jb = (int64_t)blockIdx.x * 32, kb = (int64_t)blockIdx.y * 32;
  const double* s = src + il * n * n;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = jb + r, k = kb + threadIdx.x;
    tile[r][threadIdx.x] = (j < n && k < n) ? s[j * n + k] : 0.0;
  }
  __syncthreads();
  const int64_t i = i0 + il;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t k = kb + r, j = jb + threadIdx.x;
    if (j < n && k < n) x3[(k * n + i) * np + j] = __double2bfloat16(tile[threadIdx.x][r]);
  }
}

// Per-block partial sums of x^2 over the BF16-rounded values, the tensor the
// fit sees (summed on the host in block order).
__global__ void k_als_norm(const double* __restrict__ src, int64_t total, double* part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)__bfloat162float(__double2bfloat16(src[t]));
    s = fma(x, x, s);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// G = F^T F for F (n x r, row-major FP64), 16 x 16 output tiles; G is
// symmetric, so only the tiles on and above the diagonal are computed (FP64
// runs at about two operations per clock per SM here) and mirrored.
__global__ void k_gram(const double* __restrict__ F, int64_t n, int64_t r, double* __restrict__ G) {
  if (blockIdx.x < blockIdx.y) return;  // whole block, before any barrier
  __shared__ double a[16][17], b[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t row = (int64_t)blockIdx.y * 16 + ty, col = (int64_t)blockIdx.x * 16 + tx;
  double s = 0.0;
  for (int64_t i0 = 0; i0 < n; i0 += 16) {
    const int64_t i = i0 + ty;
    a[ty][tx] = (i < n && (int64_t)blockIdx.y * 16 + tx < r) ? F[i * r + blockIdx.y * 16 + tx] : 0.0;
    b[ty][tx] = (i < n && col < r) ? F[i * r + col] : 0.0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) s = fma(a[q][ty], b[q][tx], s);
    __syncthreads();
  }
  if (row < r && col < r) {
    G[row * r + col] = s;
    G[col * r + row] = s;
  }
}

// ------------------------------------------------ SPD solves on the device
// The normal equations A = M H^-1 with H = Ga o Gb + (ridge + mu) max diag(Ga o Gb) I.

// H, with the diagonal maximum found by every block (r entries).
__global__ void k_als_normal(const double* __restrict__ Ga, const double* __restrict__ Gb, int64_t r, double rel,
                             double* __restrict__ H) {
  __shared__ double wm[32];
  double m = 0.0;
  for (int64_t a = threadIdx.x; a < r; a += blockDim.x) m = fmax(m, Ga[a * r + a] * Gb[a * r + a]);
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wm[w]);
  const double add = rel * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < r * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t / r;
    H[t] = Ga[t] * Gb[t] + (t == a * r + a ? add : 0.0);
  }
}

constexpr int CH = 32;  // Cholesky block
constexpr int UT = 16;  // trailing-update tile

// 1/sqrt(d) for a positive finite d: the exponent is split off so that the
// mantissa part m in [1, 4) takes an FP32 estimate, which two Newton-Raphson
// steps for the reciprocal square root, y <- y (3 - m y^2) / 2, bring to FP64
// precision (each step about doubles the correct bits).  FP64 division and
// square root cost thousands of cycles on this part, a step of this a few
// hundred.
__device__ __forceinline__ double rsqrt_nr(double d) {
  const int e = ilogb(d) >> 1;
  const double m = scalbn(d, -2 * e);
  double y = (double)rsqrtf((float)m);
  y = y * (1.5 - 0.5 * m * y * y);
  y = y * (1.5 - 0.5 * m * y * y);
  return scalbn(y, -e);
}

// Factors the diagonal block at (kb, kb) in place (lower), one thread per
// entry (32 x 32), right-looking, and stores the reciprocals of its pivots
// in rdiag[kb ..].  A pivot that is not positive and finite sets *flag.
__global__ void __launch_bounds__(CH * CH) k_chol_diag(double* H, int64_t r, int64_t kb, double* rdiag, int* flag) {
  __shared__ double A[CH][CH + 1];
  __shared__ double ry;
  __shared__ int bad;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // entry A[ty][tx]
  const int nb = (int)(r - kb < CH ? r - kb : CH);
  if (ty < nb && tx < nb) A[ty][tx] = H[(kb + ty) * r + kb + tx];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (threadIdx.x == 0) {
      const double d = A[c][c];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
      } else {
        const double y = rsqrt_nr(d);
        A[c][c] = d * y;
        ry = y;
        rdiag[kb + c] = y;
      }
    }
    __syncthreads();
    if (bad) break;  // read by every thread between the same two barriers
    if (tx == c && ty > c && ty < nb) A[ty][c] *= ry;
    __syncthreads();
    if (ty > c && ty < nb && tx > c && tx <= ty) A[ty][tx] -= A[ty][c] * A[tx][c];
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicExch(flag, 1);
    return;
  }
  if (ty < nb && tx < nb) H[(kb + ty) * r + kb + tx] = tx <= ty ? A[ty][tx] : 0.0;
}

// Rows i >= kb + CH: H[i][kb .. kb+CH) <- H[i][kb .. kb+CH) L11^-T (one warp
// per row, forward substitution with lane = column).
__global__ void k_chol_panel(double* H, int64_t r, int64_t kb, const double* __restrict__ rdiag) {
  __shared__ double L11[CH][CH + 1];  // column CH: reciprocals of the pivots
  const int lane = threadIdx.x & 31;
  for (int t = threadIdx.x >> 5; t < CH; t += blockDim.x >> 5) L11[t][lane] = H[(kb + t) * r + kb + lane];
  if (threadIdx.x < CH) L11[threadIdx.x][CH] = rdiag[kb + threadIdx.x];
  __syncthreads();
  const int64_t i = kb + CH + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= r) return;
  double v = H[i * r + kb + lane];
  for (int c = 0; c < CH; ++c) {
    const double xc = __shfl_sync(0xffffffffu, v, c) * L11[c][CH];
    if (lane == c) v = xc;
    else if (lane > c) v -= L11[lane][c] * xc;
  }
  H[i * r + kb + lane] = v;
}

// H[i][j] -= sum_t L[i][kb+t] L[j][kb+t] for kb + CH <= j <= i < r, one CTA
// (one thread per entry) per UT x UT tile of the lower trailing matrix.
__global__ void __launch_bounds__(UT * UT) k_chol_update(double* H, int64_t r, int64_t kb) {
  __shared__ double Pi[UT][CH + 1], Pj[UT][CH + 1];
  const int64_t x = blockIdx.x;
  int64_t ti = (int64_t)((sqrt((double)(8 * x + 1)) - 1.0) / 2.0);
  while ((ti + 1) * (ti + 2) / 2 <= x) ++ti;
  while (ti * (ti + 1) / 2 > x) --ti;
  const int64_t tj = x - ti * (ti + 1) / 2;
  const int64_t i0 = kb + CH + ti * UT, j0 = kb + CH + tj * UT;
  const int tx = threadIdx.x % UT, ty = threadIdx.x / UT;
  for (int e = threadIdx.x; e < UT * CH; e += UT * UT) {
    const int q = e / CH, t = e % CH;
    Pi[q][t] = i0 + q < r ? H[(i0 + q) * r + kb + t] : 0.0;
    Pj[q][t] = j0 + q < r ? H[(j0 + q) * r + kb + t] : 0.0;
  }
  __syncthreads();
  const int64_t i = i0 + ty, j = j0 + tx;
  if (i < r && j <= i) {
    double acc = 0.0;
#pragma unroll 8
    for (int t = 0; t < CH; ++t) acc = fma(Pi[ty][t], Pj[tx][t], acc);
    H[i * r + j] -= acc;
  }
}

__global__ void k_transpose(const double* __restrict__ L, int64_t r, double* __restrict__ Lt) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < r * r; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t / r, b = t - a * r;
    Lt[t] = L[b * r + a];
  }
}

// Lane t of the warp ends with the sum over the 32 lanes of v[t].
__device__ __forceinline__ double warp_transpose_sum(double (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int c = 0; c < s; ++c) {
      const double send = up ? v[c] : v[c + s];
      const double keep = up ? v[c + s] : v[c];
      v[c] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

constexpr int SOLVE_WARPS = 4;

// A[i][:] = M[i][:] H^-1 (M given transposed, r x n; H = L L^T): forward
// L z = m_i, backward L^T a_i = z, one warp per row i, 32 unknowns at a
// time.  Per block the earlier unknowns' contribution is summed with lanes
// over the contracted index (coalesced rows of L or L^T, a transpose-reduce
// across the lanes), then the 32 x 32 triangle, staged in shared memory with
// the reciprocals of its pivots, is solved with shuffles.

// The 32 x 32 block of M (row-major, stride r) at (a0, a0) into B (pitch 33)
// and the reciprocals of its diagonal (rdiag) into column 32; one warp.
__device__ __forceinline__ void stage_block(const double* __restrict__ M, const double* __restrict__ rdiag, int64_t r,
                                            int64_t a0, int nb, double (*B)[33], int lane) {
  for (int t = 0; t < nb; ++t)
    if (lane < nb) B[t][lane] = M[(a0 + t) * r + a0 + lane];
  if (lane < nb) B[lane][32] = rdiag[a0 + lane];
  __syncwarp();
}
__global__ void __launch_bounds__(32 * SOLVE_WARPS)
    k_als_rowsolve(const double* __restrict__ L, const double* __restrict__ Lt, const double* __restrict__ rdiag,
                   const double* __restrict__ Mt, int64_t n, int64_t r, double* __restrict__ A) {
  extern __shared__ double ybuf[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * SOLVE_WARPS + w;
  if (i >= n) return;  // warp-uniform
  double(*B)[33] = reinterpret_cast<double(*)[33]>(ybuf + (size_t)SOLVE_WARPS * r) + w * 32;
  double* y = ybuf + (size_t)w * r;
  for (int64_t c = lane; c < r; c += 32) y[c] = Mt[c * n + i];
  __syncwarp();
  for (int64_t a0 = 0; a0 < r; a0 += 32) {
    const int nb = (int)(r - a0 < 32 ? r - a0 : 32);
    double acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0.0;
    for (int64_t q = lane; q < a0; q += 32) {
      const double yq = y[q];
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (t < nb) acc[t] = fma(L[(a0 + t) * r + q], yq, acc[t]);
    }
    double v = warp_transpose_sum(acc, lane);
    v = lane < nb ? y[a0 + lane] - v : 0.0;
    stage_block(L, rdiag, r, a0, nb, B, lane);
    for (int c = 0; c < nb; ++c) {
      const double xc = __shfl_sync(0xffffffffu, v, c) * B[c][32];
      if (lane == c) v = xc;
      else if (lane > c && lane < nb) v -= B[lane][c] * xc;
    }
    if (lane < nb) y[a0 + lane] = v;
    __syncwarp();
  }
  for (int64_t a0 = (r - 1) / 32 * 32; a0 >= 0; a0 -= 32) {
    const int nb = (int)(r - a0 < 32 ? r - a0 : 32);
    double acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0.0;
    for (int64_t q = a0 + nb + lane; q < r; q += 32) {
      const double yq = y[q];
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (t < nb) acc[t] = fma(Lt[(a0 + t) * r + q], yq, acc[t]);
    }
    double v = warp_transpose_sum(acc, lane);
    v = lane < nb ? y[a0 + lane] - v : 0.0;
    stage_block(Lt, rdiag, r, a0, nb, B, lane);
    for (int c = nb - 1; c >= 0; --c) {
      const double xc = __shfl_sync(0xffffffffu, v, c) * B[c][32];
      if (lane == c) v = xc;
      else if (lane < c) v -= B[lane][c] * xc;
    }
    if (lane < nb) {
      y[a0 + lane] = v;
      A[i * r + a0 + lane] = v;
    }
    __syncwarp();
  }
}

// Block b of ALS_PARTS: partial sums of <A, M> (A n x r, M^T r x n) into
// part[b] and of sum G0 o G1 o G2 (r x r) into part[ALS_PARTS + b], each in a
// fixed order.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}

__global__ void k_als_residual_parts(const double* __restrict__ A, const double* __restrict__ Mt, int64_t n, int64_t r,
                                     const double* __restrict__ G0, const double* __restrict__ G1,
                                     const double* __restrict__ G2, double* part) {
  __shared__ double sh[32];
  double ip = 0.0, kk = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * r; t += stride) {
    const int64_t i = t / r, a = t - i * r;
    ip = fma(A[t], Mt[a * n + i], ip);
  }
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < r * r; t += stride) kk += G0[t] * G1[t] * G2[t];
  const double s1 = block_sum(ip, sh);
  __syncthreads();
  const double s2 = block_sum(kk, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    part[ALS_PARTS + blockIdx.x] = s2;
  }
}

// ALS-skew factors from A1 = [A1_1 A1_2] (n x r) and B1 (n x h):
// A2 = [B1 B1], A3 = [A1_2, -A1_1].
__global__ void k_skew_derive(const double* __restrict__ A1, const double* __restrict__ B1, int64_t n, int64_t h,
                              double* __restrict__ A2, double* __restrict__ A3) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * h; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / h, a = t - i * h, r = 2 * h;
    if (A2) A2[i * r + a] = A2[i * r + h + a] = B1[t];
    if (A3) {
      A3[i * r + a] = A1[i * r + h + a];
      A3[i * r + h + a] = -A1[i * r + a];
    }
  }
}

// B1 = mean of the two halves of a fresh A2 update.
__global__ void k_skew_halves(const double* __restrict__ An, int64_t n, int64_t h, double* __restrict__ B1) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * h; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / h, a = t - i * h;
    B1[t] = 0.5 * (An[i * 2 * h + a] + An[i * 2 * h + h + a]);
  }
}

// A1 = lambda A1 + (1 - lambda) An.
__global__ void k_momentum(double* __restrict__ A1, const double* __restrict__ An, int64_t cnt, double lambda) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
    A1[t] = lambda * A1[t] + (1.0 - lambda) * An[t];
}

unsigned grid_for(int64_t cnt) {
  const int64_t b = (cnt + 255) / 256;
  return (unsigned)(b < 1 ? 1 : b > 4096 ? 4096 : b);
}

void als_free_fit(grom_als* s) {
  for (double*& p : s->f)
    if (p) cudaFree(p), p = nullptr;
  for (double*& p : s->gram)
    if (p) cudaFree(p), p = nullptr;
  for (double** p : {&s->anew, &s->b1, &s->mt, &s->h, &s->lt, &s->rdiag, &s->part})
    if (*p) cudaFree(*p), *p = nullptr;
  if (s->flag) cudaFree(s->flag), s->flag = nullptr;
  if (s->k2s) cudaFree(s->k2s), s->k2s = nullptr;
  s->rcap = 0;
  s->k2s_bytes = 0;
}

grom_status als_grow(grom_als* s, int64_t r) {
  // the split-K scratch of the MTTKRP is not monotonic in the rank: size it per fit
  const size_t need = k2_scratch_bytes(k2_plan(s->n, (int)r, s->sm_count));
  if (r <= s->rcap && need > s->k2s_bytes) {
    if (s->k2s) cudaFree(s->k2s);
    s->k2s = nullptr;
    if (cudaMalloc(&s->k2s, need) != cudaSuccess) {
      cudaGetLastError();
      als_free_fit(s);
      return fail(GROM_ERR_OOM, "grom_als_fit: device allocation");
    }
    s->k2s_bytes = need;
  }
  if (r <= s->rcap) return GROM_OK;
  als_free_fit(s);
  const size_t fb = (size_t)(s->n * r) * sizeof(double), gb = (size_t)(r * r) * sizeof(double);
  cudaError_t e = cudaSuccess;
  for (double*& p : s->f)
    if (e == cudaSuccess) e = cudaMalloc(&p, fb);
  for (double*& p : s->gram)
    if (e == cudaSuccess) e = cudaMalloc(&p, gb);
  if (e == cudaSuccess) e = cudaMalloc(&s->anew, fb);
  if (e == cudaSuccess) e = cudaMalloc(&s->b1, fb);
  if (e == cudaSuccess) e = cudaMalloc(&s->mt, fb);
  if (e == cudaSuccess) e = cudaMalloc(&s->h, gb);
  if (e == cudaSuccess) e = cudaMalloc(&s->lt, gb);
  if (e == cudaSuccess) e = cudaMalloc(&s->rdiag, (size_t)r * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->part, 2 * ALS_PARTS * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&s->k2s, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    als_free_fit(s);
    return fail(e == cudaErrorMemoryAllocation ? GROM_ERR_OOM : GROM_ERR_CUDA, "grom_als_fit: device allocation");
  }
  s->k2s_bytes = need;
  s->rcap = r;
  return GROM_OK;
}

// Gram matrix of factor q (on the device).
grom_status gram_of(grom_als* s, int q, int64_t r) {
  dim3 grid((unsigned)((r + 15) / 16), (unsigned)((r + 15) / 16));
  k_gram<<<grid, dim3(16, 16), 0, s->stream>>>(s->f[q], s->n, r, s->gram[q]);
  GROM_CUDA_TRY(cudaGetLastError());
  return GROM_OK;
}

// MTTKRP of layout m (0, 1, 2) with factors P (middle index) and Q (inner
// index) into s->mt (r x n).
grom_status mttkrp(grom_als* s, int m, int fp, int fq, int64_t r) {
  const K2Plan pl = k2_plan(s->n, (int)r, s->sm_count);
  K2Args a{};
  a.fp = s->f[fp];
  a.fq = s->f[fq];
  a.f_stride = r;
  a.batch = (int)r;
  a.c = s->mt;
  a.c_stride = s->n;
  a.scratch = s->k2s;
  a.err = s->err;
  a.ev0 = s->ev0;
  a.ev1 = s->ev1;
  GROM_CUDA_TRY(k2_launch(pl, &s->tmap[m], a, s->stream));
  GROM_CUDA_TRY(cudaStreamSynchronize(s->stream));
  float ms = 0.f;
  GROM_CUDA_TRY(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  s->mttkrp_ms += ms;
  ++s->mttkrp_calls;
  int flag = 0;
  GROM_CUDA_TRY(cudaMemcpy(&flag, s->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag & DEV_ERR_TIMEOUT) {
    cudaMemset(s->err, 0, sizeof(int));
    return fail(GROM_ERR_TIMEOUT, "grom_als_fit: a device-side wait timed out");
  }
  return GROM_OK;
}

// Cholesky of s->h in place (lower); false if a pivot broke down.
grom_status cholesky_dev(grom_als* s, int64_t r, bool* ok) {
  GROM_CUDA_TRY(cudaMemsetAsync(s->flag, 0, sizeof(int), s->stream));
  for (int64_t kb = 0; kb < r; kb += CH) {
    k_chol_diag<<<1, CH * CH, 0, s->stream>>>(s->h, r, kb, s->rdiag, s->flag);
    if (kb + CH < r) {
      const int64_t rows = r - kb - CH, m = (rows + UT - 1) / UT;
      k_chol_panel<<<(unsigned)((rows + 7) / 8), 256, 0, s->stream>>>(s->h, r, kb, s->rdiag);
      k_chol_update<<<(unsigned)(m * (m + 1) / 2), UT * UT, 0, s->stream>>>(s->h, r, kb);
    }
  }
  GROM_CUDA_TRY(cudaGetLastError());
  int flag = 0;
  GROM_CUDA_TRY(cudaMemcpyAsync(&flag, s->flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  GROM_CUDA_TRY(cudaStreamSynchronize(s->stream));
  *ok = flag == 0;
  return GROM_OK;
}

// The normal-equation update dst = M H^-1 (M = s->mt), H = Ga o Gb +
// ridge max diag(Ga o Gb) I.  If H is numerically singular (ALS on a tensor
// dominated by a few components drives the factor columns towards each
// other), retry with an extra mu max diag I, mu = 1e-12 growing 100x up to
// three times.
grom_status ls_update(grom_als* s, const double* Ga, const double* Gb, int64_t r, double ridge, double* dst) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = s->n;
  bool ok = false;
  double mu = 0.0;
  grom_status st;
  for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
    k_als_normal<<<grid_for(r * r), 256, 0, s->stream>>>(Ga, Gb, r, ridge + mu, s->h);
    if ((st = cholesky_dev(s, r, &ok))) return st;
    mu = mu == 0.0 ? 1e-12 : mu * 100.0;
  }
  if (!ok) return fail(GROM_ERR_INVALID_ARG, "grom_als_fit: a Gram matrix is not positive definite");
  k_transpose<<<grid_for(r * r), 256, 0, s->stream>>>(s->h, r, s->lt);
  const size_t smem = (size_t)SOLVE_WARPS * (r + 32 * 33) * sizeof(double);
  if (smem > 48 * 1024)
    GROM_CUDA_TRY(cudaFuncSetAttribute(k_als_rowsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_als_rowsolve<<<(unsigned)((n + SOLVE_WARPS - 1) / SOLVE_WARPS), 32 * SOLVE_WARPS, smem, s->stream>>>(
      s->h, s->lt, s->rdiag, s->mt, n, r, dst);
  GROM_CUDA_TRY(cudaGetLastError());
  GROM_CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->solve_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return GROM_OK;
}

// Relative residual ||X - [[A1, A2, A3]]|| / ||X|| from <X, K> = <A1, M_1>
// (s->mt holds the mode-1 MTTKRP of the current factors) and
// ||K||^2 = sum G1 o G2 o G3.
grom_status residual_of(grom_als* s, int64_t r, double* out) {
  k_als_residual_parts<<<ALS_PARTS, 256, 0, s->stream>>>(s->f[0], s->mt, s->n, r, s->gram[0], s->gram[1], s->gram[2],
                                                        s->part);
  GROM_CUDA_TRY(cudaGetLastError());
  double ph[2 * ALS_PARTS];
  GROM_CUDA_TRY(cudaMemcpyAsync(ph, s->part, sizeof(ph), cudaMemcpyDeviceToHost, s->stream));
  GROM_CUDA_TRY(cudaStreamSynchronize(s->stream));
  double ip = 0.0, kk = 0.0;
  for (int q = 0; q < ALS_PARTS; ++q) {
    ip += ph[q];
    kk += ph[ALS_PARTS + q];
  }
  const double r2 = s->xnorm2 - 2.0 * ip + kk;
  *out = std::sqrt(std::max(r2, 0.0) / s->xnorm2);
  return GROM_OK;
}

grom_status copy(grom_als* s, void* dst, const void* src, size_t bytes) {
  GROM_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s->stream));
  GROM_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return GROM_OK;
}

}  // namespace

extern "C" {

grom_status grom_als_create(int32_t n, const double* tensor, void* stream, grom_als** out) {
  if (!tensor || !out || n < 1) return fail(GROM_ERR_INVALID_ARG, "grom_als_create: bad argument");
  *out = nullptr;
  if (n > grom_max_n(GROM_FORM_FULL, GROM_BF16))
    return fail(GROM_ERR_UNSUPPORTED, "grom_als_create: n exceeds the BF16 row limit");
  grom_als* s = new (std::nothrow) grom_als();
  if (!s) return fail(GROM_ERR_OOM, "grom_als_create: host allocation");
  s->n = n;
  s->np = padded_n(n);
  s->stream = static_cast<cudaStream_t>(stream);
  int dev = 0;
  auto bail = [&](grom_status st) {
    grom_als_destroy(s);
    return st;
  };
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(GROM_ERR_CUDA, "grom_als_create: no usable CUDA device"));
  }
  const size_t lbytes = (size_t)n * n * s->np * sizeof(__nv_bfloat16);
  for (auto& x : s->x) {
    if (cudaMalloc(&x, lbytes) != cudaSuccess || cudaMemsetAsync(x, 0, lbytes, s->stream) != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(GROM_ERR_OOM, "grom_als_create: device allocation"));
    }
  }
  if (cudaMalloc(&s->err, sizeof(int)) != cudaSuccess || cudaMemsetAsync(s->err, 0, sizeof(int), s->stream) != cudaSuccess)
    return bail(fail(GROM_ERR_OOM, "grom_als_create: device allocation"));
  if (cudaEventCreate(&s->ev0) != cudaSuccess || cudaEventCreate(&s->ev1) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "grom_als_create: events"));
  // stream the FP64 tensor through a staging buffer by test index
  const int64_t per_i = (int64_t)n * n;
  const int64_t si = std::min<int64_t>(n, std::max<int64_t>(1, (int64_t)(256ll << 20) / (per_i * 8)));
  double *stage = nullptr, *part = nullptr;
  constexpr int NB = 1024;
  if (cudaMalloc(&stage, (size_t)(si * per_i * 8)) != cudaSuccess || cudaMalloc(&part, NB * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    if (stage) cudaFree(stage);
    return bail(fail(GROM_ERR_OOM, "grom_als_create: staging allocation"));
  }
  std::vector<double> ph(NB);
  double norm2 = 0.0;
  cudaError_t e = cudaSuccess;
  for (int64_t a = 0; e == cudaSuccess && a < n; a += si) {
    const int64_t cnt = std::min(si, (int64_t)n - a);
    e = cudaMemcpyAsync(stage, tensor + a * per_i, (size_t)(cnt * per_i * 8), cudaMemcpyDefault, s->stream);
    if (e != cudaSuccess) break;
    int64_t blocks = std::min<int64_t>(65536, (cnt * per_i + 255) / 256);
    k_als_x12<<<(unsigned)blocks, 256, 0, s->stream>>>(stage, cnt, n, s->np, a, reinterpret_cast<__nv_bfloat16*>(s->x[0]),
                                                       reinterpret_cast<__nv_bfloat16*>(s->x[1]));
    dim3 g3((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32), (unsigned)cnt);
    k_als_x3<<<g3, dim3(32, 8), 0, s->stream>>>(stage, n, s->np, a, reinterpret_cast<__nv_bfloat16*>(s->x[2]));
    k_als_norm<<<NB, 256, 0, s->stream>>>(stage, cnt * per_i, part);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(ph.data(), part, NB * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    for (int q = 0; q < NB; ++q) norm2 += ph[q];
  }
  cudaFree(stage);
  cudaFree(part);
  if (e != cudaSuccess) return bail(cuda_fail(e, "grom_als_create: tensor upload"));
  s->xnorm2 = norm2;
  for (int q = 0; q < 3; ++q)
    if (!k2_make_tmap(&s->tmap[q], s->x[q], n, s->np))
      return bail(fail(GROM_ERR_UNSUPPORTED, "grom_als_create: tensor map encoding failed"));
  *out = s;
  return GROM_OK;
}

grom_status grom_als_fit(grom_als* s, int32_t rank, int32_t method, int32_t iters, double lambda, int32_t subiters,
                         double ridge, double* fa, double* fb, double* fc, double* residual) {
  TraceRange trace("grom_als_fit");
  if (!s || !fa || !fb || rank < 1 || iters < 0 || !(ridge >= 0.0))
    return fail(GROM_ERR_INVALID_ARG, "grom_als_fit: bad argument");
  if (method != GROM_ALS_PLAIN && method != GROM_ALS_SKEW) return fail(GROM_ERR_INVALID_ARG, "grom_als_fit: bad method");
  if (method == GROM_ALS_PLAIN && !fc) return fail(GROM_ERR_INVALID_ARG, "grom_als_fit: fc is NULL");
  if (method == GROM_ALS_SKEW && (rank % 2 || subiters < 1 || !(lambda >= 0.0 && lambda < 1.0)))
    return fail(GROM_ERR_INVALID_ARG, "grom_als_fit: ALS-skew needs an even rank, subiters >= 1, 0 <= lambda < 1");
  const int64_t n = s->n, r = rank, h = r / 2;
  grom_status st = als_grow(s, r);
  if (st) return st;
  const size_t fbytes = (size_t)(n * r) * sizeof(double);
  if (method == GROM_ALS_PLAIN) {
    if ((st = copy(s, s->f[0], fa, fbytes)) || (st = copy(s, s->f[1], fb, fbytes)) ||
        (st = copy(s, s->f[2], fc, fbytes)))
      return st;
    for (int q = 0; q < 3; ++q)
      if ((st = gram_of(s, q, r))) return st;
    for (int it = 0; it < iters; ++it) {
      for (int m = 0; m < 3; ++m) {
        // layout m: rows of mode m; P, Q = the factors of its middle and inner index
        const int fp = m == 0 ? 1 : 0, fq = m == 2 ? 1 : 2;
        if ((st = mttkrp(s, m, fp, fq, r)) || (st = ls_update(s, s->gram[fp], s->gram[fq], r, ridge, s->f[m])) ||
            (st = gram_of(s, m, r)))
          return st;
      }
      // <X, K> from a fresh mode-1 MTTKRP with the final factors: the M the
      // last update used carries the noise that update amplified along the
      // near-null directions of its normal matrix, and would hide it
      if (residual && ((st = mttkrp(s, 0, 1, 2, r)) || (st = residual_of(s, r, &residual[it])))) return st;
    }
    if ((st = copy(s, fa, s->f[0], fbytes)) || (st = copy(s, fb, s->f[1], fbytes)) || (st = copy(s, fc, s->f[2], fbytes)))
      return st;
    return GROM_OK;
  }
  // ALS-skew: A1 = [A1_1 A1_2] (factor 0), A2 = [B1 B1], A3 = [A1_2, -A1_1]
  const unsigned gh = grid_for(n * h);
  if ((st = copy(s, s->f[0], fa, fbytes)) || (st = copy(s, s->b1, fb, (size_t)(n * h) * sizeof(double)))) return st;
  k_skew_derive<<<gh, 256, 0, s->stream>>>(s->f[0], s->b1, n, h, s->f[1], s->f[2]);
  GROM_CUDA_TRY(cudaGetLastError());
  for (int q = 0; q < 3; ++q)
    if ((st = gram_of(s, q, r))) return st;
  for (int it = 0; it < iters; ++it) {
    // A2 as in ALS (layout X2: P = A1, Q = A3), halves averaged
    if ((st = mttkrp(s, 1, 0, 2, r)) || (st = ls_update(s, s->gram[0], s->gram[2], r, ridge, s->anew))) return st;
    k_skew_halves<<<gh, 256, 0, s->stream>>>(s->anew, n, h, s->b1);
    k_skew_derive<<<gh, 256, 0, s->stream>>>(s->f[0], s->b1, n, h, s->f[1], nullptr);
    GROM_CUDA_TRY(cudaGetLastError());
    if ((st = gram_of(s, 1, r))) return st;
    for (int sub = 0; sub < subiters; ++sub) {
      // A1_next with A2, A3 fixed (layout X1: P = A2, Q = A3), then momentum
      if ((st = mttkrp(s, 0, 1, 2, r)) || (st = ls_update(s, s->gram[1], s->gram[2], r, ridge, s->anew))) return st;
      k_momentum<<<grid_for(n * r), 256, 0, s->stream>>>(s->f[0], s->anew, n * r, lambda);
      k_skew_derive<<<gh, 256, 0, s->stream>>>(s->f[0], s->b1, n, h, nullptr, s->f[2]);
      GROM_CUDA_TRY(cudaGetLastError());
      if ((st = gram_of(s, 0, r)) || (st = gram_of(s, 2, r))) return st;
    }
    if (residual && ((st = mttkrp(s, 0, 1, 2, r)) || (st = residual_of(s, r, &residual[it])))) return st;
  }
  if ((st = copy(s, fa, s->f[0], fbytes)) || (st = copy(s, fb, s->b1, (size_t)(n * h) * sizeof(double)))) return st;
  return GROM_OK;
}

grom_status grom_als_stats(grom_als* s, double* mttkrp_ms, int64_t* mttkrp_calls, double* solve_ms) {
  if (!s || !mttkrp_ms || !mttkrp_calls || !solve_ms) return fail(GROM_ERR_INVALID_ARG, "grom_als_stats: null argument");
  *mttkrp_ms = s->mttkrp_ms;
  *mttkrp_calls = s->mttkrp_calls;
  *solve_ms = s->solve_ms;
  s->mttkrp_ms = s->solve_ms = 0.0;
  s->mttkrp_calls = 0;
  return GROM_OK;
}

grom_status grom_als_destroy(grom_als* s) {
  if (!s) return GROM_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->ev0) cudaEventDestroy(s->ev0);
  if (s->ev1) cudaEventDestroy(s->ev1);
  for (auto p : s->x)
    if (p) cudaFree(p);
  als_free_fit(s);
  if (s->err) cudaFree(s->err);
  delete s;
  return GROM_OK;
}

}  // extern "C"
