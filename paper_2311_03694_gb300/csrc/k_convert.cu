// One-time conversion of FP64 operators into the device storage layouts.
#include "grom_internal.h"

namespace grom {

// rows x n doubles -> rows x np stored elements (k padded with zeros).
// F32X2 rows are [hi(np floats) | lo(np floats)] with hi = rn(x),
// lo = rn(x - hi).
__global__ void k_convert_rows(const double* __restrict__ src, int64_t rows, int64_t n, int64_t np, int storage,
                               uint8_t* __restrict__ dst) {
  const int64_t total = rows * np;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / np, k = t - r * np;
    const double x = k < n ? src[r * n + k] : 0.0;
    switch (storage) {
      case GROM_F64:
        reinterpret_cast<double*>(dst)[t] = x;
        break;
      case GROM_F32X2: {
        const float hi = __double2float_rn(x);
        const float lo = __double2float_rn(x - (double)hi);
        float* row = reinterpret_cast<float*>(dst) + r * 2 * np;
        row[k] = hi;
        row[np + k] = lo;
        break;
      }
      case GROM_F32:
        reinterpret_cast<float*>(dst)[t] = __double2float_rn(x);
        break;
      case GROM_BF16:
        reinterpret_cast<__nv_bfloat16*>(dst)[t] = __double2bfloat16(x);
        break;
    }
  }
}

cudaError_t convert_rows_launch(const double* src, int64_t rows, int64_t n, int64_t np, int storage, uint8_t* dst,
                                cudaStream_t s) {
  const int64_t total = rows * np;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  if (blocks < 1) blocks = 1;
  k_convert_rows<<<(unsigned)blocks, 256, 0, s>>>(src, rows, n, np, storage, dst);
  return cudaGetLastError();
}

// Dense FP64 rows (i, j), i from i0, -> skew-packed rows of lp elements:
// position p < h = n/2 holds C[i][j][(i + 1 + p) mod n], except that for
// even n the distance n/2 is kept only in rows with i < n/2; other
// positions are zero.  Same rounding and F32X2 planes as k_convert_rows.
__global__ void k_convert_rows_packed(const double* __restrict__ src, int64_t rows, int64_t n, int64_t m, int64_t i0,
                                      int64_t lp, int storage, uint8_t* __restrict__ dst) {
  const int64_t total = rows * lp, h = n / 2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / lp, p = t - r * lp;
    const int64_t i = i0 + r / m;
    double x = 0.0;
    if (p < h && !((n % 2 == 0) && p == h - 1 && i >= h)) {
      int64_t k = i + 1 + p;
      if (k >= n) k -= n;
      x = src[r * n + k];
    }
    switch (storage) {
      case GROM_F64:
        reinterpret_cast<double*>(dst)[t] = x;
        break;
      case GROM_F32X2: {
        const float hi = __double2float_rn(x);
        const float lo = __double2float_rn(x - (double)hi);
        float* row = reinterpret_cast<float*>(dst) + r * 2 * lp;
        row[p] = hi;
        row[lp + p] = lo;
        break;
      }
      case GROM_F32:
        reinterpret_cast<float*>(dst)[t] = __double2float_rn(x);
        break;
      case GROM_BF16:
        reinterpret_cast<__nv_bfloat16*>(dst)[t] = __double2bfloat16(x);
        break;
    }
  }
}

cudaError_t convert_rows_packed_launch(const double* src, int64_t rows, int64_t n, int64_t m, int64_t i0, int64_t lp,
                                       int storage, uint8_t* dst, cudaStream_t s) {
  const int64_t total = rows * lp;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  if (blocks < 1) blocks = 1;
  k_convert_rows_packed<<<(unsigned)blocks, 256, 0, s>>>(src, rows, n, m, i0, lp, storage, dst);
  return cudaGetLastError();
}

// Seeded +-1 entries of the probe vectors (a fixed integer hash of the index
// and the probe number; any fixed choice works).
__device__ __forceinline__ double probe_sign(int64_t idx, uint32_t salt) {
  uint64_t z = (uint64_t)idx * 0x9E3779B97F4A7C15ull + salt;
  z ^= z >> 31;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 29;
  return (z >> 40) & 1 ? 1.0 : -1.0;
}

// For a skew tensor (C_ijk = -C_kji) sum_ijk x_i y_j x_k C_ijk vanishes for
// every x, y.  One warp per row (i, j) (m rows per test index): adds
// x_i y_j sum_k C_ijk x_k for two (x, y) pairs and sum_k C_ijk^2 into acc[0..2].
__global__ void k_skew_probe(const double* __restrict__ src, int64_t rows, int64_t n, int64_t m, int64_t i0,
                             double* acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  double p1 = 0.0, p2 = 0.0, sq = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const int64_t i = i0 + r / m, j = r % m;
    double s1 = 0.0, s2 = 0.0, q = 0.0;
    for (int64_t k = lane; k < n; k += 32) {
      const double c = src[r * n + k];
      s1 = fma(c, probe_sign(k, 1u), s1);
      s2 = fma(c, probe_sign(k, 3u), s2);
      q = fma(c, c, q);
    }
    p1 = fma(probe_sign(i, 1u) * probe_sign(j, 2u), s1, p1);
    p2 = fma(probe_sign(i, 3u) * probe_sign(j, 4u), s2, p2);
    sq += q;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    p1 += __shfl_xor_sync(0xffffffffu, p1, off);
    p2 += __shfl_xor_sync(0xffffffffu, p2, off);
    sq += __shfl_xor_sync(0xffffffffu, sq, off);
  }
  if (lane == 0) {
    atomicAdd(acc, p1);
    atomicAdd(acc + 1, p2);
    atomicAdd(acc + 2, sq);
  }
}

cudaError_t skew_probe_launch(const double* src, int64_t rows, int64_t n, int64_t m, int64_t i0, double* acc,
                              cudaStream_t s) {
  int64_t blocks = (rows + 7) / 8;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_skew_probe<<<(unsigned)blocks, 256, 0, s>>>(src, rows, n, m, i0, acc);
  return cudaGetLastError();
}

// Splits an augmented tensor slab into its core rows and zeroth-mode terms
// (eq. zeroth_contribution); see grom_desc.augmented.
__global__ void k_aug_split(const double* __restrict__ src, int64_t cnt, int64_t n, double* __restrict__ core,
                            double* __restrict__ L, double* __restrict__ f) {
  const int64_t n1 = n + 1, total = cnt * n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / (n * n), rem = t - i * n * n, j = rem / n, k = rem - j * n;
    const double* Ci = src + i * n1 * n1;
    core[t] = Ci[(j + 1) * n1 + k + 1];
    if (j == 0) {
      L[i * n + k] = Ci[k + 1] + Ci[(k + 1) * n1];
      if (k == 0) f[i] = Ci[0];
    }
  }
}

cudaError_t aug_split_launch(const double* src, int64_t cnt, int64_t n, double* core, double* L, double* f,
                             cudaStream_t s) {
  const int64_t total = cnt * n * n;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  if (blocks < 1) blocks = 1;
  k_aug_split<<<(unsigned)blocks, 256, 0, s>>>(src, cnt, n, core, L, f);
  return cudaGetLastError();
}

// n x r doubles -> n x rp stored elements (rank padded with zero columns).
cudaError_t convert_panels_launch(const double* src, int64_t n, int64_t r, int64_t rp, int storage, uint8_t* dst,
                                  cudaStream_t s) {
  return convert_rows_launch(src, n, r, rp, storage, dst, s);
}

}  // namespace grom
