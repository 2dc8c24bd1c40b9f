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

// n x r doubles -> n x rp stored elements (rank padded with zero columns).
cudaError_t convert_panels_launch(const double* src, int64_t n, int64_t r, int64_t rp, int storage, uint8_t* dst,
                                  cudaStream_t s) {
  return convert_rows_launch(src, n, r, rp, storage, dst, s);
}

}  // namespace grom
