// K3: CP-form advection term (Sec. 3.1, eq. tc_ap; skew structure Sec. 3.3,
// eq. skew_abc_struct).
//
//   general:  p = B^T u,  q = C^T u,            c = A (p o q)
//   skew:     p = V^T u,  q = W^T u,  s = U^T u,  c = U (p o q) - W (p o s)
//
// The skew form is the expanded rank-2R model A1 = [U W], A2 = [V V],
// A3 = [W -U] evaluated without materialising the repeated blocks.
//
// Factors are stored row-major n x rp (rank padded with zero columns to a
// multiple of 8).  Three launches per pass:
//   project  grid (column tiles of 64) x (row slices): each warp streams rows of
//            its slice with coalesced 64-column loads; partial sums per slice.
//   combine  sums the slices in fixed order and forms the Hadamard products.
//   expand   one warp per test index: c_i = sum_r A_ir h1_r (- W_ir h2_r).
#include "grom_internal.h"

namespace grom {

constexpr int K3_COLS = 64;   // columns per project CTA (2 per lane)
constexpr int K3_WARPS = 8;

template <int ST>
struct K3T;
template <>
struct K3T<GROM_F64> {
  using acc_t = double;
  static __device__ __forceinline__ void load2(const uint8_t* base, int64_t idx, double& x0, double& x1) {
    const double2 v = *reinterpret_cast<const double2*>(base + idx * 8);
    x0 = v.x;
    x1 = v.y;
  }
  static __device__ __forceinline__ double load1(const uint8_t* base, int64_t idx) {
    return reinterpret_cast<const double*>(base)[idx];
  }
  static __device__ __forceinline__ double cvt_u(double v) { return v; }
};
template <>
struct K3T<GROM_F32> {
  using acc_t = float;
  static __device__ __forceinline__ void load2(const uint8_t* base, int64_t idx, float& x0, float& x1) {
    const float2 v = *reinterpret_cast<const float2*>(base + idx * 4);
    x0 = v.x;
    x1 = v.y;
  }
  static __device__ __forceinline__ float load1(const uint8_t* base, int64_t idx) {
    return reinterpret_cast<const float*>(base)[idx];
  }
  static __device__ __forceinline__ float cvt_u(double v) { return __double2float_rn(v); }
};
template <>
struct K3T<GROM_BF16> {
  using acc_t = float;
  static __device__ __forceinline__ void load2(const uint8_t* base, int64_t idx, float& x0, float& x1) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(base + idx * 2);
    x0 = __uint_as_float(w << 16);
    x1 = __uint_as_float(w & 0xffff0000u);
  }
  static __device__ __forceinline__ float load1(const uint8_t* base, int64_t idx) {
    const uint16_t h = reinterpret_cast<const uint16_t*>(base)[idx];
    return __uint_as_float((uint32_t)h << 16);
  }
  static __device__ __forceinline__ float cvt_u(double v) { return __double2float_rn(v); }
};

struct K3Shape {
  int64_t n, rp;
  int slices;
  int nf;  // projected factors: 2 (general) or 3 (skew)
};

__device__ __forceinline__ const double* k3_u_ptr(const K3Args& a, int bg, int64_t n) {
  return a.taken ? a.hist + bg * a.hist_stride + (a.taken[bg] % 3) * n : a.u + bg * a.u_stride;
}

// partial layout: [slice][f][b][rp] in acc_t
template <int ST, int NB>
__global__ void __launch_bounds__(256) k3_project_kernel(const K3Shape sh, const K3Args a, const int b0,
                                                         void* partial) {
  using T = K3T<ST>;
  using acc_t = typename T::acc_t;
  __shared__ acc_t red[K3_WARPS][3][NB][K3_COLS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = sh.n, rp = sh.rp;
  const int64_t col = (int64_t)blockIdx.x * K3_COLS + 2 * lane;
  const int slice = blockIdx.y;
  const int64_t i0 = (int64_t)slice * n / sh.slices, i1 = ((int64_t)slice + 1) * n / sh.slices;
  // projected factors in order: general (fb, fc); skew (fb, fc, fa)
  const uint8_t* F[3] = {a.fb, a.fc, a.fa};
  acc_t acc[3][NB][2];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[f][b][0] = acc[f][b][1] = acc_t(0);
  const bool in = col < rp;
  const double* ub[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) ub[b] = (b < a.nb) ? k3_u_ptr(a, b0 + b, n) : nullptr;
  for (int64_t i = i0 + warp; i < i1; i += K3_WARPS) {
    acc_t ui[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const bool on = b < a.nb && (a.active == nullptr || a.active[b0 + b]);
      ui[b] = on ? T::cvt_u(ub[b][i]) : acc_t(0);
    }
    if (in) {
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        if (f < sh.nf) {
          acc_t x0, x1;
          T::load2(F[f], i * rp + col, x0, x1);
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            acc[f][b][0] = fma(x0, ui[b], acc[f][b][0]);
            acc[f][b][1] = fma(x1, ui[b], acc[f][b][1]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      red[warp][f][b][2 * lane] = acc[f][b][0];
      red[warp][f][b][2 * lane + 1] = acc[f][b][1];
    }
  __syncthreads();
  acc_t* out = reinterpret_cast<acc_t*>(partial);
  for (int t = threadIdx.x; t < sh.nf * NB * K3_COLS; t += blockDim.x) {
    const int f = t / (NB * K3_COLS), b = (t / K3_COLS) % NB, cc = t % K3_COLS;
    const int64_t c = (int64_t)blockIdx.x * K3_COLS + cc;
    if (c >= rp) continue;
    acc_t s = acc_t(0);
#pragma unroll
    for (int w = 0; w < K3_WARPS; ++w) s += red[w][f][b][cc];
    out[(((int64_t)slice * sh.nf + f) * NB + b) * rp + c] = s;
  }
}

// h layout: [2][b][rp]: h1 = p o q, h2 = p o s (skew only)
template <int ST, int NB>
__global__ void k3_combine_kernel(const K3Shape sh, const K3Args a, const void* partial, void* hbuf) {
  using acc_t = typename K3T<ST>::acc_t;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rp = sh.rp;
  if (t >= (int64_t)NB * rp) return;
  const int b = (int)(t / rp);
  const int64_t r = t - (int64_t)b * rp;
  const acc_t* P = reinterpret_cast<const acc_t*>(partial);
  acc_t v[3] = {acc_t(0), acc_t(0), acc_t(0)};
  for (int s = 0; s < sh.slices; ++s)
    for (int f = 0; f < sh.nf; ++f) v[f] += P[(((int64_t)s * sh.nf + f) * NB + b) * rp + r];
  acc_t* h = reinterpret_cast<acc_t*>(hbuf);
  h[(int64_t)b * rp + r] = v[0] * v[1];
  if (sh.nf == 3) h[((int64_t)NB + b) * rp + r] = v[0] * v[2];
}

template <int ST, int NB>
__global__ void __launch_bounds__(256) k3_expand_kernel(const K3Shape sh, const K3Args a, const int b0,
                                                        const void* hbuf) {
  using T = K3T<ST>;
  using acc_t = typename T::acc_t;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * K3_WARPS + warp;
  const int64_t n = sh.n, rp = sh.rp;
  if (i >= n) return;
  const acc_t* h = reinterpret_cast<const acc_t*>(hbuf);
  acc_t acc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) acc[b] = acc_t(0);
  for (int64_t r = 2 * lane; r < rp; r += 64) {
    acc_t x0, x1;
    T::load2(a.fa, i * rp + r, x0, x1);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      acc[b] = fma(x0, h[(int64_t)b * rp + r], acc[b]);
      acc[b] = fma(x1, h[(int64_t)b * rp + r + 1], acc[b]);
    }
    if (sh.nf == 3) {
      T::load2(a.fc, i * rp + r, x0, x1);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        acc[b] = fma(-x0, h[((int64_t)NB + b) * rp + r], acc[b]);
        acc[b] = fma(-x1, h[((int64_t)NB + b) * rp + r + 1], acc[b]);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    acc_t v = acc[b];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    acc[b] = v;
  }
  if (lane < NB) {
    const int b = lane;
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (q == b) v = (double)acc[q];
    const int bg = b0 + b;
    if (b < a.nb && (a.active == nullptr || a.active[bg])) {
      double* dst = a.taken ? a.hist + bg * a.hist_stride + (3 + a.taken[bg] % 3) * n : a.c + bg * a.c_stride;
      dst[i] = v;
    }
  }
}

K3Plan k3_plan(int64_t n, int64_t r, int storage, int sm_count) {
  K3Plan p{};
  p.n = n;
  p.r = r;
  p.rb = (r + 7) / 8 * 8;  // padded rank (row pitch of the stored factors)
  const int64_t tiles = (p.rb + K3_COLS - 1) / K3_COLS;
  int64_t slices = (2 * sm_count + tiles - 1) / tiles;
  const int64_t max_slices = (n + 31) / 32;  // keep >= 32 rows per slice
  if (slices > max_slices) slices = max_slices;
  if (slices < 1) slices = 1;
  p.nblk = slices;
  p.nb_max = 4;
  (void)storage;
  return p;
}

size_t k3_scratch_bytes(const K3Plan& p, int storage) {
  const size_t es = storage == GROM_F64 ? 8 : 4;
  return es * (size_t)p.rb * (size_t)p.nb_max * (3 * (size_t)p.nblk + 2);
}

template <int ST, int NB>
static cudaError_t k3_run(const K3Plan& p, const K3Args& a, int b0, cudaStream_t s) {
  K3Shape sh{p.n, p.rb, (int)p.nblk, a.form == GROM_FORM_CP_SKEW ? 3 : 2};
  using acc_t = typename K3T<ST>::acc_t;
  void* partial = a.part;
  void* hbuf = reinterpret_cast<uint8_t*>(a.part) + sizeof(acc_t) * (size_t)p.rb * NB * 3 * p.nblk;
  dim3 g1((unsigned)((p.rb + K3_COLS - 1) / K3_COLS), (unsigned)p.nblk);
  k3_project_kernel<ST, NB><<<g1, 256, 0, s>>>(sh, a, b0, partial);
  k3_combine_kernel<ST, NB><<<(unsigned)((NB * p.rb + 255) / 256), 256, 0, s>>>(sh, a, partial, hbuf);
  k3_expand_kernel<ST, NB><<<(unsigned)((p.n + K3_WARPS - 1) / K3_WARPS), 256, 0, s>>>(sh, a, b0, hbuf);
  return cudaGetLastError();
}

template <int ST>
static cudaError_t k3_nb(int nb, const K3Plan& p, const K3Args& a, int b0, cudaStream_t s) {
  switch (nb) {
    case 1: return k3_run<ST, 1>(p, a, b0, s);
    case 2: return k3_run<ST, 2>(p, a, b0, s);
    case 4: return k3_run<ST, 4>(p, a, b0, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t k3_launch(const K3Plan& p, int storage, const K3Args& a0, int batch, cudaStream_t s) {
  for (int b0 = 0; b0 < batch; b0 += p.nb_max) {
    K3Args a = a0;
    a.nb = batch - b0 < p.nb_max ? batch - b0 : p.nb_max;
    const int nb = a.nb == 1 ? 1 : a.nb == 2 ? 2 : 4;
    cudaError_t e;
    switch (storage) {
      case GROM_F64: e = k3_nb<GROM_F64>(nb, p, a, b0, s); break;
      case GROM_F32: e = k3_nb<GROM_F32>(nb, p, a, b0, s); break;
      case GROM_BF16: e = k3_nb<GROM_BF16>(nb, p, a, b0, s); break;
      default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace grom
