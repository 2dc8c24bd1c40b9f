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
// The Gram matrices are FP64 on the device; the rank x rank SPD solves are
// FP64 Cholesky on the host (rank^3/3 + 2 n rank^2 flops per update).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "grom_internal.h"

using namespace grom;

struct grom_als {
  int64_t n = 0, np = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  uint8_t* x[3] = {nullptr, nullptr, nullptr};  // BF16 layouts X1, X2, X3
  CUtensorMap tmap[3];
  double xnorm2 = 0.0;  // ||X||_F^2 of the BF16 tensor the fit sees
  int* err = nullptr;
  // per-fit buffers (grown on demand)
  int64_t rcap = 0;
  double* f[3] = {nullptr, nullptr, nullptr};  // factors on the device, n x rank FP64
  double* mt = nullptr;                        // MTTKRP output, rank x n FP64
  double* gram = nullptr;                      // rank x rank FP64
  void* k2s = nullptr;
  size_t k2s_bytes = 0;
  // timing since the last grom_als_stats: MTTKRP device time (CUDA events
  // around each tensor-core launch) and host time of the SPD solves
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

// G = F^T F for F (n x r, row-major FP64), 16 x 16 output tiles.
__global__ void k_gram(const double* __restrict__ F, int64_t n, int64_t r, double* __restrict__ G) {
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
  if (row < r && col < r) G[row * r + col] = s;
}

// Cholesky factor of the SPD matrix H (r x r, row-major) in place (lower).
bool cholesky(std::vector<double>& H, int64_t r) {
  for (int64_t j = 0; j < r; ++j) {
    double d = H[j * r + j];
    for (int64_t q = 0; q < j; ++q) d -= H[j * r + q] * H[j * r + q];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    d = std::sqrt(d);
    H[j * r + j] = d;
    for (int64_t i = j + 1; i < r; ++i) {
      double s = H[i * r + j];
      for (int64_t q = 0; q < j; ++q) s -= H[i * r + q] * H[j * r + q];
      H[i * r + j] = s / d;
    }
  }
  return true;
}

// A[i][:] = H^{-1} M[i][:] for every row i, with M given transposed (Mt,
// r x n) and H = L L^T; rows in parallel.
void solve_rows(const std::vector<double>& L, int64_t r, const std::vector<double>& Mt, int64_t n,
                std::vector<double>& A) {
  A.assign((size_t)(n * r), 0.0);
  const int nt = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), 32));
  auto work = [&](int tid) {
    std::vector<double> y((size_t)r);
    for (int64_t i = tid; i < n; i += nt) {
      for (int64_t a = 0; a < r; ++a) {
        double s = Mt[a * n + i];
        for (int64_t q = 0; q < a; ++q) s -= L[a * r + q] * y[q];
        y[a] = s / L[a * r + a];
      }
      for (int64_t a = r - 1; a >= 0; --a) {
        double s = y[a];
        for (int64_t q = a + 1; q < r; ++q) s -= L[q * r + a] * A[i * r + q];
        A[i * r + a] = s / L[a * r + a];
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& t : th) t.join();
}

grom_status als_grow(grom_als* s, int64_t r) {
  // the split-K scratch of the MTTKRP is not monotonic in the rank: size it per fit
  const size_t need = k2_scratch_bytes(k2_plan(s->n, (int)r, s->sm_count));
  if (r <= s->rcap && need > s->k2s_bytes) {
    if (s->k2s) cudaFree(s->k2s);
    s->k2s = nullptr;
    if (cudaMalloc(&s->k2s, need) != cudaSuccess) {
      cudaGetLastError();
      s->rcap = 0;
      return fail(GROM_ERR_OOM, "grom_als_fit: device allocation");
    }
    s->k2s_bytes = need;
  }
  if (r <= s->rcap) return GROM_OK;
  for (double*& p : s->f)
    if (p) cudaFree(p), p = nullptr;
  if (s->mt) cudaFree(s->mt), s->mt = nullptr;
  if (s->gram) cudaFree(s->gram), s->gram = nullptr;
  if (s->k2s) cudaFree(s->k2s), s->k2s = nullptr;
  s->rcap = 0;
  const size_t fb = (size_t)(s->n * r) * sizeof(double);
  cudaError_t e = cudaSuccess;
  for (double*& p : s->f)
    if (e == cudaSuccess) e = cudaMalloc(&p, fb);
  if (e == cudaSuccess) e = cudaMalloc(&s->mt, fb);
  if (e == cudaSuccess) e = cudaMalloc(&s->gram, (size_t)(r * r) * sizeof(double));
  s->k2s_bytes = need;
  if (e == cudaSuccess) e = cudaMalloc(&s->k2s, s->k2s_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? GROM_ERR_OOM : GROM_ERR_CUDA, "grom_als_fit: device allocation");
  }
  s->rcap = r;
  return GROM_OK;
}

// Gram matrix of device factor q into host G.
grom_status gram_of(grom_als* s, int q, int64_t r, std::vector<double>& G) {
  dim3 grid((unsigned)((r + 15) / 16), (unsigned)((r + 15) / 16));
  k_gram<<<grid, dim3(16, 16), 0, s->stream>>>(s->f[q], s->n, r, s->gram);
  GROM_CUDA_TRY(cudaGetLastError());
  G.resize((size_t)(r * r));
  GROM_CUDA_TRY(cudaMemcpyAsync(G.data(), s->gram, G.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  GROM_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return GROM_OK;
}

// MTTKRP of layout m (0, 1, 2) with factors P (middle index) and Q (inner
// index) on the device into host Mt (r x n).
grom_status mttkrp(grom_als* s, int m, int fp, int fq, int64_t r, std::vector<double>& Mt) {
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
  Mt.resize((size_t)(r * s->n));
  GROM_CUDA_TRY(cudaMemcpyAsync(Mt.data(), s->mt, Mt.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
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

// The normal-equation update A = M H^-1, H = Ga o Gb + ridge max diag(Ga o Gb) I.
grom_status ls_update(grom_als* s, const std::vector<double>& Mt, const std::vector<double>& Ga,
                      const std::vector<double>& Gb, int64_t n, int64_t r, double ridge, std::vector<double>& A) {
  const auto t0 = std::chrono::steady_clock::now();
  // Cholesky of H = Ga o Gb; if H is numerically singular (ALS on a tensor
  // dominated by a few components drives the factor columns towards each
  // other), retry with a ridge mu I, mu = 1e-12 max diag(H), growing 100x up
  // to three times
  std::vector<double> H0((size_t)(r * r)), H;
  double dmax = 0.0;
  for (size_t q = 0; q < H0.size(); ++q) H0[q] = Ga[q] * Gb[q];
  for (int64_t a = 0; a < r; ++a) dmax = std::max(dmax, H0[a * r + a]);
  for (int64_t a = 0; a < r; ++a) H0[a * r + a] += ridge * dmax;
  bool ok = false;
  double mu = 0.0;
  for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
    H = H0;
    for (int64_t a = 0; a < r; ++a) H[a * r + a] += mu;
    ok = cholesky(H, r);
    mu = mu == 0.0 ? 1e-12 * dmax : mu * 100.0;
  }
  if (!ok) return fail(GROM_ERR_INVALID_ARG, "grom_als_fit: a Gram matrix is not positive definite");
  solve_rows(H, r, Mt, n, A);
  s->solve_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return GROM_OK;
}

grom_status put(grom_als* s, int q, const std::vector<double>& A) {
  GROM_CUDA_TRY(cudaMemcpyAsync(s->f[q], A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice, s->stream));
  GROM_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return GROM_OK;
}

double relres(const grom_als* s, double ip, const std::vector<double>& G0, const std::vector<double>& G1,
              const std::vector<double>& G2) {
  double kk = 0.0;
  for (size_t q = 0; q < G0.size(); ++q) kk += G0[q] * G1[q] * G2[q];
  const double r2 = s->xnorm2 - 2.0 * ip + kk;
  return std::sqrt(std::max(r2, 0.0) / s->xnorm2);
}

// <X, [[A1, A2, A3]]> = sum_{i,r} A_m[i][r] MTTKRP_m[i][r].
double inner(const std::vector<double>& A, const std::vector<double>& Mt, int64_t n, int64_t r) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t a = 0; a < r; ++a) s += A[i * r + a] * Mt[a * n + i];
  return s;
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
  if (!s || !fa || !fb || rank < 1 || iters < 0 || !(ridge >= 0.0))
    return fail(GROM_ERR_INVALID_ARG, "grom_als_fit: bad argument");
  if (method != GROM_ALS_PLAIN && method != GROM_ALS_SKEW) return fail(GROM_ERR_INVALID_ARG, "grom_als_fit: bad method");
  if (method == GROM_ALS_PLAIN && !fc) return fail(GROM_ERR_INVALID_ARG, "grom_als_fit: fc is NULL");
  if (method == GROM_ALS_SKEW && (rank % 2 || subiters < 1 || !(lambda >= 0.0 && lambda < 1.0)))
    return fail(GROM_ERR_INVALID_ARG, "grom_als_fit: ALS-skew needs an even rank, subiters >= 1, 0 <= lambda < 1");
  const int64_t n = s->n, r = rank, h = r / 2;
  grom_status st = als_grow(s, r);
  if (st) return st;
  std::vector<double> F[3], G[3], Mt, Anew;
  if (method == GROM_ALS_PLAIN) {
    F[0].assign(fa, fa + n * r);
    F[1].assign(fb, fb + n * r);
    F[2].assign(fc, fc + n * r);
    for (int q = 0; q < 3; ++q)
      if ((st = put(s, q, F[q])) || (st = gram_of(s, q, r, G[q]))) return st;
    for (int it = 0; it < iters; ++it) {
      for (int m = 0; m < 3; ++m) {
        // layout m: rows of mode m; P, Q = the factors of its middle and inner index
        const int fp = m == 0 ? 1 : 0, fq = m == 2 ? 1 : 2;
        if ((st = mttkrp(s, m, fp, fq, r, Mt))) return st;
        if ((st = ls_update(s, Mt, G[fp], G[fq], n, r, ridge, F[m]))) return st;
        if ((st = put(s, m, F[m])) || (st = gram_of(s, m, r, G[m]))) return st;
      }
      // <X, K> from a fresh mode-1 MTTKRP with the final factors: the M the
      // last update used carries the noise that update amplified along the
      // near-null directions of its normal matrix, and would hide it
      if (residual) {
        if ((st = mttkrp(s, 0, 1, 2, r, Mt))) return st;
        residual[it] = relres(s, inner(F[0], Mt, n, r), G[0], G[1], G[2]);
      }
    }
    std::memcpy(fa, F[0].data(), F[0].size() * sizeof(double));
    std::memcpy(fb, F[1].data(), F[1].size() * sizeof(double));
    std::memcpy(fc, F[2].data(), F[2].size() * sizeof(double));
    return GROM_OK;
  }
  // ALS-skew: A1 = [A1_1 A1_2], A2 = [B1 B1], A3 = [A1_2, -A1_1]
  std::vector<double> A1(fa, fa + n * r), B1(fb, fb + n * h);
  auto derive = [&]() {
    F[0] = A1;
    F[1].resize((size_t)(n * r));
    F[2].resize((size_t)(n * r));
    for (int64_t i = 0; i < n; ++i)
      for (int64_t a = 0; a < h; ++a) {
        F[1][i * r + a] = F[1][i * r + h + a] = B1[i * h + a];
        F[2][i * r + a] = A1[i * r + h + a];
        F[2][i * r + h + a] = -A1[i * r + a];
      }
  };
  derive();
  for (int q = 0; q < 3; ++q)
    if ((st = put(s, q, F[q])) || (st = gram_of(s, q, r, G[q]))) return st;
  for (int it = 0; it < iters; ++it) {
    // A2 as in ALS (layout X2: P = A1, Q = A3), halves averaged
    if ((st = mttkrp(s, 1, 0, 2, r, Mt)) || (st = ls_update(s, Mt, G[0], G[2], n, r, ridge, Anew))) return st;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t a = 0; a < h; ++a) B1[i * h + a] = 0.5 * (Anew[i * r + a] + Anew[i * r + h + a]);
    derive();
    if ((st = put(s, 1, F[1])) || (st = gram_of(s, 1, r, G[1]))) return st;
    for (int sub = 0; sub < subiters; ++sub) {
      // A1_next with A2, A3 fixed (layout X1: P = A2, Q = A3), then momentum
      if ((st = mttkrp(s, 0, 1, 2, r, Mt)) || (st = ls_update(s, Mt, G[1], G[2], n, r, ridge, Anew))) return st;
      for (size_t q = 0; q < A1.size(); ++q) A1[q] = lambda * A1[q] + (1.0 - lambda) * Anew[q];
      derive();
      if ((st = put(s, 0, F[0])) || (st = put(s, 2, F[2])) || (st = gram_of(s, 0, r, G[0])) ||
          (st = gram_of(s, 2, r, G[2])))
        return st;
    }
    if (residual) {
      if ((st = mttkrp(s, 0, 1, 2, r, Mt))) return st;
      residual[it] = relres(s, inner(F[0], Mt, n, r), G[0], G[1], G[2]);
    }
  }
  std::memcpy(fa, A1.data(), A1.size() * sizeof(double));
  std::memcpy(fb, B1.data(), B1.size() * sizeof(double));
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
  for (auto p : s->f)
    if (p) cudaFree(p);
  if (s->mt) cudaFree(s->mt);
  if (s->gram) cudaFree(s->gram);
  if (s->k2s) cudaFree(s->k2s);
  if (s->err) cudaFree(s->err);
  delete s;
  return GROM_OK;
}

}  // extern "C"
