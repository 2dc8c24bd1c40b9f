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
// multiple of 8).  Two launches per pass:
//   project  grid (column tiles of 64) x (row slices): each warp streams rows of
//            its slice with coalesced 64-column loads; partial sums per slice.
//            The last CTA of a column tile to finish (arrival counter, no
//            waiting) sums the slices in fixed order and forms the Hadamard
//            products h1 = p o q (and h2 = p o s).
//   expand   one warp per test index: c_i = sum_r A_ir h1_r (- W_ir h2_r), with
//            16-byte loads; optionally followed, in the same kernel, by the
//            diagonal BDFk/EXTk step of that row (last-CTA reduction of the
//            energy and invariant per trajectory).
#include "grom_internal.h"

namespace grom {

constexpr int K3_COLS = 64;  // columns per project CTA (2 per lane)
constexpr int K3_WARPS = 8;

template <int ST>
struct K3T;
template <>
struct K3T<GROM_F64> {
  using acc_t = double;
  static constexpr int EV = 2;  // elements per 16-byte vector
  static __device__ __forceinline__ void load2(const uint8_t* base, int64_t idx, double& x0, double& x1) {
    const double2 v = *reinterpret_cast<const double2*>(base + idx * 8);
    x0 = v.x;
    x1 = v.y;
  }
  static __device__ __forceinline__ void loadv(const uint8_t* base, int64_t idx, double (&x)[EV]) {
    const double2 v = *reinterpret_cast<const double2*>(base + idx * 8);
    x[0] = v.x;
    x[1] = v.y;
  }
  static __device__ __forceinline__ double cvt_u(double v) { return v; }
};
template <>
struct K3T<GROM_F32> {
  using acc_t = float;
  static constexpr int EV = 4;
  static __device__ __forceinline__ void load2(const uint8_t* base, int64_t idx, float& x0, float& x1) {
    const float2 v = *reinterpret_cast<const float2*>(base + idx * 4);
    x0 = v.x;
    x1 = v.y;
  }
  static __device__ __forceinline__ void loadv(const uint8_t* base, int64_t idx, float (&x)[EV]) {
    const float4 v = *reinterpret_cast<const float4*>(base + idx * 4);
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
  }
  static __device__ __forceinline__ float cvt_u(double v) { return __double2float_rn(v); }
};
template <>
struct K3T<GROM_BF16> {
  using acc_t = float;
  static constexpr int EV = 8;
  static __device__ __forceinline__ void load2(const uint8_t* base, int64_t idx, float& x0, float& x1) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(base + idx * 2);
    x0 = __uint_as_float(w << 16);
    x1 = __uint_as_float(w & 0xffff0000u);
  }
  static __device__ __forceinline__ void loadv(const uint8_t* base, int64_t idx, float (&x)[EV]) {
    const uint4 v = *reinterpret_cast<const uint4*>(base + idx * 2);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      x[2 * q] = __uint_as_float(w[q] << 16);
      x[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
    }
  }
  static __device__ __forceinline__ float cvt_u(double v) { return __double2float_rn(v); }
};

struct K3Shape {
  int64_t n, rp;
  int slices, tiles;
  int nf;  // projected factors: 2 (general) or 3 (skew)
};

__device__ __forceinline__ const double* k3_u_ptr(const K3Args& a, int bg, int64_t n) {
  return a.taken ? a.hist + bg * a.hist_stride + (a.taken[bg] % 3) * n : a.u + bg * a.u_stride;
}

__constant__ double k3_beta[3][4] = {
    {1.0, -1.0, 0.0, 0.0},
    {1.5, -2.0, 0.5, 0.0},
    {11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0},
};
__constant__ double k3_alpha[3][3] = {
    {1.0, 0.0, 0.0},
    {2.0, -1.0, 0.0},
    {3.0, -3.0, 1.0},
};

// partial layout: [slice][f][b][rp]; h layout: [2][b][rp] (h2 for skew only)
template <int ST, int NB>
__global__ void __launch_bounds__(256) k3_project_kernel(const K3Shape sh, const K3Args a, const int b0, void* partial,
                                                         void* hbuf, unsigned int* tile_cnt) {
  using T = K3T<ST>;
  using acc_t = typename T::acc_t;
  __shared__ acc_t red[K3_WARPS][3][NB][K3_COLS];
  __shared__ int last;
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
  // the last slice of this column tile to finish forms h for the tile
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&tile_cnt[blockIdx.x], 1u) == (unsigned)(sh.slices - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  acc_t* h = reinterpret_cast<acc_t*>(hbuf);
  for (int t = threadIdx.x; t < NB * K3_COLS; t += blockDim.x) {
    const int b = t / K3_COLS, cc = t % K3_COLS;
    const int64_t c = (int64_t)blockIdx.x * K3_COLS + cc;
    if (c >= rp) continue;
    acc_t v[3] = {acc_t(0), acc_t(0), acc_t(0)};
    for (int s = 0; s < sh.slices; ++s)
#pragma unroll
      for (int f = 0; f < 3; ++f)
        if (f < sh.nf) v[f] += __ldcg(out + (((int64_t)s * sh.nf + f) * NB + b) * rp + c);
    h[(int64_t)b * rp + c] = v[0] * v[1];
    if (sh.nf == 3) h[((int64_t)NB + b) * rp + c] = v[0] * v[2];
  }
  if (threadIdx.x == 0) tile_cnt[blockIdx.x] = 0u;
}

template <int ST, int NB>
__global__ void __launch_bounds__(256) k3_expand_kernel(const K3Shape sh, const K3Args a, const int b0, const void* hbuf,
                                                        const StepArgs st, const int fuse_step, const int step_index) {
  using T = K3T<ST>;
  using acc_t = typename T::acc_t;
  constexpr int EV = T::EV;
  __shared__ double se[K3_WARPS][NB], si[K3_WARPS][NB];
  __shared__ int sbad[NB];
  __shared__ int last[NB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * K3_WARPS + warp;
  const int64_t n = sh.n, rp = sh.rp;
  const acc_t* h = reinterpret_cast<const acc_t*>(hbuf);
  acc_t acc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) acc[b] = acc_t(0);
  if (i < n) {
    for (int64_t r = (int64_t)EV * lane; r < rp; r += 32 * EV) {
      acc_t x[EV];
      T::loadv(a.fa, i * rp + r, x);
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int e = 0; e < EV; ++e) acc[b] = fma(x[e], h[(int64_t)b * rp + r + e], acc[b]);
      if (sh.nf == 3) {
        T::loadv(a.fc, i * rp + r, x);
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int e = 0; e < EV; ++e) acc[b] = fma(-x[e], h[((int64_t)NB + b) * rp + r + e], acc[b]);
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
  // lane b of the warp owns trajectory b0+b of row i
  double cval = 0.0;
#pragma unroll
  for (int q = 0; q < NB; ++q)
    if (q == lane) cval = (double)acc[q];
  const int bg = b0 + lane;
  const bool mine = lane < a.nb && i < n && (a.active == nullptr || a.active[bg]);
  if (!fuse_step) {
    if (mine) {
      double* dst = a.taken ? a.hist + bg * a.hist_stride + (3 + a.taken[bg] % 3) * n : a.c + bg * a.c_stride;
      dst[i] = cval;
    }
    return;
  }
  // ---- fused diagonal BDFk/EXTk step of row i (see k_step.cu for the scheme)
  if (threadIdx.x < NB) sbad[threadIdx.x] = 0;
  double e_part = 0.0, i_part = 0.0;
  if (lane < NB) {
    se[warp][lane] = 0.0;
    si[warp][lane] = 0.0;
  }
  __syncthreads();
  if (mine) {
    const int64_t l = st.taken[bg];
    const int k = (int)(l + 1 < st.order ? l + 1 : st.order);
    double* hh = st.hist + bg * st.hist_stride;
    hh[(3 + l % 3) * n + i] = cval;
    const double mb = st.mass_diag ? st.mass_diag[i] : 1.0;
    const double ld = st.lin_diag ? st.lin_diag[i] : 0.0;
    const double f = st.forcing ? st.forcing[i] : 0.0;
    const double inv_dt = st.inv_dt;
    double ext = 0.0, bdf = 0.0, u0 = 0.0;
    for (int q = 0; q < k; ++q) {
      const int64_t m = ((l - q) % 3 + 3) % 3;
      const double uq = hh[m * n + i];
      const double nq = q == 0 ? cval : hh[(3 + m) * n + i];
      if (q == 0) u0 = uq;
      ext += k3_alpha[k - 1][q] * (nq + ld * uq + f);
      bdf += k3_beta[k - 1][q + 1] * inv_dt * uq;
    }
    const double un = (-ext - mb * bdf) * st.hdiag[k - 1][i];
    hh[((l + 1) % 3) * n + i] = un;
    e_part = mb * un * un;
    i_part = u0 * cval;
    if (!isfinite(un)) sbad[lane] = 1;
    se[warp][lane] = e_part;
    si[warp][lane] = i_part;
  }
  __syncthreads();
  // warp b closes trajectory b (NB <= K3_WARPS): lane 0 publishes the block's
  // partials; in the last block to arrive the warp sums all blocks' partials
  // (lane q adds blocks q, q+32, ... in order, then a fixed shuffle tree)
  static_assert(NB <= K3_WARPS, "one warp per trajectory");
  if (warp < NB && warp < a.nb) {
    const int b = warp, bgl = b0 + b;
    if (a.active == nullptr || a.active[bgl]) {
      if (lane == 0) {
        double e = 0.0, inv = 0.0;
#pragma unroll
        for (int w = 0; w < K3_WARPS; ++w) {
          e += se[w][b];
          inv += si[w][b];
        }
        if (sbad[b]) {
          atomicOr(st.err, DEV_ERR_NONFINITE);
          atomicMin(st.first_bad, bgl);
        }
        double* r = st.red + ((int64_t)bgl * st.nblk + blockIdx.x) * 2;
        r[0] = e;
        r[1] = inv;
        __threadfence();
        last[b] = atomicAdd(&st.cnt[bgl], 1u) == (unsigned)(st.nblk - 1);
      }
      __syncwarp();
      if (last[b]) {
        __threadfence();
        double es = 0.0, is = 0.0;
        const double* rr = st.red + (int64_t)bgl * st.nblk * 2;
        for (int q = lane; q < st.nblk; q += 32) {
          es += __ldcg(rr + 2 * q);
          is += __ldcg(rr + 2 * q + 1);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          es += __shfl_xor_sync(0xffffffffu, es, off);
          is += __shfl_xor_sync(0xffffffffu, is, off);
        }
        if (lane == 0) {
          if (st.energy) st.energy[(int64_t)step_index * st.batch + bgl] = 0.5 * es;
          if (st.invariant) st.invariant[(int64_t)step_index * st.batch + bgl] = is;
          step_done(st, bgl, st.taken[bgl]);
          st.cnt[bgl] = 0u;
        }
      }
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

// partials, h and the per-tile arrival counters
size_t k3_scratch_bytes(const K3Plan& p, int storage) {
  const size_t es = storage == GROM_F64 ? 8 : 4;
  const size_t tiles = (size_t)((p.rb + K3_COLS - 1) / K3_COLS);
  return es * (size_t)p.rb * (size_t)p.nb_max * (3 * (size_t)p.nblk + 2) + 256 + tiles * sizeof(unsigned int);
}

size_t k3_counter_offset(const K3Plan& p, int storage) {
  const size_t es = storage == GROM_F64 ? 8 : 4;
  return (es * (size_t)p.rb * (size_t)p.nb_max * (3 * (size_t)p.nblk + 2) + 255) / 256 * 256;
}

int k3_expand_blocks(int64_t n) { return (int)((n + K3_WARPS - 1) / K3_WARPS); }

template <int ST, int NB>
static cudaError_t k3_run(const K3Plan& p, const K3Args& a, int b0, const StepArgs* st, int step_index,
                          cudaStream_t s) {
  const int tiles = (int)((p.rb + K3_COLS - 1) / K3_COLS);
  K3Shape sh{p.n, p.rb, (int)p.nblk, tiles, a.form == GROM_FORM_CP_SKEW ? 3 : 2};
  using acc_t = typename K3T<ST>::acc_t;
  uint8_t* base = reinterpret_cast<uint8_t*>(a.part);
  void* partial = base;
  void* hbuf = base + sizeof(acc_t) * (size_t)p.rb * NB * 3 * p.nblk;
  unsigned int* cnt = reinterpret_cast<unsigned int*>(base + k3_counter_offset(p, ST));
  dim3 g1((unsigned)tiles, (unsigned)p.nblk);
  k3_project_kernel<ST, NB><<<g1, 256, 0, s>>>(sh, a, b0, partial, hbuf, cnt);
  StepArgs none{};
  k3_expand_kernel<ST, NB><<<(unsigned)k3_expand_blocks(p.n), 256, 0, s>>>(sh, a, b0, hbuf, st ? *st : none,
                                                                           st ? 1 : 0, step_index);
  return cudaGetLastError();
}

template <int ST>
static cudaError_t k3_nb(int nb, const K3Plan& p, const K3Args& a, int b0, const StepArgs* st, int step_index,
                         cudaStream_t s) {
  switch (nb) {
    case 1: return k3_run<ST, 1>(p, a, b0, st, step_index, s);
    case 2: return k3_run<ST, 2>(p, a, b0, st, step_index, s);
    case 4: return k3_run<ST, 4>(p, a, b0, st, step_index, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t k3_launch_step(const K3Plan& p, int storage, const K3Args& a0, int batch, const StepArgs* st,
                           int step_index, cudaStream_t s) {
  for (int b0 = 0; b0 < batch; b0 += p.nb_max) {
    K3Args a = a0;
    a.nb = batch - b0 < p.nb_max ? batch - b0 : p.nb_max;
    const int nb = a.nb == 1 ? 1 : a.nb == 2 ? 2 : 4;
    cudaError_t e;
    switch (storage) {
      case GROM_F64: e = k3_nb<GROM_F64>(nb, p, a, b0, st, step_index, s); break;
      case GROM_F32: e = k3_nb<GROM_F32>(nb, p, a, b0, st, step_index, s); break;
      case GROM_BF16: e = k3_nb<GROM_BF16>(nb, p, a, b0, st, step_index, s); break;
      default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t k3_launch(const K3Plan& p, int storage, const K3Args& a0, int batch, cudaStream_t s) {
  return k3_launch_step(p, storage, a0, batch, nullptr, 0, s);
}

}  // namespace grom
