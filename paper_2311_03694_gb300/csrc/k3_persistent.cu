// Persistent CPD-ROM stepper for one to four trajectories: every step of a
// grom_step call in a single cooperative launch (one CTA per SM, all
// co-resident), the CP advection term (Sec. 3.1, eq. tc_ap; skew structure
// Sec. 3.3) and the diagonal BDFk/EXTk step (Sec. 2.2, eq. nse_d1).
//
// CTA g owns a block of rank columns and keeps its columns of the three
// factors in shared memory for the whole launch, so per step only the states
// and the partial sums travel.  It also owns a block of test indices.  A step:
//   1  load u^l (all n entries) into shared memory;
//   2  projections p = V^T u, q = W^T u (s = U^T u) for the owned columns,
//      Hadamard products h1 = p o q (h2 = p o s), and the partial expansion
//      c_i^(g) = sum_{r owned} U_ir h1_r (- W_ir h2_r) for every i, written
//      to global memory;
//   -- grid barrier --
//   3  for the owned test indices: c_i = sum over CTAs of c_i^(g) in a fixed
//      order, then the step of those rows; per-CTA energy/invariant partials;
//   -- grid barrier --
//   4  CTA 0 sums the energy/invariant partials in CTA order.
// The step count lives in registers during the launch (written once at the
// end).  Every barrier wait gives up after one second (device timeout flag,
// kernel returns).
#include "grom_internal.h"
#include "ptx.cuh"

namespace grom {

constexpr int KP_THREADS = 256;
constexpr int KP_WARPS = KP_THREADS / 32;
constexpr int KP_COLS = 64;

template <int ST>
struct KPT;
template <>
struct KPT<GROM_F64> {
  using acc_t = double;
  static constexpr int EV = 2;
  static __device__ __forceinline__ void load2(const uint8_t* b, int64_t i, double& x0, double& x1) {
    const double2 v = *reinterpret_cast<const double2*>(b + i * 8);
    x0 = v.x;
    x1 = v.y;
  }
  static __device__ __forceinline__ void loadv(const uint8_t* b, int64_t i, double (&x)[EV]) {
    const double2 v = *reinterpret_cast<const double2*>(b + i * 8);
    x[0] = v.x;
    x[1] = v.y;
  }
  static __device__ __forceinline__ double cu(double v) { return v; }
};
template <>
struct KPT<GROM_F32> {
  using acc_t = float;
  static constexpr int EV = 4;
  static __device__ __forceinline__ void load2(const uint8_t* b, int64_t i, float& x0, float& x1) {
    const float2 v = *reinterpret_cast<const float2*>(b + i * 4);
    x0 = v.x;
    x1 = v.y;
  }
  static __device__ __forceinline__ void loadv(const uint8_t* b, int64_t i, float (&x)[EV]) {
    const float4 v = *reinterpret_cast<const float4*>(b + i * 4);
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
  }
  static __device__ __forceinline__ float cu(double v) { return __double2float_rn(v); }
};
template <>
struct KPT<GROM_BF16> {
  using acc_t = float;
  static constexpr int EV = 8;
  static __device__ __forceinline__ void load2(const uint8_t* b, int64_t i, float& x0, float& x1) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(b + i * 2);
    x0 = __uint_as_float(w << 16);
    x1 = __uint_as_float(w & 0xffff0000u);
  }
  static __device__ __forceinline__ void loadv(const uint8_t* b, int64_t i, float (&x)[EV]) {
    const uint4 v = *reinterpret_cast<const uint4*>(b + i * 2);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      x[2 * q] = __uint_as_float(w[q] << 16);
      x[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
    }
  }
  static __device__ __forceinline__ float cu(double v) { return __double2float_rn(v); }
};

__constant__ double kp_beta[3][4] = {
    {1.0, -1.0, 0.0, 0.0},
    {1.5, -2.0, 0.5, 0.0},
    {11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0},
};
__constant__ double kp_alpha[3][3] = {
    {1.0, 0.0, 0.0},
    {2.0, -1.0, 0.0},
    {3.0, -3.0, 1.0},
};

struct KPArgs {
  const uint8_t* fa;  // U (skew) or A (general), n x rp stored
  const uint8_t* fb;  // V or B
  const uint8_t* fc;  // W or C
  int nf;             // 3 skew, 2 general
  int64_t n, rp;
  int rbw;            // rank columns per CTA (upper bound)
  int batch, nsteps;
  double* cpart;      // grid x NB x n partial expansions (FP64)
  double* red;        // grid x NB x 2
  unsigned int* bar;  // grid barrier word (self-resetting)
  StepArgs st;
};

// Grid barrier: CTA 0 adds 2^31 - (G - 1), every other CTA adds 1, so the
// word's top bit flips exactly once per barrier and the low bits return to
// their value (no reset between launches).  Returns false on timeout.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* err) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    __threadfence();
    const unsigned int old = atomicAdd(bar, inc);
    int ok = 1;
    const uint64_t t0 = ptx::globaltimer();
    for (uint32_t spin = 0;; ++spin) {
      const unsigned int now = *reinterpret_cast<volatile unsigned int*>(bar);
      if ((now ^ old) & 0x80000000u) break;
      if ((spin & 255u) == 255u && ptx::globaltimer() - t0 > ptx::WAIT_LIMIT_NS) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

template <int ST>
struct KPS;  // element type kept in shared memory
template <>
struct KPS<GROM_F64> {
  using el = double;
  static __device__ __forceinline__ double get(const uint8_t* b, int64_t i) { return reinterpret_cast<const double*>(b)[i]; }
  static __device__ __forceinline__ double val(double v) { return v; }
};
template <>
struct KPS<GROM_F32> {
  using el = float;
  static __device__ __forceinline__ float get(const uint8_t* b, int64_t i) { return reinterpret_cast<const float*>(b)[i]; }
  static __device__ __forceinline__ float val(float v) { return v; }
};
template <>
struct KPS<GROM_BF16> {
  using el = uint16_t;
  static __device__ __forceinline__ uint16_t get(const uint8_t* b, int64_t i) {
    return reinterpret_cast<const uint16_t*>(b)[i];
  }
  static __device__ __forceinline__ float val(uint16_t v) { return __uint_as_float((uint32_t)v << 16); }
};

// rows a CTA owns at most
__host__ __device__ inline int64_t kp_rows_max(int64_t n, int grid) { return n / grid + 1; }

struct KPSmem {
  size_t us, hs, wred, se, hist, sbad, total;
};
__host__ __device__ inline KPSmem kp_smem_layout(int64_t n, int rbw, int el_bytes, int acc_bytes, int nb, int grid) {
  KPSmem L{};
  size_t off = (((size_t)3 * n * rbw * el_bytes + 15) / 16) * 16;
  L.us = off;
  off += (size_t)nb * n * acc_bytes;
  L.hs = off;
  off += (size_t)2 * nb * rbw * acc_bytes;
  L.wred = off;
  off += (size_t)KP_THREADS * 3 * nb * acc_bytes;
  off = (off + 15) / 16 * 16;
  L.se = off;
  off += (size_t)2 * KP_WARPS * nb * 8;
  L.hist = off;  // owned rows' history: [nb][rows_max][6] doubles
  off += (size_t)nb * kp_rows_max(n, grid) * 6 * 8;
  L.sbad = off;
  off += (size_t)nb * 4;
  L.total = (off + 15) / 16 * 16;
  return L;
}

template <int ST, int NB>
__global__ void __launch_bounds__(KP_THREADS, 1) k3p_kernel(const KPArgs p) {
  using T = KPT<ST>;
  using S = KPS<ST>;
  using acc_t = typename T::acc_t;
  using el = typename S::el;
  extern __shared__ __align__(16) uint8_t kp_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, g = blockIdx.x;
  const int64_t n = p.n;
  const StepArgs& st = p.st;
  // owned rank columns [r0, r1) and test indices [i0, i1)
  const int64_t r0 = (int64_t)g * p.rp / G, r1 = ((int64_t)g + 1) * p.rp / G;
  const int rb = (int)(r1 - r0);
  const int64_t i0 = (int64_t)g * n / G, i1 = ((int64_t)g + 1) * n / G;
  // shared memory: factor columns [3][n][rbw], states [NB][n], Hadamard
  // products [2][NB][rbw], thread partials [KP_THREADS][3][NB], warp sums
  const KPSmem L = kp_smem_layout(n, p.rbw, (int)sizeof(el), (int)sizeof(acc_t), NB, G);
  el* fs = reinterpret_cast<el*>(kp_smem);
  acc_t* us = reinterpret_cast<acc_t*>(kp_smem + L.us);
  acc_t* hs = reinterpret_cast<acc_t*>(kp_smem + L.hs);
  acc_t* wred = reinterpret_cast<acc_t*>(kp_smem + L.wred);
  double* se = reinterpret_cast<double*>(kp_smem + L.se);
  double* si = se + KP_WARPS * NB;
  int* sbad = reinterpret_cast<int*>(kp_smem + L.sbad);
  double* hsh = reinterpret_cast<double*>(kp_smem + L.hist);  // [NB][rows][6]: u^l, u^l-1, u^l-2, n^l, n^l-1, n^l-2
  const int64_t rows_max = kp_rows_max(n, G);
  const uint8_t* F[3] = {p.fb, p.fc, p.fa};  // projected factors: general (fb, fc), skew (fb, fc, fa)
  for (int64_t t = threadIdx.x; t < (int64_t)3 * n * rb; t += KP_THREADS) {
    const int f = (int)(t / (n * rb));
    const int64_t rem = t - (int64_t)f * n * rb, i = rem / rb, c = rem - i * rb;
    fs[((int64_t)f * n + i) * p.rbw + c] = (f < p.nf) ? S::get(F[f], i * p.rp + r0 + c) : el(0);
  }
  if (threadIdx.x < NB) sbad[threadIdx.x] = 0;
  int64_t l0[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) l0[b] = b < p.batch ? st.taken[b] : 0;
  const double inv_dt = st.inv_dt;
  // the owned rows' history stays in shared memory for the whole launch
  for (int t = threadIdx.x; t < NB * (int)(i1 - i0) * 6; t += KP_THREADS) {
    const int b = t / ((int)(i1 - i0) * 6), rem = t % ((int)(i1 - i0) * 6), ri = rem / 6, q = rem % 6;
    double v = 0.0;
    if (b < p.batch) {
      const int64_t l = st.taken[b];
      const int64_t m = ((l - (q % 3)) % 3 + 3) % 3;
      v = st.hist[b * st.hist_stride + ((q < 3 ? 0 : 3) + m) * n + i0 + ri];
    }
    hsh[((int64_t)b * rows_max + ri) * 6 + q] = v;
  }
  __syncthreads();
  // slot 2 holds the expansion factor (U, or A for the general form, which is
  // not one of the projected factors)
  if (p.nf == 2) {
    for (int64_t t = threadIdx.x; t < n * rb; t += KP_THREADS) {
      const int64_t i = t / rb, c = t - i * rb;
      fs[((int64_t)2 * n + i) * p.rbw + c] = S::get(p.fa, i * p.rp + r0 + c);
    }
    __syncthreads();
  }

  for (int step = 0; step < p.nsteps; ++step) {
    // ---- 1: states of this step
    for (int64_t t = threadIdx.x; t < (int64_t)NB * n; t += KP_THREADS) {
      const int b = (int)(t / n);
      const int64_t i = t - (int64_t)b * n;
      us[t] = b < p.batch ? T::cu(__ldcg(st.hist + b * st.hist_stride + ((l0[b] + step) % 3) * n + i)) : acc_t(0);
    }
    __syncthreads();
    // ---- 2a: projections of the owned columns: thread t takes column t % rb
    //          and every (KP_THREADS / rb)-th row starting at t / rb
    const int nphase = rb > 0 ? KP_THREADS / rb : 0;
    if (rb > 0 && (int)threadIdx.x < nphase * rb) {
      const int c = threadIdx.x % rb, ph = threadIdx.x / rb;
      acc_t acc[3][NB];
#pragma unroll
      for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[f][b] = acc_t(0);
      for (int64_t i = ph; i < n; i += nphase) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          if (f < p.nf) {
            const acc_t x = (acc_t)S::val(fs[((int64_t)f * n + i) * p.rbw + c]);
#pragma unroll
            for (int b = 0; b < NB; ++b) acc[f][b] = fma(x, us[(int64_t)b * n + i], acc[f][b]);
          }
        }
      }
#pragma unroll
      for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int b = 0; b < NB; ++b) wred[((int64_t)threadIdx.x * 3 + f) * NB + b] = acc[f][b];
    }
    __syncthreads();
    // ---- 2b: Hadamard products of the owned columns (phases summed in order)
    for (int t = threadIdx.x; t < NB * rb; t += KP_THREADS) {
      const int b = t / rb, c = t % rb;
      acc_t v[3] = {acc_t(0), acc_t(0), acc_t(0)};
      for (int ph = 0; ph < nphase; ++ph)
#pragma unroll
        for (int f = 0; f < 3; ++f)
          if (f < p.nf) v[f] += wred[((int64_t)(ph * rb + c) * 3 + f) * NB + b];
      hs[b * p.rbw + c] = v[0] * v[1];
      hs[((int64_t)NB + b) * p.rbw + c] = p.nf == 3 ? v[0] * v[2] : acc_t(0);
    }
    __syncthreads();
    // ---- 2c: partial expansion for every test index
    for (int64_t i = threadIdx.x; i < n; i += KP_THREADS) {
      acc_t acc[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) acc[b] = acc_t(0);
      for (int c = 0; c < rb; ++c) {
        const acc_t xa = (acc_t)S::val(fs[((int64_t)2 * n + i) * p.rbw + c]);
        const acc_t xw = p.nf == 3 ? (acc_t)S::val(fs[((int64_t)1 * n + i) * p.rbw + c]) : acc_t(0);
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          acc[b] = fma(xa, hs[b * p.rbw + c], acc[b]);
          acc[b] = fma(-xw, hs[((int64_t)NB + b) * p.rbw + c], acc[b]);
        }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) p.cpart[((int64_t)g * NB + b) * n + i] = (double)acc[b];
    }
    if (!grid_barrier(p.bar, st.err)) return;
    // ---- 3: owned test indices: sum the partial expansions, then the step
    double e_acc[NB], i_acc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) e_acc[b] = i_acc[b] = 0.0;
    for (int64_t i = i0 + warp; i < i1; i += KP_WARPS) {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (b >= p.batch) continue;
        double v = 0.0;
        for (int q = lane; q < G; q += 32) v += __ldcg(p.cpart + ((int64_t)q * NB + b) * n + i);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) {
          const double cval = v;
          const int64_t l = l0[b] + step;
          const int k = (int)(l + 1 < st.order ? l + 1 : st.order);
          double* hr = hsh + ((int64_t)b * rows_max + (i - i0)) * 6;  // u^l, u^l-1, u^l-2, n^l, n^l-1, n^l-2
          hr[3] = cval;
          const double mb = st.mass_diag ? st.mass_diag[i] : 1.0;
          const double ld = st.lin_diag ? st.lin_diag[i] : 0.0;
          const double f = st.forcing ? st.forcing[i] : 0.0;
          double ext = 0.0, bdf = 0.0;
          for (int q = 0; q < k; ++q) {
            ext += kp_alpha[k - 1][q] * (hr[3 + q] + ld * hr[q] + f);
            bdf += kp_beta[k - 1][q + 1] * inv_dt * hr[q];
          }
          const double un = (-ext - mb * bdf) * st.hdiag[k - 1][i];
          if (!isfinite(un)) sbad[b] = 1;
          e_acc[b] += mb * un * un;
          i_acc[b] += hr[0] * cval;
          // rotate; the new state goes to global memory for every CTA's next projection
          hr[2] = hr[1]; hr[1] = hr[0]; hr[0] = un;
          hr[5] = hr[4]; hr[4] = hr[3];
          st.hist[b * st.hist_stride + ((l + 1) % 3) * n + i] = un;
        }
      }
    }
    if (lane == 0)
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        se[warp * NB + b] = e_acc[b];
        si[warp * NB + b] = i_acc[b];
      }
    __syncthreads();
    if (threadIdx.x < NB && threadIdx.x < p.batch) {
      const int b = threadIdx.x;
      double ev = 0.0, iv = 0.0;
#pragma unroll
      for (int w = 0; w < KP_WARPS; ++w) {
        ev += se[w * NB + b];
        iv += si[w * NB + b];
      }
      p.red[((int64_t)g * NB + b) * 2] = ev;
      p.red[((int64_t)g * NB + b) * 2 + 1] = iv;
      if (sbad[b]) {
        atomicOr(st.err, DEV_ERR_NONFINITE);
        atomicMin(st.first_bad, b);
        sbad[b] = 0;
      }
    }
    if (!grid_barrier(p.bar, st.err)) return;
    // ---- 4: energy / invariant of this step
    // warp b of CTA 0 sums trajectory b's CTA partials (lane q adds CTAs q,
    // q+32, ... in order, then a fixed shuffle tree)
    static_assert(NB <= KP_WARPS, "one warp per trajectory");
    if (g == 0 && warp < NB && warp < p.batch && (st.energy || st.invariant)) {
      const int b = warp;
      double ev = 0.0, iv = 0.0;
      for (int q = lane; q < G; q += 32) {
        ev += __ldcg(p.red + ((int64_t)q * NB + b) * 2);
        iv += __ldcg(p.red + ((int64_t)q * NB + b) * 2 + 1);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        ev += __shfl_xor_sync(0xffffffffu, ev, off);
        iv += __shfl_xor_sync(0xffffffffu, iv, off);
      }
      if (lane == 0) {
        if (st.energy) st.energy[(int64_t)step * st.batch + b] = 0.5 * ev;
        if (st.invariant) st.invariant[(int64_t)step * st.batch + b] = iv;
      }
    }
  }
  // write the owned rows' history back into the ring (n^l of the newest
  // state is recomputed by whoever needs it; its slot keeps the last n)
  __syncthreads();
  for (int t = threadIdx.x; t < NB * (int)(i1 - i0) * 6; t += KP_THREADS) {
    const int b = t / ((int)(i1 - i0) * 6), rem = t % ((int)(i1 - i0) * 6), ri = rem / 6, q = rem % 6;
    if (b >= p.batch) continue;
    const int64_t l = l0[b] + p.nsteps;
    if (q == 3) continue;  // n^l of the newest state is not known yet
    const int64_t m = ((l - (q % 3)) % 3 + 3) % 3;
    st.hist[b * st.hist_stride + ((q < 3 ? 0 : 3) + m) * n + i0 + ri] = hsh[((int64_t)b * rows_max + ri) * 6 + q];
  }
  if (g == 0 && threadIdx.x < NB && threadIdx.x < p.batch) st.taken[threadIdx.x] = l0[threadIdx.x] + p.nsteps;
}

template <int ST, int NB>
static size_t kp_smem(int64_t n, int rbw, int grid) {
  using acc_t = typename KPT<ST>::acc_t;
  using el = typename KPS<ST>::el;
  return kp_smem_layout(n, rbw, (int)sizeof(el), (int)sizeof(acc_t), NB, grid).total;
}

size_t k3p_scratch_bytes(int64_t n, int64_t rp, int storage, int sm_count) {
  (void)rp;
  (void)storage;
  return 256 + 8 * ((size_t)sm_count * 4 * (size_t)n + (size_t)sm_count * 4 * 2);
}

// Steps `batch` trajectories (<= k3p_max_batch) nsteps times in one cooperative launch.
int k3p_max_batch(int storage) { return storage == GROM_F64 ? 2 : 4; }

template <int ST, int NB>
static cudaError_t k3p_run(KPArgs p, int grid, cudaStream_t s) {
  auto kern = k3p_kernel<ST, NB>;
  const size_t smem = kp_smem<ST, NB>(p.n, p.rbw, grid);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;  // factors do not fit: caller falls back
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, KP_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {&p};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid), dim3(KP_THREADS), args, smem, s);
}

bool k3p_fits(int64_t n, int64_t rp, int storage, int batch, int sm_count) {
  const int rbw = (int)((rp + sm_count - 1) / sm_count);
  if (rbw > KP_THREADS) return false;  // a thread per owned column is needed
  const int nb = batch <= 1 ? 1 : batch <= 2 ? 2 : 4;
  size_t smem = 0;
  switch (storage) {
    case GROM_F64: smem = nb == 1 ? kp_smem<GROM_F64, 1>(n, rbw, sm_count) : kp_smem<GROM_F64, 2>(n, rbw, sm_count); break;
    case GROM_F32: smem = nb == 1 ? kp_smem<GROM_F32, 1>(n, rbw, sm_count) : nb == 2 ? kp_smem<GROM_F32, 2>(n, rbw, sm_count) : kp_smem<GROM_F32, 4>(n, rbw, sm_count); break;
    case GROM_BF16: smem = nb == 1 ? kp_smem<GROM_BF16, 1>(n, rbw, sm_count) : nb == 2 ? kp_smem<GROM_BF16, 2>(n, rbw, sm_count) : kp_smem<GROM_BF16, 4>(n, rbw, sm_count); break;
    default: return false;
  }
  return smem <= 220 * 1024;
}

cudaError_t k3p_launch(const uint8_t* fa, const uint8_t* fb, const uint8_t* fc, int form, int64_t n, int64_t rp,
                       int storage, int batch, int nsteps, const StepArgs& st, void* scratch, int sm_count,
                       cudaStream_t s) {
  uint8_t* base = reinterpret_cast<uint8_t*>(scratch);
  KPArgs p{};
  p.fa = fa;
  p.fb = fb;
  p.fc = fc;
  p.nf = form == GROM_FORM_CP_SKEW ? 3 : 2;
  p.n = n;
  p.rp = rp;
  p.rbw = (int)((rp + sm_count - 1) / sm_count);
  p.batch = batch;
  p.nsteps = nsteps;
  p.bar = reinterpret_cast<unsigned int*>(base);
  p.cpart = reinterpret_cast<double*>(base + 256);
  p.red = p.cpart + (size_t)sm_count * 4 * n;
  p.st = st;
  const int nb = batch <= 1 ? 1 : batch <= 2 ? 2 : 4;
  switch (storage) {
    case GROM_F64:  // the FP64 shared-memory footprint limits this path to two trajectories
      return nb == 1 ? k3p_run<GROM_F64, 1>(p, sm_count, s)
                     : nb == 2 ? k3p_run<GROM_F64, 2>(p, sm_count, s) : cudaErrorInvalidValue;
    case GROM_F32:
      return nb == 1 ? k3p_run<GROM_F32, 1>(p, sm_count, s)
                     : nb == 2 ? k3p_run<GROM_F32, 2>(p, sm_count, s) : k3p_run<GROM_F32, 4>(p, sm_count, s);
    case GROM_BF16:
      return nb == 1 ? k3p_run<GROM_BF16, 1>(p, sm_count, s)
                     : nb == 2 ? k3p_run<GROM_BF16, 2>(p, sm_count, s) : k3p_run<GROM_BF16, 4>(p, sm_count, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace grom
