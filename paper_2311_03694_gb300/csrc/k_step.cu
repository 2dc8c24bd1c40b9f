// K4-K6: the BDFk/EXTk reduced step (Sec. 2.2, eq. nse_d1), FP64.
//
// History ring per trajectory (6 slots of n doubles): u^{m} lives in slot
// m mod 3 and n^{m} = C(u^m)u^m in slot 3 + m mod 3, where m counts steps
// taken.  A step at l = taken uses order k = min(l + 1, order):
//   rhs = -sum_{q<k} alpha_q (n^{l-q} + L u^{l-q} + f) - B sum_{q<k} beta_{q+1}/dt u^{l-q}
//   u^{l+1} = H_k^{-1} rhs,  H_k = beta0_k/dt B + nu A
// and writes u^{l+1} over u^{l-2} (slot (l+1) mod 3).  It also returns the
// energy 1/2 u^T B u of the new state, the invariant u^T n of the old state
// and flags non-finite states.
#include <cuda_bf16.h>

#include "grom_internal.h"
#include "ptx.cuh"
#include "step_elem.cuh"
#include "step_mc.cuh"

namespace grom {

constexpr int STEP_THREADS = 256;

// Deterministic block sum of two values (fixed tree), result in thread 0.
__device__ __forceinline__ void block_sum2(double& x, double& y, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, off);
    y += __shfl_down_sync(0xffffffffu, y, off);
  }
  if (lane == 0) {
    sh[warp] = x;
    sh[32 + warp] = y;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    x = lane < nw ? sh[lane] : 0.0;
    y = lane < nw ? sh[32 + lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, off);
      y += __shfl_down_sync(0xffffffffu, y, off);
    }
  }
}


// Diagonal step spread over nblk CTAs per trajectory (STEP_MC_THREADS each,
// a.ept elements per thread, strided by the block size).
// Per-CTA energy/invariant partials are summed in CTA order by the last CTA
// of the trajectory to arrive (arrival counter, no waiting), which also
// advances the step count.  With k1 set, the K1 partials of the element are
// summed first (the streaming kernel's finalize, fused).
template <bool PLAIN>
__global__ void __launch_bounds__(STEP_MC_THREADS) k_step_diag_mc(const StepArgs a, const int step_index,
                                                                  const K1Plan pl, const K1Args k1a, const int fuse,
                                                                  const int b0, const int nbk, const K3TStepFuse kf) {
  __shared__ double sh[64];
  __shared__ int bad;
  __shared__ int last;
  step_mc_block<PLAIN>(a, step_index, pl, k1a, fuse, b0, nbk, kf, blockIdx.x, blockIdx.y, threadIdx.x,
                       [] { __syncthreads(); }, sh, &bad, &last);
}

cudaError_t step_diag_mc_launch(const StepArgs& a, int step_index, const K1Plan* k1, const K1Args* k1a, int b0, int nb,
                                int nbk, cudaStream_t s) {
  dim3 grid((unsigned)a.nblk, (unsigned)nb);
  K1Plan pl{};
  K1Args ka{};
  if (k1) pl = *k1;
  if (k1a) ka = *k1a;
  if (step_plain(a))
    k_step_diag_mc<true><<<grid, STEP_MC_THREADS, 0, s>>>(a, step_index, pl, ka, k1 ? 1 : 0, b0, nbk, K3TStepFuse{});
  else
    k_step_diag_mc<false><<<grid, STEP_MC_THREADS, 0, s>>>(a, step_index, pl, ka, k1 ? 1 : 0, b0, nbk, K3TStepFuse{});
  return cudaGetLastError();
}

static cudaError_t step_diag_mc_fused(const StepArgs& a, int step_index, int fuse, const K3TStepFuse& f,
                                      cudaStream_t s) {
  dim3 grid((unsigned)a.nblk, (unsigned)a.batch);
  if (step_plain(a))
    k_step_diag_mc<true><<<grid, STEP_MC_THREADS, 0, s>>>(a, step_index, K1Plan{}, K1Args{}, fuse, 0, 1, f);
  else
    k_step_diag_mc<false><<<grid, STEP_MC_THREADS, 0, s>>>(a, step_index, K1Plan{}, K1Args{}, fuse, 0, 1, f);
  return cudaGetLastError();
}

cudaError_t step_diag_mc_k3t_launch(const StepArgs& a, int step_index, const K3TStepFuse& f, cudaStream_t s) {
  return step_diag_mc_fused(a, step_index, 2, f, s);
}

cudaError_t step_diag_mc_k3d_launch(const StepArgs& a, int step_index, const K3TStepFuse& f, cudaStream_t s) {
  return step_diag_mc_fused(a, step_index, 3, f, s);
}

// Diagonal step fused with the finalize of the skew-packed streaming kernel
// (k1_packed.cuh): n^l_i = (row sums of test index i) - (transposed-term
// windows of every CTA at k = i), then the step of element i.  A block covers
// 32 test indices of one trajectory; warp w sums the windows of CTAs
// [w G/32, (w+1) G/32) and warp 0 adds the row sums and steps the elements.
// Energy/invariant partials of the blocks are summed in block order by the
// last block to arrive, which also advances the step count.
__global__ void __launch_bounds__(STEP_PK_THREADS) k_step_diag_packed(const StepArgs a, const int step_index,
                                                                      const K1Plan pl, const K1Args k1a,
                                                                      const int b0, const int nbk) {
  __shared__ double sh[32][33];
  __shared__ int fi_tab[STEP_PK_MAX_GRID];
  __shared__ int last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bl = blockIdx.y;
  const int b = b0 + bl;
  if (a.active && !a.active[b]) return;  // uniform over the block
  const int64_t n = a.n;
  const int G = pl.grid;
  const int64_t T = pl.T;
  for (int g = threadIdx.x; g < G; g += blockDim.x) fi_tab[g] = (int)(((int64_t)g * T / G) / pl.cpi);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  double s = 0.0;
  if (i < n) {
    const int g0 = warp * G / 32, g1 = (warp + 1) * G / 32;
    if (pl.lw <= n && g1 - g0 <= 8) {
      // at most one window entry per CTA: independent loads, summed in CTA order
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int g = g0 + q;
        v[q] = 0.0;
        if (g < g1) {
          int64_t w = i - fi_tab[g] - 1;
          if (w < 0) w += n;
          if (w < pl.lw) v[q] = k1a.tg[((int64_t)g * nbk + bl) * pl.lw + w];
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) s += v[q];
    } else {
      for (int g = g0; g < g1; ++g) {
        int64_t w = i - fi_tab[g] - 1;
        if (w < 0) w += n;
        const double* win = k1a.tg + ((int64_t)g * nbk + bl) * pl.lw;
        for (; w < pl.lw; w += n) s += win[w];
      }
    }
  }
  sh[warp][lane] = s;
  double rs = 0.0;
  if (warp == 0 && i < n) {
    const int64_t g_lo = ((i * pl.cpi + 1) * G - 1) / T, g_hi = (((i + 1) * pl.cpi) * G - 1) / T;
    for (int64_t g = g_lo; g <= g_hi; ++g) {
      const double* src = k1a.part + ((g * pl.maxseg + (i - fi_tab[g])) * (K1_CONSUMERS / 32)) * nbk + bl;
      double v[K1_CONSUMERS / 32];
#pragma unroll
      for (int w = 0; w < K1_CONSUMERS / 32; ++w) v[w] = src[w * nbk];
#pragma unroll
      for (int w = 0; w < K1_CONSUMERS / 32; ++w) rs += v[w];
    }
  }
  __syncthreads();
  if (warp != 0) return;
  const int64_t l = a.taken[b];
  const int k = (int)(l + 1 < a.order ? l + 1 : a.order);
  double* h = a.hist + b * a.hist_stride;
  double e_part = 0.0, i_part = 0.0;
  int bad = 0;
  if (i < n) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 32; ++w) t += sh[w][lane];
    const double nl = rs - t;
    h[(3 + l % 3) * n + i] = nl;
    step_elem(a, h, n, l, k, i, nl, e_part, i_part, bad);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    e_part += __shfl_down_sync(0xffffffffu, e_part, off);
    i_part += __shfl_down_sync(0xffffffffu, i_part, off);
  }
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    if (bad) report_nonfinite(a, b);
    double* r = a.red + ((int64_t)b * a.nblk + blockIdx.x) * 2;
    r[0] = e_part;
    r[1] = i_part;
    __threadfence();
    const unsigned prev = atomicAdd(&a.cnt[b], 1u);
    last = prev == (unsigned)(a.nblk - 1);
  }
  __syncwarp();
  if (last) step_finish_last(a, b, l, step_index);
}

cudaError_t step_diag_packed_launch(const StepArgs& a0, int step_index, const K1Plan& pl, const K1Args& k1a, int b0,
                                    int nb, int nbk, cudaStream_t s) {
  if (pl.grid > STEP_PK_MAX_GRID) return cudaErrorInvalidValue;
  StepArgs a = a0;
  a.nblk = step_pk_blocks(a.n);
  dim3 grid((unsigned)a.nblk, (unsigned)nb);
  k_step_diag_packed<<<grid, STEP_PK_THREADS, 0, s>>>(a, step_index, pl, k1a, b0, nbk);
  return cudaGetLastError();
}

// ------------------------------------------------------------ dense path
// work layout per trajectory: [y | t | z | v] (n each)

__global__ void k_step_prep(const StepArgs a) {
  const int b = blockIdx.y;
  if (a.active && !a.active[b]) return;
  const int64_t n = a.n;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t l = a.taken[b];
  const int k = (int)(l + 1 < a.order ? l + 1 : a.order);
  const double* h = a.hist + b * a.hist_stride;
  double* w = a.work + (int64_t)b * 4 * n;
  double y = 0.0, t = 0.0, z = 0.0;
  const double f = a.forcing ? a.forcing[i] : 0.0;
  for (int q = 0; q < k; ++q) {
    const int64_t m = ((l - q) % 3 + 3) % 3;
    const double uq = h[m * n + i];
    y -= c_alpha[k - 1][q] * (h[(3 + m) * n + i] + f);
    t += c_beta[k - 1][q + 1] * a.inv_dt * uq;
    z += c_alpha[k - 1][q] * uq;
  }
  if (!a.mass) y -= (a.mass_diag ? a.mass_diag[i] : 1.0) * t;
  if (!a.linear && a.lin_diag) y -= a.lin_diag[i] * z;
  w[i] = y;
  w[n + i] = t;
  w[2 * n + i] = z;
}

// out[b] (+)= sign * M x[b]; one warp per row.  mode: 0 = L z -> y, 1 = B t -> y,
// 2 = H_k^{-1} y -> v, 3 = B v -> t (for the energy).
__global__ void k_step_gemv(const StepArgs a, const int mode) {
  const int b = blockIdx.y;
  if (a.active && !a.active[b]) return;
  const int64_t n = a.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= n) return;
  double* w = a.work + (int64_t)b * 4 * n;
  const double* M;
  const double* x;
  if (mode == 0) {
    M = a.linear; x = w + 2 * n;
  } else if (mode == 1) {
    M = a.mass; x = w + n;
  } else if (mode == 2) {
    const int64_t l = a.taken[b];
    const int k = (int)(l + 1 < a.order ? l + 1 : a.order);
    M = a.hinv[k - 1]; x = w;
  } else {
    M = a.mass; x = w + 3 * n;
  }
  double s = 0.0;
  for (int64_t j = lane; j < n; j += 32) s = fma(M[i * n + j], x[j], s);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    if (mode == 0 || mode == 1) w[i] -= s;        // y -= L z, y -= B t
    else if (mode == 2) w[3 * n + i] = s;         // v = H^-1 y
    else w[n + i] = s;                            // t = B v
  }
}

__global__ void __launch_bounds__(STEP_THREADS) k_step_finish(const StepArgs a, const int step_index, const int use_hdiag) {
  __shared__ double sh[64];
  __shared__ int bad;
  const int b = blockIdx.x;
  if (a.active && !a.active[b]) return;
  const int64_t n = a.n;
  const int64_t l = a.taken[b];
  const int k = (int)(l + 1 < a.order ? l + 1 : a.order);
  double* h = a.hist + b * a.hist_stride;
  double* w = a.work + (int64_t)b * 4 * n;
  const int64_t m0 = l % 3;
  double* u_new = h + ((l + 1) % 3) * n;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  double e_part = 0.0, i_part = 0.0;
  int my_bad = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double un = use_hdiag ? w[i] * a.hdiag[k - 1][i] : w[3 * n + i];
    i_part += h[m0 * n + i] * h[(3 + m0) * n + i];
    const double bu = a.mass ? w[n + i] : (a.mass_diag ? a.mass_diag[i] : 1.0) * un;
    e_part += un * bu;
    if (!isfinite(un)) my_bad = 1;
    u_new[i] = un;
  }
  if (my_bad) bad = 1;
  block_sum2(e_part, i_part, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (a.energy) a.energy[(int64_t)step_index * a.batch + b] = 0.5 * e_part;
    if (a.invariant) a.invariant[(int64_t)step_index * a.batch + b] = i_part;
    if (bad) report_nonfinite(a, b);
    step_done(a, b, l);
  }
}

// v = hdiag_k * y for the energy pass when H is diagonal but B is dense.
__global__ void k_step_hdiag(const StepArgs a) {
  const int b = blockIdx.y;
  if (a.active && !a.active[b]) return;
  const int64_t n = a.n;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t l = a.taken[b];
  const int k = (int)(l + 1 < a.order ? l + 1 : a.order);
  double* w = a.work + (int64_t)b * 4 * n;
  w[3 * n + i] = w[i] * a.hdiag[k - 1][i];
}

cudaError_t step_launch_indexed(const StepArgs& a, bool diagonal, int step_index, cudaStream_t s) {
  if (diagonal) return step_diag_mc_launch(a, step_index, nullptr, nullptr, 0, a.batch, 1, s);
  const int64_t n = a.n;
  dim3 ge((unsigned)((n + 255) / 256), (unsigned)a.batch);
  dim3 gw((unsigned)((n + 7) / 8), (unsigned)a.batch);
  k_step_prep<<<ge, 256, 0, s>>>(a);
  if (a.linear) k_step_gemv<<<gw, 256, 0, s>>>(a, 0);
  if (a.mass) k_step_gemv<<<gw, 256, 0, s>>>(a, 1);
  const bool hdense = a.hinv[0] != nullptr;
  if (hdense) {
    k_step_gemv<<<gw, 256, 0, s>>>(a, 2);
  } else if (a.mass) {
    k_step_hdiag<<<ge, 256, 0, s>>>(a);
  }
  if (a.mass) k_step_gemv<<<gw, 256, 0, s>>>(a, 3);
  k_step_finish<<<a.batch, STEP_THREADS, 0, s>>>(a, step_index, (hdense || a.mass) ? 0 : 1);
  return cudaGetLastError();
}

// Serving admission: slot slots[q] gets the initial state u0s[q] (no steps
// taken, empty history), a budget of horizons[q] steps and is activated.
__global__ void k_slot_admit(double* hist, int64_t* taken, int32_t* steps_left, int32_t* active, int64_t n,
                             int count, const int32_t* slots, const int32_t* horizons, const double* u0s) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)count * 6 * n) return;
  const int q = (int)(t / (6 * n));
  const int64_t e = t - (int64_t)q * 6 * n;
  const int b = slots[q];
  hist[(int64_t)b * 6 * n + e] = e < n ? u0s[(int64_t)q * n + e] : 0.0;
  if (e == 0) {
    taken[b] = 0;
    steps_left[b] = horizons[q];
    active[b] = 1;
  }
}

cudaError_t slot_admit_launch(double* hist, int64_t* taken, int32_t* steps_left, int32_t* active, int64_t n,
                              int count, const int32_t* slots, const int32_t* horizons, const double* u0s,
                              cudaStream_t s) {
  const int64_t total = (int64_t)count * 6 * n;
  k_slot_admit<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(hist, taken, steps_left, active, n, count, slots,
                                                               horizons, u0s);
  return cudaGetLastError();
}

__global__ void k_state_io(double* hist, const int64_t* taken, int64_t n, int batch, double* u, int inject) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * batch) return;
  const int64_t b = t / n, i = t - b * n;
  double* slot = hist + b * 6 * n + (taken[b] % 3) * n;
  if (inject)
    slot[i] = u[t];
  else
    u[t] = slot[i];
}

cudaError_t state_io_launch(double* hist, const int64_t* taken, int64_t n, int batch, double* u, bool inject,
                            cudaStream_t s) {
  const int64_t total = n * batch;
  k_state_io<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(hist, taken, n, batch, u, inject ? 1 : 0);
  return cudaGetLastError();
}


}  // namespace grom

namespace grom {

// Self-test of the bounded device waits: waits on an mbarrier that nothing
// ever arrives on, gives up after limit_ns and raises the timeout flag, as
// the production kernels do.
__global__ void k_selftest_wait(int* err, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !ptx::mbar_wait_limit(&bar, 0, nullptr, limit_ns)) atomicOr(err, DEV_ERR_TIMEOUT);
}

cudaError_t selftest_wait_launch(int* err, uint64_t limit_ns, cudaStream_t s) {
  k_selftest_wait<<<1, 32, 0, s>>>(err, limit_ns);
  return cudaGetLastError();
}

}  // namespace grom
