// One block of the multi-CTA diagonal step (k_step_diag_mc): the elements
// ((blk * ept + e) * STEP_MC_THREADS + tid) of trajectory b0 + bl, their
// energy/invariant partial, and, for the last block of the trajectory to
// arrive, the fixed-order sum of all blocks' partials and the step count.
// Written once for the standalone kernel (a CTA of STEP_MC_THREADS threads,
// __syncthreads) and the persistent batched stepper (the first
// STEP_MC_THREADS threads of its CTA, a named barrier), so both compute the
// same bits.
#pragma once

#include <cuda_bf16.h>

#include "ds_arith.cuh"
#include "grom_internal.h"
#include "step_elem.cuh"

namespace grom {

// Deterministic sum of two values over the nw warps of the calling threads
// (a fixed shuffle tree, then warp 0 over the warp sums); result in thread 0.
template <typename Sync>
__device__ __forceinline__ void block_sum2_n(double& x, double& y, double* sh, int tid, int nw, Sync sync) {
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, off);
    y += __shfl_down_sync(0xffffffffu, y, off);
  }
  if (lane == 0) {
    sh[warp] = x;
    sh[32 + warp] = y;
  }
  sync();
  if (warp == 0) {
    x = lane < nw ? sh[lane] : 0.0;
    y = lane < nw ? sh[32 + lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, off);
      y += __shfl_down_sync(0xffffffffu, y, off);
    }
  }
}

__device__ __forceinline__ void report_nonfinite(const StepArgs& a, int b) {
  atomicOr(a.err, DEV_ERR_NONFINITE);
  atomicMin(a.first_bad, b);
}

// fuse: 0 n^l from the history ring; 1 the K1 partials (finalize fused);
// 2 the K3T expansion partials, with the new state's BF16 hi/lo rows written
// for the next projections (the values the state prep would write);
// 3 the K3D expansion's double-single split pairs (or, with one split, the
// ring, which the expansion wrote), with the new state's FP32 hi/lo planes
// ([i][b], pitch np) written for the next projections.
// PLAIN: identity mass, no linear or forcing term, no energy or invariant.
template <bool PLAIN, typename Sync>
__device__ __forceinline__ void step_mc_block(const StepArgs& a, int step_index, const K1Plan& pl, const K1Args& k1a,
                                              int fuse, int b0, int nbk, const K3TStepFuse& kf, int blk, int bl,
                                              int tid, Sync sync, double* sh, volatile int* bad,
                                              volatile int* last) {
  const int b = b0 + bl;  // trajectory index
  if (a.active && !a.active[b]) return;
  const int64_t n = a.n;
  const int64_t l = a.taken[b];
  const int k = (int)(l + 1 < a.order ? l + 1 : a.order);
  double* h = a.hist + b * a.hist_stride;
  if (tid == 0) *bad = 0;
  sync();
  const bool sums = !PLAIN && (a.energy || a.invariant);  // energy and invariant asked for
  double e_part = 0.0, i_part = 0.0;
  int my_bad = 0;
  for (int e = 0; e < a.ept; ++e) {
    const int64_t i = ((int64_t)blk * a.ept + e) * STEP_MC_THREADS + tid;
    if (i >= n) break;
    double nl;
    if (fuse == 3) {
      // expansion splits in split order, double-single (as the K3D finish)
      if (kf.s2 > 1) {
        const int64_t oplane = kf.bp * n;
        float S = 0.f, s = 0.f;
        for (int q0 = 0; q0 < kf.s2; q0 += 4) {  // four splits' loads in flight, summed in split order
          float w[4][2];
#pragma unroll
          for (int z = 0; z < 4; ++z)
            if (q0 + z < kf.s2) {
              const float* p = kf.d2 + (int64_t)(q0 + z) * 2 * oplane + (int64_t)b * n + i;
              w[z][0] = __ldcg(p);
              w[z][1] = __ldcg(p + oplane);
            }
#pragma unroll
          for (int z = 0; z < 4; ++z)
            if (q0 + z < kf.s2) ds_add(S, s, w[z][0], w[z][1]);
        }
        nl = (double)S + (double)s;
        h[(3 + l % 3) * n + i] = nl;
      } else {
        nl = h[(3 + l % 3) * n + i];
      }
    } else if (fuse == 2) {
      // expansion splits in split order, FP64
      double sum = 0.0;
      for (int q = 0; q < kf.s2; ++q) sum += (double)kf.d2[((int64_t)q * kf.bp + b) * n + i];
      h[(3 + l % 3) * n + i] = sum;
      nl = sum;
    } else if (fuse) {
      // K1 finalize: partials of every CTA whose chunk range covers test index i, in CTA order
      const int64_t G = pl.grid, T = pl.T;
      const int64_t g_lo = ((i * pl.cpi + 1) * G - 1) / T, g_hi = (((i + 1) * pl.cpi) * G - 1) / T;
      double sum = 0.0;
      for (int64_t g = g_lo; g <= g_hi; ++g) {
        const int64_t first_i = (g * T / G) / pl.cpi;
        const double* src = k1a.part + ((g * pl.maxseg + (i - first_i)) * (K1_CONSUMERS / 32)) * nbk + bl;
#pragma unroll
        for (int w = 0; w < K1_CONSUMERS / 32; ++w) sum += src[w * nbk];
      }
      h[(3 + l % 3) * n + i] = sum;
      nl = sum;
    } else {
      nl = h[(3 + l % 3) * n + i];
    }
    double ep, ip;
    int eb;
    const double un = step_elem<PLAIN>(a, h, n, l, k, i, nl, ep, ip, eb, sums);
    if (fuse == 3) {
      float hi, lo;
      ds_split(un, hi, lo);
      static_cast<float*>(kf.xh)[i * kf.np + b] = hi;  // planes [i][b]
      static_cast<float*>(kf.xl)[i * kf.np + b] = lo;
    } else if (fuse == 2) {
      const float v = __double2float_rn(un);
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      static_cast<__nv_bfloat16*>(kf.xh)[(int64_t)b * kf.np + i] = hi;
      static_cast<__nv_bfloat16*>(kf.xl)[(int64_t)b * kf.np + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
    if (sums) {
      e_part = __dadd_rn(e_part, ep);
      i_part = __dadd_rn(i_part, ip);
    }
    my_bad |= eb;
  }
  if (my_bad) *bad = 1;
  if (sums) {
    block_sum2_n(e_part, i_part, sh, tid, STEP_MC_THREADS / 32, sync);
  } else {
    sync();  // `bad` complete before thread 0 reads it
  }
  if (tid == 0) {
    if (*bad) report_nonfinite(a, b);
    double* r = a.red + ((int64_t)b * a.nblk + blk) * 2;
    r[0] = e_part;
    r[1] = i_part;
    __threadfence();
    const unsigned prev = atomicAdd(&a.cnt[b], 1u);
    *last = prev == (unsigned)(a.nblk - 1);
  }
  sync();
  if (*last && tid < 32) step_finish_last(a, b, l, step_index);
}

}  // namespace grom
