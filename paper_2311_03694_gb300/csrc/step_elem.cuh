// BDFk/EXTk coefficients and the per-element diagonal step (Sec. 2.2,
// eq. nse_d1), shared by the step kernels.  Each translation unit that
// includes this gets its own copy of the constant tables.
#pragma once

#include "grom_internal.h"

namespace grom {

// beta_0 .. beta_k of BDFk and alpha_1 .. alpha_k of EXTk, k = 1, 2, 3
static __constant__ double c_beta[3][4] = {
    {1.0, -1.0, 0.0, 0.0},
    {1.5, -2.0, 0.5, 0.0},
    {11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0},
};
static __constant__ double c_alpha[3][3] = {
    {1.0, 0.0, 0.0},
    {2.0, -1.0, 0.0},
    {3.0, -3.0, 1.0},
};

// One element of the diagonal step: u^{l+1}_i from the history and n^l_i = nl.
__device__ __forceinline__ void step_elem(const StepArgs& a, double* h, int64_t n, int64_t l, int k, int64_t i,
                                          double nl, double& e_part, double& i_part, int& bad) {
  const double mb = a.mass_diag ? a.mass_diag[i] : 1.0;
  const double ld = a.lin_diag ? a.lin_diag[i] : 0.0;
  const double f = a.forcing ? a.forcing[i] : 0.0;
  const double inv_dt = 1.0 / a.dt;
  double ext = 0.0, bdf = 0.0, u0 = 0.0;
  for (int q = 0; q < k; ++q) {
    const int64_t m = ((l - q) % 3 + 3) % 3;
    const double uq = h[m * n + i];
    const double nq = q == 0 ? nl : h[(3 + m) * n + i];
    if (q == 0) u0 = uq;
    ext += c_alpha[k - 1][q] * (nq + ld * uq + f);
    bdf += c_beta[k - 1][q + 1] * inv_dt * uq;
  }
  const double un = (-ext - mb * bdf) * a.hdiag[k - 1][i];
  i_part = u0 * nl;
  e_part = mb * un * un;
  bad = !isfinite(un);
  h[((l + 1) % 3) * n + i] = un;
}

// Called by all lanes of one warp of the last block of trajectory b to
// arrive: sums the nblk per-block (energy, invariant) partials (lane q adds
// blocks q, q+32, ... in order, then a fixed shuffle tree), writes the outputs
// and advances the step count.
__device__ __forceinline__ void step_finish_last(const StepArgs& a, int b, int64_t l, int step_index) {
  const int lane = threadIdx.x & 31;
  __threadfence();
  double e = 0.0, inv = 0.0;
  const double* rr = a.red + (int64_t)b * a.nblk * 2;
  for (int q = lane; q < a.nblk; q += 32) {
    e += __ldcg(rr + 2 * q);
    inv += __ldcg(rr + 2 * q + 1);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, off);
    inv += __shfl_xor_sync(0xffffffffu, inv, off);
  }
  if (lane == 0) {
    if (a.energy) a.energy[(int64_t)step_index * a.batch + b] = 0.5 * e;
    if (a.invariant) a.invariant[(int64_t)step_index * a.batch + b] = inv;
    step_done(a, b, l);
    a.cnt[b] = 0u;
  }
}

}  // namespace grom
