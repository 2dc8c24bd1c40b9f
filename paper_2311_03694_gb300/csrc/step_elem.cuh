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
// FP64 runs at about two operations per clock per SM on this part, so the
// terms of absent operators (mass, linear, forcing: null pointers, uniform
// branches) are skipped, beta/dt comes from the host, the energy and
// invariant terms are formed only when `sums` is set, and finiteness is
// read from the exponent bits: about eight FP64 operations per element in
// the common case.  PLAIN (no mass, linear or forcing term, no sums) removes
// those terms at compile time: a runtime test still issues its predicated
// FP64 instructions, which measured ~26 FP64 instructions per element on the
// batched step against the 8 of the plain arithmetic.
template <bool PLAIN = false>
__device__ __forceinline__ double step_elem(const StepArgs& a, double* h, int64_t n, int64_t l, int k, int64_t i,
                                            double nl, double& e_part, double& i_part, int& bad, bool sums = true) {
  const bool lin = !PLAIN && a.lin_diag != nullptr, frc = !PLAIN && a.forcing != nullptr,
             mass = !PLAIN && a.mass_diag != nullptr;
  if (PLAIN) sums = false;
  const double ld = lin ? a.lin_diag[i] : 0.0;
  const double f = frc ? a.forcing[i] : 0.0;
  const int m0 = (int)(l % 3);
  double ext = 0.0, bdf = 0.0, u0 = 0.0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q < k) {
      const int m = m0 - q < 0 ? m0 - q + 3 : m0 - q;
      const double uq = h[m * n + i];
      double g = q == 0 ? nl : h[(3 + m) * n + i];
      if (q == 0) u0 = uq;
      if (lin) g = fma(ld, uq, g);
      if (frc) g += f;
      ext = fma(c_alpha[k - 1][q], g, ext);
      bdf = fma(a.bdt[k - 1][q], uq, bdf);
    }
  }
  double un, mb = 1.0;
  if (mass) {
    mb = a.mass_diag[i];
    un = fma(-mb, bdf, -ext) * a.hdiag[k - 1][i];
  } else {
    un = -(ext + bdf) * a.hdiag[k - 1][i];
  }
  e_part = 0.0;
  i_part = 0.0;
  if (sums) {
    // explicit roundings: the products must not contract into the caller's
    // sums (FMA), whose form would then depend on the kernel inlining them
    e_part = mass ? __dmul_rn(__dmul_rn(mb, un), un) : __dmul_rn(un, un);
    i_part = __dmul_rn(u0, nl);
  }
  bad = ((__double_as_longlong(un) >> 52) & 0x7FF) == 0x7FF;  // inf or NaN
  h[((l + 1) % 3) * n + i] = un;
  return un;
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
  const int nsum = (a.energy || a.invariant) ? a.nblk : 0;  // no sums asked for: only the step count
  for (int q = lane; q < nsum; q += 32) {
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
