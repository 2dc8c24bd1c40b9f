// K3O: the batched CP-form advection term (Sec. 3.1, eq. tc_ap; skew
// structure Sec. 3.3) of FP64 ROMs at FP64 tolerance on the BF16 tensor
// cores, by splitting every operand into integer slices (Ozaki's scheme for
// accurate matrix products from low-precision ones).
//
// A vector x that enters a dot product (a row of a factor over the summed
// index, or a state) is scaled by sigma = 2^ceil(log2 max|x|) and written as
// x = sigma sum_{p < S} d_p 2^-6(p+1) with integer digits d_p (|d_0| <= 64,
// |d_p| <= 32 after), each taken by rounding what the previous digits left
// (exact in FP64).  Digits are exact in BF16, a product of two is at most
// 2^12, and a sum of K <= 4096 of them at most 2^24, so every slice-by-slice
// dot product that the tensor cores accumulate in FP32 is exact, whatever
// the inputs.  The dot product is then
//   x . v = sigma_x sigma_v sum_{p + q < S} 2^-6(p+q+2) (d^x_p . d^v_q)
// truncated to the triangle p + q < S (45 slice pairs with S = 9).  A CPU
// emulation of the whole evaluation on the workload's factors gives 5.1e-15
// per evaluation against FP64 at N = R = 1024 (1.2e-12 with S = 8; with
// 7-bit digits, 2.7e-15 at S = 8, but exactness then holds only for K <=
// 1024).  The projections of ROMs of N <= 1024 (K = N) therefore use eight
// 7-bit digits (36 slice pairs, exact; 2.7e-15 in the emulation), the
// expansion (K = 2R or R, up to 4096) the nine 6-bit ones.  The sums over
// slice pairs run in double-single FP32 arithmetic (ds_arith.cuh) from the
// smallest weights up.
//
//   slice_states  per trajectory: the state's scale and digits        (B rows)
//   gemm          D1 = [digits of V W U]^T x [digits of the states]   (tcgen05)
//   combine_proj  P, Q, S per (r, b) from D1, H1 = P o Q, H2 = P o S,
//                 and each trajectory's largest |H|
//   slice_h       per trajectory: the scale and digits of [H1 H2]
//   gemm          D2 = [digits of U, -W] x [digits of H]             (tcgen05)
//   combine_exp   c per (b, i) from D2, FP64 into the output or the ring
// The factor digits and scales are made once, at create.  The GEMM computes
// only the 128 x 128 tiles that hold a slice pair of the triangle.
#include <algorithm>

#include <cuda_bf16.h>

#include "ds_arith.cuh"
#include "grom_internal.h"
#include "step_mc.cuh"

namespace grom {

constexpr int OZ_S = 9;     // slices per operand: 6-bit digits (exact for K <= 4096)
constexpr int OZ_BITS = 6;
constexpr int OZ_S7 = 8;    // projections of N <= 1024: 7-bit digits (exact for K <= 1024)
constexpr int OZ_BITS7 = 7;
constexpr int64_t OZ_MAX_K = 4096;  // longest exact dot product of 6-bit digits
constexpr int64_t OZ_MAX_K7 = 1024; // of 7-bit digits

static inline int64_t oz_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct ODims {
  int64_t n, rp, r;  // modes, pitch of the FP64 factor panels, rank
  int nf, nt;        // projected factors (3 skew, 2 general), expansion terms (2, 1)
  int64_t mp;        // projection rows per slice: nf r rounded up to 128
  int64_t nk;        // projection K: n rounded up to 64
  int64_t me;        // expansion rows per slice: n rounded up to 128
  int64_t rk;        // expansion K: nt r rounded up to 64
  int64_t bq;        // columns per slice: the batch rounded up to 64
  int64_t nc;        // expansion GEMM columns: S bq rounded up to the GEMM's tile width (the rest unused)
  int sp;            // projection slices: OZ_S7 (7-bit digits) when nk <= OZ_MAX_K7, else OZ_S
  int64_t ncp;       // projection GEMM columns: sp bq rounded up likewise
  int batch;
};

static ODims oz_dims(int64_t n, int64_t rp, int64_t r, int form, int batch) {
  ODims d{};
  d.n = n;
  d.rp = rp;
  d.r = r;
  d.nf = form == GROM_FORM_CP_SKEW ? 3 : 2;
  d.nt = form == GROM_FORM_CP_SKEW ? 2 : 1;
  d.mp = oz_up(d.nf * r, 128);
  d.nk = oz_up(n, 64);
  d.me = oz_up(n, 128);
  d.rk = oz_up(d.nt * r, 64);
  d.bq = oz_up(batch, 64);
  d.nc = oz_up(OZ_S * d.bq, 128);
  if (d.nc >= 512) d.nc = oz_up(d.nc, 256);  // the GEMM's 256-wide tiles
  d.sp = d.nk <= OZ_MAX_K7 ? OZ_S7 : OZ_S;
  d.ncp = oz_up((int64_t)d.sp * d.bq, 128);
  if (d.ncp >= 512) d.ncp = oz_up(d.ncp, 256);
  d.batch = batch;
  return d;
}

static size_t oz_round(size_t b) { return (b + 255) / 256 * 256; }

// Factor data: [digits of the projected factors: S x mp x nk BF16]
// [digits of the expansion factors: S x me x rk BF16] [scale exponents:
// mp + me ints].  A scale is 2^e with every entry of its vector below 2^e.
struct OFactors {
  size_t aproj, aexp, sproj, sexp, total;
};
static OFactors oz_factor_layout(const ODims& d) {
  OFactors L{};
  L.aproj = 0;
  L.aexp = oz_round(2 * (size_t)d.sp * d.mp * d.nk);
  L.sproj = L.aexp + oz_round(2 * (size_t)OZ_S * d.me * d.rk);
  L.sexp = L.sproj + oz_round(4 * (size_t)d.mp);
  L.total = L.sexp + oz_round(4 * (size_t)d.me);
  return L;
}

// Scratch of a batch: [state digits: nc x nk BF16, slice q at rows q bq]
// [state scale exponents: bq] [D1: nc x (S mp) FP32] [H hi and lo: 2 x nt x
// bq x r FP32] [bits of max |H hi|: bq] [H digits: nc x rk BF16] [H scale
// exponents: bq] [D2: nc x (S me) FP32].  Rows past S bq of the digit
// planes are GEMM padding whose products are never read.
struct OScratch {
  size_t bst, tau, d1, h, hmax, bh, tau2, d2, total;
};
static OScratch oz_scratch_layout(const ODims& d) {
  OScratch L{};
  size_t off = 0;
  L.bst = off;
  off += oz_round(2 * (size_t)d.ncp * d.nk);
  L.tau = off;
  off += oz_round(4 * (size_t)d.bq);
  L.d1 = off;
  off += oz_round(4 * (size_t)d.ncp * d.sp * d.mp);
  L.h = off;
  off += oz_round(4 * 2 * (size_t)d.nt * d.bq * d.r);
  L.hmax = off;
  off += oz_round(4 * (size_t)d.bq);
  L.bh = off;
  off += oz_round(2 * (size_t)d.nc * d.rk);
  L.tau2 = off;
  off += oz_round(4 * (size_t)d.bq);
  L.d2 = off;
  off += oz_round(4 * (size_t)d.nc * OZ_S * d.me);
  L.total = off;
  return L;
}

// Everything per element is integer arithmetic on the bit patterns: this
// part's FP64 pipe is slow.  A value x with |x| < 2^e becomes the F-bit
// fixed-point integer Y = rint(x 2^(F - e)) (|Y| <= 2^F), from its
// significand and exponent: significand m, x = m 2^(ex - bias - mbits).
__device__ __forceinline__ long long oz_fix(long long m, int sh, bool neg) {
  long long Y;
  if (sh >= 0)
    Y = m << sh;  // sh <= 1 when |x| < 2^e
  else if (sh > -63)
    Y = (m + (1LL << (-sh - 1))) >> -sh;
  else
    Y = 0;
  return neg ? -Y : Y;
}
// F = S BITS fixed-point bits (54 for 6-bit digits, 56 for 7-bit ones).
template <int F>
__device__ __forceinline__ long long oz_fix_d(double x, int e) {
  const long long B = __double_as_longlong(x);
  const int ex = (int)((B >> 52) & 0x7ff);
  if (ex == 0) return 0;  // zero or below 2^-1022: far below the last digit
  return oz_fix((B & 0xfffffffffffffLL) | 0x10000000000000LL, ex - 1075 + F - e, B < 0);
}
template <int F>
__device__ __forceinline__ long long oz_fix_f(float x, int e) {
  const int B = __float_as_int(x);
  const int ex = (B >> 23) & 0xff;
  if (ex == 0) return 0;
  return oz_fix((long long)((B & 0x7fffff) | 0x800000), ex - 150 + F - e, B < 0);
}

// The S digits of Y: balanced base-2^BITS digits from the top, each the
// rounded quotient of what the digits before it left (|d_0| <= 2^BITS,
// |d_p| <= 2^(BITS-1) after); sum_p d_p 2^(BITS (S - 1 - p)) = Y exactly.
template <int S, int BITS>
__device__ __forceinline__ void oz_digits(long long Y, __nv_bfloat16 (&dg)[S]) {
#pragma unroll
  for (int p = 0; p < S; ++p) {
    const int sh = BITS * (S - 1 - p);
    const long long d = sh ? (Y + (1LL << (sh - 1))) >> sh : Y;
    Y -= d << sh;
    dg[p] = __int2bfloat16_rn((int)d);
  }
}

// The scale exponent of a vector from the bits of its largest magnitude:
// every entry below 2^e (e = 0 for a zero vector).
__device__ __forceinline__ int oz_exp_d(unsigned long long maxbits) {
  return maxbits ? (int)(maxbits >> 52) - 1023 + 1 : 0;
}
__device__ __forceinline__ int oz_exp_f(unsigned int maxbits) { return maxbits ? (int)(maxbits >> 23) - 127 + 1 : 0; }

// Block-wide maximum (256 threads), in every thread.
__device__ __forceinline__ unsigned long long oz_block_max(unsigned long long v, unsigned long long* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ull;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
      v = o > v ? o : v;
    }
    if (lane == 0) sh[32] = v;
  }
  __syncthreads();
  const unsigned long long m = sh[32];
  __syncthreads();
  return m;
}

__device__ __forceinline__ unsigned long long oz_absbits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// ------------------------------------------------------------ factor data
// Projection row m = f r + j (f: fb, fc, fa; j the rank index): the column j
// of factor f over the modes k.  One CTA per row (padding rows: zeros).
template <int S, int BITS>
__global__ void __launch_bounds__(256) k3o_build_proj(const uint8_t* op, size_t panel_bytes, const ODims d,
                                                      __nv_bfloat16* aproj, int* sproj) {
  __shared__ unsigned long long sh[33];
  const int64_t m = blockIdx.x;
  const bool on = m < (int64_t)d.nf * d.r;
  const int f = on ? (int)(m / d.r) : 0;
  const int64_t j = on ? m - (int64_t)f * d.r : 0;
  const int q = f == 0 ? 1 : f == 1 ? 2 : 0;  // panel index: fb, fc, fa
  const double* F = reinterpret_cast<const double*>(op + (size_t)q * panel_bytes);
  unsigned long long mx = 0;
  if (on)
    for (int64_t k = threadIdx.x; k < d.n; k += blockDim.x) {
      const unsigned long long v = oz_absbits(F[k * d.rp + j]);
      mx = v > mx ? v : mx;
    }
  const int e = oz_exp_d(oz_block_max(mx, sh));
  if (threadIdx.x == 0) sproj[m] = e;
  for (int64_t k = threadIdx.x; k < d.nk; k += blockDim.x) {
    __nv_bfloat16 dg[S];
    oz_digits<S, BITS>(on && k < d.n ? oz_fix_d<S * BITS>(F[k * d.rp + j], e) : 0, dg);
#pragma unroll
    for (int p = 0; p < S; ++p) aproj[((int64_t)p * d.mp + m) * d.nk + k] = dg[p];
  }
}

// Expansion row i: [fa_i | -fc_i] (skew) or fa_i (general) over the rank.
__global__ void __launch_bounds__(256) k3o_build_exp(const uint8_t* op, size_t panel_bytes, const ODims d,
                                                     __nv_bfloat16* aexp, int* sexp) {
  __shared__ unsigned long long sh[33];
  const int64_t i = blockIdx.x;
  const bool on = i < d.n;
  const double* Fa = reinterpret_cast<const double*>(op);
  const double* Fc = reinterpret_cast<const double*>(op + 2 * panel_bytes);
  auto val = [&](int64_t k) -> double {
    if (!on || k >= (int64_t)d.nt * d.r) return 0.0;
    const int t = (int)(k / d.r);
    const int64_t j = k - (int64_t)t * d.r;
    return t == 0 ? Fa[i * d.rp + j] : -Fc[i * d.rp + j];
  };
  unsigned long long mx = 0;
  for (int64_t k = threadIdx.x; k < d.rk; k += blockDim.x) {
    const unsigned long long v = oz_absbits(val(k));
    mx = v > mx ? v : mx;
  }
  const int e = oz_exp_d(oz_block_max(mx, sh));
  if (threadIdx.x == 0) sexp[i] = e;
  for (int64_t k = threadIdx.x; k < d.rk; k += blockDim.x) {
    __nv_bfloat16 dg[OZ_S];
    oz_digits<OZ_S, OZ_BITS>(oz_fix_d<OZ_S * OZ_BITS>(val(k), e), dg);
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) aexp[((int64_t)p * d.me + i) * d.rk + k] = dg[p];
  }
}

// ------------------------------------------------------------ per evaluation
// CTAs (b, chunk of 256 modes), b < bq: the state's scale (each CTA of the
// column finds it) and the chunk's digits (zeros for padding and inactive
// trajectories); also clears the trajectory's largest |H|.
template <int S, int BITS>
__global__ void __launch_bounds__(256) k3o_slice_states(const ODims d, const K3Args a, __nv_bfloat16* bst, int* tau,
                                                        unsigned int* hmax) {
  __shared__ unsigned long long sh[33];
  const int b = blockIdx.x;
  const int64_t k0 = (int64_t)blockIdx.y * 256, k1 = k0 + 256 < d.nk ? k0 + 256 : d.nk;  // this CTA's digits
  const bool on = b < d.batch && (a.active == nullptr || a.active[b]);
  const double* u = on ? (a.taken ? a.hist + b * a.hist_stride + (a.taken[b] % 3) * d.n : a.u + b * a.u_stride)
                       : nullptr;
  unsigned long long mx = 0;
  if (on)
    for (int64_t k = threadIdx.x; k < d.n; k += blockDim.x) {
      const unsigned long long v = oz_absbits(u[k]);
      mx = v > mx ? v : mx;
    }
  const int e = oz_exp_d(oz_block_max(mx, sh));
  if (threadIdx.x == 0 && blockIdx.y == 0) {
    tau[b] = e;
    hmax[b] = 0u;
  }
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    __nv_bfloat16 dg[S];
    oz_digits<S, BITS>(on && k < d.n ? oz_fix_d<S * BITS>(u[k], e) : 0, dg);
#pragma unroll
    for (int p = 0; p < S; ++p) bst[((int64_t)p * d.bq + b) * d.nk + k] = dg[p];
  }
}

// The triangle's slice pairs of one output, D[(q bq + b) M + p mrows + m]:
// all loaded first (one round trip), each level L = p + q summed exactly in
// integers (|sum| <= 9 2^24 < 2^31), then the levels, weighted
// 2^-BITS(L+2), in double-single arithmetic from the smallest weight up.
template <int NS, int BITS>
__device__ __forceinline__ void oz_sum(const float* __restrict__ D, int64_t M, int64_t mrows, int64_t bq, int b,
                                       int64_t m, float& S, float& s) {
  float v[NS * (NS + 1) / 2];
#pragma unroll
  for (int L = 0, x = 0; L < NS; ++L)
#pragma unroll
    for (int p = 0; p <= L; ++p, ++x) v[x] = __ldcg(D + ((int64_t)(L - p) * bq + b) * M + (int64_t)p * mrows + m);
  S = 0.f;
  s = 0.f;
#pragma unroll
  for (int L = NS - 1; L >= 0; --L) {
    int acc = 0;
#pragma unroll
    for (int p = 0; p <= L; ++p) acc += __float2int_rn(v[L * (L + 1) / 2 + p]);
    const float hi = __int2float_rn(acc);
    const float lo = __int2float_rn(acc - __float2int_rz(hi));  // exact: |acc| < 2^31, |lo| <= 2^4
    const float w = __int_as_float((127 - BITS * (L + 2)) << 23);  // 2^-BITS(L+2)
    ds_add(S, s, __fmul_rn(hi, w), __fmul_rn(lo, w));
  }
}

// (S, s) times 2^e, exactly (e in the FP32 exponent range).
__device__ __forceinline__ void oz_scale_ds(float& S, float& s, int e) {
  const float f = __int_as_float((e + 127) << 23);
  S = __fmul_rn(S, f);
  s = __fmul_rn(s, f);
}

// CTAs (64 rank indices j, trajectory b), one thread per (factor, j): the
// factor's projection of j (P, Q or S) from D1; then, for each j, H1 = P o Q
// (and H2 = P o S) as double-single pairs and the bits of the trajectory's
// largest |H hi|.  (Three threads per output keep three times the loads in
// flight of one thread per (b, j).)
template <int S, int BITS>
__global__ void __launch_bounds__(192) k3o_combine_proj(const ODims d, const float* __restrict__ D1,
                                                        const int* __restrict__ sproj, const int* __restrict__ tau,
                                                        float* Hh, float* Hl, unsigned int* hmax) {
  __shared__ float V[3][64][2];
  const int f = threadIdx.x >> 6, jl = threadIdx.x & 63;
  const int b = blockIdx.y;
  const int64_t j = (int64_t)blockIdx.x * 64 + jl;
  const int64_t M = S * d.mp;
  if (f < d.nf && j < d.r) {
    const int64_t m = (int64_t)f * d.r + j;
    float hi, lo;
    oz_sum<S, BITS>(D1, M, d.mp, d.bq, b, m, hi, lo);
    oz_scale_ds(hi, lo, sproj[m] + tau[b]);
    V[f][jl][0] = hi;
    V[f][jl][1] = lo;
  }
  __syncthreads();
  if (f != 0 || j >= d.r) return;
  const int64_t hplane = (int64_t)d.bq * d.r;
  float h, l;
  ds_mul(V[0][jl][0], V[0][jl][1], V[1][jl][0], V[1][jl][1], h, l);
  Hh[(int64_t)b * d.r + j] = h;
  Hl[(int64_t)b * d.r + j] = l;
  unsigned int hm = (unsigned int)__float_as_int(h) & 0x7fffffffu;
  if (d.nt == 2) {
    ds_mul(V[0][jl][0], V[0][jl][1], V[2][jl][0], V[2][jl][1], h, l);
    Hh[hplane + (int64_t)b * d.r + j] = h;
    Hl[hplane + (int64_t)b * d.r + j] = l;
    const unsigned int h2 = (unsigned int)__float_as_int(h) & 0x7fffffffu;
    hm = h2 > hm ? h2 : hm;
  }
  atomicMax(&hmax[b], hm);
}

// CTAs (b, chunk of 256), b < bq: the scale and digits of [H1 | H2] of
// trajectory b.  The scale is twice the power of two above max |hi|, so that
// hi + lo stays below it.
__global__ void __launch_bounds__(256) k3o_slice_h(const ODims d, const K3Args a, const float* Hh, const float* Hl,
                                                   const unsigned int* hmax, __nv_bfloat16* bh, int* tau2) {
  const int b = blockIdx.x;
  const int64_t k0 = (int64_t)blockIdx.y * 256, k1 = k0 + 256 < d.rk ? k0 + 256 : d.rk;  // this CTA's digits
  const bool on = b < d.batch && (a.active == nullptr || a.active[b]);
  const int e = on && hmax[b] ? oz_exp_f(hmax[b]) + 1 : 0;
  if (threadIdx.x == 0 && blockIdx.y == 0) tau2[b] = e;
  const int64_t hplane = (int64_t)d.bq * d.r;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    long long Y = 0;
    if (on && k < (int64_t)d.nt * d.r) {
      const int t = (int)(k / d.r);
      const int64_t x = t * hplane + (int64_t)b * d.r + (k - (int64_t)t * d.r);
      Y = oz_fix_f<OZ_S * OZ_BITS>(Hh[x], e) + oz_fix_f<OZ_S * OZ_BITS>(Hl[x], e);
    }
    __nv_bfloat16 dg[OZ_S];
    oz_digits<OZ_S, OZ_BITS>(Y, dg);
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) bh[((int64_t)p * d.bq + b) * d.rk + k] = dg[p];
  }
}

// One thread per (b, i), i fastest: c_bi into the output or the ring.
__global__ void __launch_bounds__(256) k3o_combine_exp(const ODims d, const K3Args a, const float* __restrict__ D2,
                                                       const int* __restrict__ sexp, const int* __restrict__ tau2) {
  const int64_t total = (int64_t)d.batch * d.n;
  const int64_t M = OZ_S * d.me;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(o / d.n);
    const int64_t i = o - (int64_t)b * d.n;
    if (a.active && !a.active[b]) continue;
    float S, s;
    oz_sum<OZ_S, OZ_BITS>(D2, M, d.me, d.bq, b, i, S, s);
    oz_scale_ds(S, s, sexp[i] + tau2[b]);
    double* dst = a.taken ? a.hist + b * a.hist_stride + (3 + a.taken[b] % 3) * d.n : a.c + b * a.c_stride;
    dst[i] = (double)S + (double)s;
  }
}

// The expansion's combine fused with the diagonal BDF3/EXT3 step: a block of
// the step (k_step_diag_mc's grid and element mapping) first forms c_bi for
// exactly the elements its threads then step, as k3o_combine_exp does, and
// writes it into the history ring; each thread then reads back only what it
// wrote itself.  One launch and one pass over c fewer than the combine
// followed by the step kernel, with the same bits.
template <bool PLAIN>
__global__ void __launch_bounds__(STEP_MC_THREADS)
    k3o_exp_step(const ODims d, const float* __restrict__ D2, const int* __restrict__ sexp,
                 const int* __restrict__ tau2, const StepArgs st, const int step_index) {
  __shared__ double sh[64];
  __shared__ int bad;
  __shared__ int last;
  const int blk = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
  if (!st.active || st.active[b]) {
    const int64_t M = OZ_S * d.me;
    double* ring = st.hist + b * st.hist_stride + (3 + st.taken[b] % 3) * d.n;
    for (int e = 0; e < st.ept; ++e) {
      const int64_t i = ((int64_t)blk * st.ept + e) * STEP_MC_THREADS + tid;
      if (i >= d.n) break;
      float S, s;
      oz_sum<OZ_S, OZ_BITS>(D2, M, d.me, d.bq, b, i, S, s);
      oz_scale_ds(S, s, sexp[i] + tau2[b]);
      ring[i] = (double)S + (double)s;
    }
  }
  step_mc_block<PLAIN>(st, step_index, K1Plan{}, K1Args{}, 0, 0, 1, K3TStepFuse{}, blk, b, tid,
                       [] { __syncthreads(); }, sh, &bad, &last);
}

// ------------------------------------------------------------------- host
bool k3o_supported(int64_t n, int64_t r, int form) {
  const ODims d = oz_dims(n, r, r, form, 1);
  return d.nk <= OZ_MAX_K && d.rk <= OZ_MAX_K;
}

size_t k3o_factor_bytes(int64_t n, int64_t rp, int64_t r, int form) {
  return oz_factor_layout(oz_dims(n, rp, r, form, 1)).total;
}

size_t k3o_scratch_bytes(int64_t n, int64_t rp, int64_t r, int form, int max_batch) {
  return oz_scratch_layout(oz_dims(n, rp, r, form, max_batch)).total;  // grows with the batch
}

cudaError_t k3o_build_factors(const uint8_t* op, size_t panel_bytes, int64_t n, int64_t rp, int64_t r, int form,
                              void* out, cudaStream_t s) {
  const ODims d = oz_dims(n, rp, r, form, 1);
  const OFactors L = oz_factor_layout(d);
  uint8_t* base = static_cast<uint8_t*>(out);
  auto* ap = reinterpret_cast<__nv_bfloat16*>(base + L.aproj);
  auto* sp = reinterpret_cast<int*>(base + L.sproj);
  if (d.sp == OZ_S7)
    k3o_build_proj<OZ_S7, OZ_BITS7><<<(unsigned)d.mp, 256, 0, s>>>(op, panel_bytes, d, ap, sp);
  else
    k3o_build_proj<OZ_S, OZ_BITS><<<(unsigned)d.mp, 256, 0, s>>>(op, panel_bytes, d, ap, sp);
  k3o_build_exp<<<(unsigned)d.me, 256, 0, s>>>(op, panel_bytes, d, reinterpret_cast<__nv_bfloat16*>(base + L.aexp),
                                               reinterpret_cast<int*>(base + L.sexp));
  return cudaGetLastError();
}

static unsigned oz_flat_blocks(int64_t count, int sm_count) {
  const int64_t b = (count + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 8 * (int64_t)sm_count));
}

// Everything up to the expansion GEMM (digit slices of the states, the
// projections and their combine, the slices of [H1 H2], the expansion's
// slice products in d2); returns d2 and the expansion scales.
static cudaError_t k3o_front(const ODims& d, const K3Args& a, const void* factors, void* scratch, int* err,
                             int sm_count, cudaStream_t s, const float** d2_out, const int** sexp_out,
                             const int** tau2_out) {
  const OFactors F = oz_factor_layout(d);
  const OScratch L = oz_scratch_layout(d);
  const uint8_t* fb = static_cast<const uint8_t*>(factors);
  uint8_t* sb = static_cast<uint8_t*>(scratch);
  auto* bst = reinterpret_cast<__nv_bfloat16*>(sb + L.bst);
  auto* tau = reinterpret_cast<int*>(sb + L.tau);
  auto* d1 = reinterpret_cast<float*>(sb + L.d1);
  auto* hh = reinterpret_cast<float*>(sb + L.h);
  auto* hl = hh + (int64_t)d.nt * d.bq * d.r;
  auto* hmax = reinterpret_cast<unsigned int*>(sb + L.hmax);
  auto* bh = reinterpret_cast<__nv_bfloat16*>(sb + L.bh);
  auto* tau2 = reinterpret_cast<int*>(sb + L.tau2);
  auto* d2 = reinterpret_cast<float*>(sb + L.d2);
  const dim3 gs((unsigned)d.bq, (unsigned)((d.nk + 255) / 256)), gc((unsigned)((d.r + 63) / 64), (unsigned)d.batch);
  const int* spj = reinterpret_cast<const int*>(fb + F.sproj);
  if (d.sp == OZ_S7)
    k3o_slice_states<OZ_S7, OZ_BITS7><<<gs, 256, 0, s>>>(d, a, bst, tau, hmax);
  else
    k3o_slice_states<OZ_S, OZ_BITS><<<gs, 256, 0, s>>>(d, a, bst, tau, hmax);
  cudaError_t e = k3o_gemm_launch(fb + F.aproj, (int64_t)d.sp * d.mp, d.mp, bst, d.ncp, d.bq, d.nk, d.sp, d1, err,
                                  sm_count, s);
  if (e != cudaSuccess) return e;
  if (d.sp == OZ_S7)
    k3o_combine_proj<OZ_S7, OZ_BITS7><<<gc, 192, 0, s>>>(d, d1, spj, tau, hh, hl, hmax);
  else
    k3o_combine_proj<OZ_S, OZ_BITS><<<gc, 192, 0, s>>>(d, d1, spj, tau, hh, hl, hmax);
  k3o_slice_h<<<dim3((unsigned)d.bq, (unsigned)((d.rk + 255) / 256)), 256, 0, s>>>(d, a, hh, hl, hmax, bh, tau2);
  e = k3o_gemm_launch(fb + F.aexp, OZ_S * d.me, d.me, bh, d.nc, d.bq, d.rk, OZ_S, d2, err, sm_count, s);
  *d2_out = d2;
  *sexp_out = reinterpret_cast<const int*>(fb + F.sexp);
  *tau2_out = tau2;
  return e;
}

cudaError_t k3o_launch(int64_t n, int64_t rp, int64_t r, const K3Args& a, const void* factors, int batch,
                       void* scratch, int* err, int sm_count, cudaStream_t s) {
  const ODims d = oz_dims(n, rp, r, a.form, batch);
  const float* d2;
  const int *sexp, *tau2;
  cudaError_t e = k3o_front(d, a, factors, scratch, err, sm_count, s, &d2, &sexp, &tau2);
  if (e != cudaSuccess) return e;
  k3o_combine_exp<<<oz_flat_blocks((int64_t)batch * d.n, sm_count), 256, 0, s>>>(d, a, d2, sexp, tau2);
  return cudaGetLastError();
}

cudaError_t k3o_launch_step(int64_t n, int64_t rp, int64_t r, const K3Args& a, const void* factors, int batch,
                            void* scratch, int* err, int sm_count, const StepArgs& st, int step_index,
                            cudaStream_t s) {
  const ODims d = oz_dims(n, rp, r, a.form, batch);
  const float* d2;
  const int *sexp, *tau2;
  cudaError_t e = k3o_front(d, a, factors, scratch, err, sm_count, s, &d2, &sexp, &tau2);
  if (e != cudaSuccess) return e;
  // one element per thread: each carries a 45-pair combine before its step
  StepArgs st1 = st;
  st1.ept = 1;
  st1.nblk = step_mc_blocks(n);
  const dim3 grid((unsigned)st1.nblk, (unsigned)batch);
  if (step_plain(st1))
    k3o_exp_step<true><<<grid, STEP_MC_THREADS, 0, s>>>(d, d2, sexp, tau2, st1, step_index);
  else
    k3o_exp_step<false><<<grid, STEP_MC_THREADS, 0, s>>>(d, d2, sexp, tau2, st1, step_index);
  return cudaGetLastError();
}

}  // namespace grom
