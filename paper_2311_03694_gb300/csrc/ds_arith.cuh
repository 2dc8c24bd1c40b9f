// Double-single arithmetic on the FP32 pipe: a value is an unevaluated sum of
// two floats, hi = rn32(x) and lo = rn32(x - hi) (a 48-bit significand).
// GB300 issues about two FP64 FMAs per clock per SM against 128 FP32 ones,
// so FP64-tolerance contractions run in this arithmetic.  It is built from
// the error-free transformations of floating-point arithmetic: the FMA
// residual of a product (a*b - rn(a*b) is exact) and Knuth's TwoSum (the
// rounding error of a sum, exactly, in six operations), with Fast2Sum to
// renormalise a pair.  The intrinsics carry explicit rounding so that the
// compiler cannot contract or reassociate the transformations.
#pragma once

#include <cuda_runtime.h>

namespace grom {

// (S, s) += (ah + al)(bh + bl), al*bl (below 2^-48 relative) dropped.
// p = ah*bh; Knuth's TwoSum of S and p gives S1 and the exact terms
// S - (S1 - bb) and p - bb; the second and the product's rounding error
// (ah*bh - p) are folded into one residual fma(ah, bh, -bb).  The small
// terms and the cross terms ah*bl, al*bh are summed first and reach the low
// word in one addition, so each word of the accumulator carries a chain of
// one dependent operation per call.  10 FP32 operations.  The low word
// collects one rounding per call, so callers renormalise the pair
// (ds_renorm) every few terms to keep it within an ulp of the high word.
__device__ __forceinline__ void ds_mac(float ah, float al, float bh, float bl, float& S, float& s) {
  const float p = __fmul_rn(ah, bh);
  const float S1 = __fadd_rn(S, p);
  const float bb = __fsub_rn(S1, S);
  const float y = __fsub_rn(S, __fsub_rn(S1, bb));
  const float z = __fmaf_rn(ah, bh, -bb);
  float w = __fadd_rn(y, z);
  w = __fmaf_rn(al, bh, w);
  w = __fmaf_rn(ah, bl, w);
  s = __fadd_rn(s, w);
  S = S1;
}

// Fast2Sum: the pair as its rounded sum and that sum's error.
__device__ __forceinline__ void ds_renorm(float& S, float& s) {
  const float h = __fadd_rn(S, s);
  s = __fsub_rn(s, __fsub_rn(h, S));
  S = h;
}

// (S, s) += (T, t): TwoSum of the leading parts, then renormalised.
__device__ __forceinline__ void ds_add(float& S, float& s, float T, float t) {
  const float S1 = __fadd_rn(S, T);
  const float bb = __fsub_rn(S1, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(S1, bb)), __fsub_rn(T, bb));
  s = __fadd_rn(__fadd_rn(s, t), err);
  S = S1;
  ds_renorm(S, s);
}

// (h, l) = (ah + al)(bh + bl), renormalised.
__device__ __forceinline__ void ds_mul(float ah, float al, float bh, float bl, float& h, float& l) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  const float t = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
  h = __fadd_rn(p, t);
  l = __fsub_rn(t, __fsub_rn(h, p));
}

// An FP64 value as a double-single pair.
__device__ __forceinline__ void ds_split(double v, float& h, float& l) {
  h = __double2float_rn(v);
  l = __double2float_rn(v - (double)h);
}

}  // namespace grom
