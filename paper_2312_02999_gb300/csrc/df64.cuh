// Double-float arithmetic (an unevaluated sum hi + lo of two float32 values,
// about 48 significant bits) for the mixed-precision local step.  On GB300 a
// float64 FMA costs about as much issue time as 60 float32 operations, while
// a double-float multiply-add is about 25, so the float64-accurate parts of
// the per-tet local step run several times faster in this form.
//
// The building blocks are the classical error-free transformations: Knuth's
// two-sum (the rounding error of a + b), Dekker's fast two-sum for
// |a| >= |b|, and the FMA two-product (the rounding error of a * b is
// fma(a, b, -a*b) exactly).  The additions and products use the _rn
// intrinsics, which the compiler never fuses into FMAs or reorders, so the
// transformations stay error-free whatever the contraction flags.
#pragma once
#include <cuda_runtime.h>

namespace fsim {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df df_from_double(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(__dsub_rn(v, (double)h))};
}

__device__ __forceinline__ df df_from_float(float v) { return {v, 0.f}; }

__device__ __forceinline__ double df_to_double(df a) { return __dadd_rn((double)a.hi, (double)a.lo); }

// a + b with both parts' errors carried (exact-cancellation safe)
__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  const df t = df_two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return df_fast_two_sum(s.hi, s.lo);
}

// a + b by Dekker's addition: one two-sum of the high parts, the low parts
// added in float32.  About half the operations of df_add; the result is
// within a few units of 2^-44 (|a| + |b|), so it is used where a and b do
// not nearly cancel (sums of products of one sign, small corrections), and
// df_add where they may.
__device__ __forceinline__ df df_add_fast(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, s.lo);
}

// a0 b0 + a1 b1 + a2 b2, normalised once.  The products of the high parts
// and their sum are formed with error-free transformations (FMA two-product,
// two-sum).  The low-order terms are added in float32: the products'
// rounding errors, the cross terms hi * lo and lo * hi, and the sums'
// rounding errors.  It is in the accuracy class of three df_mul and two
// df_add_fast (a few units of 2^-44 of sum |a_i b_i|, for sums that do not
// nearly cancel) with about a third fewer operations.
__device__ __forceinline__ df df_dot3(df a0, df b0, df a1, df b1, df a2, df b2) {
  const float p0 = __fmul_rn(a0.hi, b0.hi), p1 = __fmul_rn(a1.hi, b1.hi), p2 = __fmul_rn(a2.hi, b2.hi);
  float e = __fmaf_rn(a0.hi, b0.hi, -p0);
  e = __fadd_rn(e, __fmaf_rn(a1.hi, b1.hi, -p1));
  e = __fadd_rn(e, __fmaf_rn(a2.hi, b2.hi, -p2));
  e = __fmaf_rn(a0.hi, b0.lo, e);
  e = __fmaf_rn(a0.lo, b0.hi, e);
  e = __fmaf_rn(a1.hi, b1.lo, e);
  e = __fmaf_rn(a1.lo, b1.hi, e);
  e = __fmaf_rn(a2.hi, b2.lo, e);
  e = __fmaf_rn(a2.lo, b2.hi, e);
  const df s = df_two_sum(p0, p1);
  const df s2 = df_two_sum(s.hi, p2);
  e = __fadd_rn(e, __fadd_rn(s.lo, s2.lo));
  return df_fast_two_sum(s2.hi, e);
}

// the same with float32 second factors
__device__ __forceinline__ df df_dot3_f(df a0, float b0, df a1, float b1, df a2, float b2) {
  const float p0 = __fmul_rn(a0.hi, b0), p1 = __fmul_rn(a1.hi, b1), p2 = __fmul_rn(a2.hi, b2);
  float e = __fmaf_rn(a0.hi, b0, -p0);
  e = __fadd_rn(e, __fmaf_rn(a1.hi, b1, -p1));
  e = __fadd_rn(e, __fmaf_rn(a2.hi, b2, -p2));
  e = __fmaf_rn(a0.lo, b0, e);
  e = __fmaf_rn(a1.lo, b1, e);
  e = __fmaf_rn(a2.lo, b2, e);
  const df s = df_two_sum(p0, p1);
  const df s2 = df_two_sum(s.hi, p2);
  e = __fadd_rn(e, __fadd_rn(s.lo, s2.lo));
  return df_fast_two_sum(s2.hi, e);
}

// a + b + c for double-float terms: the high parts summed with two-sums,
// the low parts and the sums' rounding errors in float32, normalised once
// (exact-cancellation safe in the high parts)
__device__ __forceinline__ df df_sum3(df a, df b, df c) {
  const df s = df_two_sum(a.hi, b.hi);
  const df s2 = df_two_sum(s.hi, c.hi);
  const float e = __fadd_rn(__fadd_rn(__fadd_rn(a.lo, b.lo), c.lo), __fadd_rn(s.lo, s2.lo));
  return df_two_sum(s2.hi, e);
}

// a0 b0 + a1 b1 + a2 b2 for float32 factors, as a double-float (the exact
// products' high and low parts summed as in df_dot3)
__device__ __forceinline__ df df_dot3_ff(float a0, float b0, float a1, float b1, float a2, float b2) {
  const float p0 = __fmul_rn(a0, b0), p1 = __fmul_rn(a1, b1), p2 = __fmul_rn(a2, b2);
  float e = __fmaf_rn(a0, b0, -p0);
  e = __fadd_rn(e, __fmaf_rn(a1, b1, -p1));
  e = __fadd_rn(e, __fmaf_rn(a2, b2, -p2));
  const df s = df_two_sum(p0, p1);
  const df s2 = df_two_sum(s.hi, p2);
  e = __fadd_rn(e, __fadd_rn(s.lo, s2.lo));
  return df_two_sum(s2.hi, e);
}

// a - b with the high parts' difference exact (two-sum) and the low parts'
// difference rounded once in float32: an absolute error within a few units
// of 2^-48 (|a| + |b|), also when a and b nearly cancel
__device__ __forceinline__ df df_sub_fast(df a, df b) {
  const df s = df_two_sum(a.hi, -b.hi);
  return df_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = df_two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return df_fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = df_two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return df_fast_two_sum(p.hi, p.lo);
}

// a * b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

}  // namespace fsim
