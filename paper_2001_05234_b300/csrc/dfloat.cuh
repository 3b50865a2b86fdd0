// Double-float arithmetic: a value is hi + lo with two floats (about 48 significant bits).
//
// On B300 an FP64 instruction issues at roughly 1/64 of the FP32 rate, so the mixed-precision
// refinement keeps its extended-precision residual and iterate in pairs of floats built from
// error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum and the FMA-based TwoProduct
// (see e.g. Muller et al., Handbook of Floating-Point Arithmetic).  These routines rely on IEEE
// round-to-nearest float arithmetic without reassociation, so the library is never built with
// fast-math.
#pragma once
#include <cuda_runtime.h>

namespace cans {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) {
  df r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// s + e == a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}

// s + e == a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return df_make(s, e);
}

// p + e == a * b exactly (FMA)
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return df_make(p, e);
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, lo);
}

__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  const float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, lo);
}

// split a double into hi + lo floats (hi = nearest float, lo = nearest float of the remainder)
__device__ __forceinline__ df df_from_double(double x) {
  const float hi = __double2float_rn(x);
  const float lo = __double2float_rn(x - (double)hi);
  return df_make(hi, lo);
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace cans
