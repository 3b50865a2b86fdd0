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

// ---- conversions between binary64 and binary32 in integer arithmetic --------------------------
// On B300 the double<->float conversion instructions share the slow FP64-class pipe (measured at
// about 0.6-0.7 T conversions/s per GPU, the rate of an FP64 add), so the per-point conversions of
// the mixed path are done on the bit patterns instead.  binary64: sign | 11-bit biased exponent e
// (bias 1023) | 52-bit fraction; binary32: sign | 8-bit biased exponent (bias 127) | 23-bit fraction.
// A binary64 with 897 <= e <= 1150 rounds to a normal binary32 (or overflows to infinity) whose
// exponent field is e - 896; other inputs (zeros, subnormals, tiny or huge values, inf, NaN) take
// the hardware conversion, whose results these match bit for bit.

// Hardware conversions of the rare inputs outside the integer paths' range, kept out of line so
// that the compiler branches around them instead of executing them (on the slow pipe) for every
// element and selecting (measured: the update x-inverse; not d2f_rn, see there).
static __device__ __noinline__ double f2d_hw(float x) { return (double)x; }
static __device__ __noinline__ df df_split_hw(double x) {
  const float h = __double2float_rn(x);
  return df_make(h, __double2float_rn(x - (double)h));
}

// nearest float, ties to even (= __double2float_rn)
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 254u) {
    const unsigned t = __funnelshift_l(lo, hi, 3);  // exponent and top 23 fraction bits, shifted into place
    unsigned bits = (t - (896u << 23)) | (hi & 0x80000000u);
    // round half to even on the 29 dropped fraction bits; a carry propagates into the exponent
    bits += ((lo & 0x1fffffffu) + (t & 1u) + 0x0fffffffu) >> 29;
    return __uint_as_float(bits);
  }
  return __double2float_rn(x);  // inline: an out-of-line call here costs the x forward pass registers
}

// d2f_rn on the integer path only: *ok is false (and the result meaningless) outside its range, so
// that a caller can take the hardware conversion in a branch of its own (see SrcF in kern_xw.cu)
__device__ __forceinline__ float d2f_rn_int(double x, bool* ok) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  *ok = e - 897u < 254u;
  const unsigned t = __funnelshift_l(lo, hi, 3);
  unsigned bits = (t - (896u << 23)) | (hi & 0x80000000u);
  bits += ((lo & 0x1fffffffu) + (t & 1u) + 0x0fffffffu) >> 29;
  return __uint_as_float(bits);
}

// x = hi + lo with hi = d2f_rn(x) and lo the remainder to within 2^-46 |x| (exact for |x| >= 2^-80
// up to the 6 lowest of its 29 remainder bits).  Outside 2^-80 <= |x| < 2^127 the FP64 route is used.
__device__ __forceinline__ df df_split(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 943u < 207u) {
    const unsigned t = __funnelshift_l(lo, hi, 3);
    const unsigned sgn = hi & 0x80000000u;
    const unsigned up = ((lo & 0x1fffffffu) + (t & 1u) + 0x0fffffffu) >> 29;
    const float h = __uint_as_float(((t - (896u << 23)) | sgn) + up);
    // remainder in units of 2^(e-1075): the dropped bits, minus 2^29 when hi was rounded up;
    // |r| <= 2^28, so r / 64 fits the exact float-from-integer trick 1.5*2^23 + r/64 - 1.5*2^23
    const int r = (int)(lo & 0x1fffffffu) - (int)(up << 29);
    const float rf = __int_as_float(0x4b400000 + (r >> 6)) - 12582912.0f;
    const float scale = __uint_as_float(sgn | ((e - 942u) << 23));  // +-2^(e-1069)
    return df_make(h, rf * scale);
  }
  if (((hi << 1) | lo) == 0u) return df_make(__uint_as_float(hi & 0x80000000u), 0.f);
  return df_split_hw(x);
}

// x = hi + lo with hi = x truncated to a float (towards zero) and lo the remainder to within
// 2^-46 |x|: the cheaper split for operands that only enter a sum (|lo| < ulp(hi) instead of
// ulp(hi)/2).  Same range and fallback as df_split.
__device__ __forceinline__ df df_split_rz(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 943u < 207u) {
    const unsigned sgn = hi & 0x80000000u;
    const float h = __uint_as_float((__funnelshift_l(lo, hi, 3) - (896u << 23)) | sgn);
    // the 29 dropped fraction bits, top 23 of them as an exact float, scaled by +-2^(e-1069)
    const float rf = __uint_as_float(0x4b000000u | ((lo & 0x1fffffffu) >> 6)) - 8388608.0f;
    return df_make(h, rf * __uint_as_float(sgn | ((e - 942u) << 23)));
  }
  return df_split(x);
}

// exact float -> double
__device__ __forceinline__ double f2d(float x) {
  const unsigned b = __float_as_uint(x);
  if (((b >> 23) & 0xffu) - 1u < 254u)  // normal: rebias the exponent (+896), widen the fraction
    return __hiloint2double((int)((b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (896u << 20))), (int)(b << 29));
  if ((b << 1) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return f2d_hw(x);
}

// value conversion between the storage and compute precisions of a kernel
template <typename To, typename From> struct Cvt { static __device__ __forceinline__ To run(From x) { return (To)x; } };
template <> struct Cvt<float, double> { static __device__ __forceinline__ float run(double x) { return d2f_rn(x); } };
template <> struct Cvt<double, float> { static __device__ __forceinline__ double run(float x) { return f2d(x); } };
template <typename To, typename From> __device__ __forceinline__ To cvt(From x) { return Cvt<To, From>::run(x); }

// split a double into hi + lo floats (hi = nearest float, lo = the remainder, see df_split)
__device__ __forceinline__ df df_from_double(double x) { return df_split(x); }

// hi + lo as a double: exact widening of both parts and one FP64 add
__device__ __forceinline__ double df_to_double(df a) { return f2d(a.hi) + f2d(a.lo); }

}  // namespace cans
