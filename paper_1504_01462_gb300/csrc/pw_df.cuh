// Double-FP32 ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, a 48-bit significand on the
// FP32 pipe.  GB300 retires 128 FP32 FMAs but only 2 FP64 FMAs per clock and
// SM, so the mixed form's FP64-class steps (refinement residuals, overlaps)
// run in this format: about 12 FP32 operations per real multiply-add, 5x the
// native FP64 rate.
//
// The building blocks are the error-free transformations of Knuth (TwoSum)
// and of the fused multiply-add (TwoProd: a*b = p + fma(a, b, -p) exactly), as
// in Dekker's double-length arithmetic (Numer. Math. 18, 1971) and the
// double-double library of Hida, Li & Bailey (2001).  The exponent range is
// FP32's: values here are O(1) amplitudes, overlaps and wavenumbers.
#pragma once
#include "pw_cx.cuh"

struct __align__(8) df {
  float hi, lo;
};

__host__ __device__ __forceinline__ df mkdf(float hi, float lo) {
  df r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// nearest double-float of a double (exact to 48 bits)
__device__ __forceinline__ df df_of(double x) {
  const float h = __double2float_rn(x);
  return mkdf(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_val(df a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  e = b - (s - a);
}

__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  float h, l;
  fast_two_sum(s, e, h, l);
  return mkdf(h, l);
}
__device__ __forceinline__ df df_neg(df a) { return mkdf(-a.hi, -a.lo); }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return mkdf(h, l);
}
// acc += a * b, leaving acc unnormalised (lo collects the rounding terms);
// df_renorm restores |lo| <= ulp(hi)/2.  Between renormalisations lo grows
// by about one ulp(hi) per step, so callers renormalise every few dozen steps.
__device__ __forceinline__ void df_fma_lazy(df &acc, df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo += e + t;
}
__device__ __forceinline__ void df_renorm(df &a) {
  float h, l;
  fast_two_sum(a.hi, a.lo, h, l);
  a.hi = h;
  a.lo = l;
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_from_float(float x) { return mkdf(x, 0.f); }
// a * b for a float b (exact product of the high parts plus the low term)
__device__ __forceinline__ df df_mul_f(df a, float b) {
  const float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return mkdf(h, l);
}
// a / b by one correction of the FP32 quotient (Dekker's division):
// q1 = a_hi / b_hi, r = a - q1 b (formed exactly enough in double-float),
// q = q1 + r_hi / b_hi
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = a.hi / b.hi;
  const df r = df_sub(a, df_mul_f(b, q1));
  const float q2 = r.hi / b.hi;
  float h, l;
  fast_two_sum(q1, q2, h, l);
  return mkdf(h, l);
}
// sqrt(a), a >= 0, by one Newton correction of the FP32 root:
// x = sqrt(a_hi), x + (a - x^2) / (2 x) with x^2 formed exactly (TwoProd)
__device__ __forceinline__ df df_sqrt(df a) {
  if (!(a.hi > 0.f)) return mkdf(0.f, 0.f);
  const float x = sqrtf(a.hi);
  const float p = x * x, pe = fmaf(x, x, -p);
  const float r = ((a.hi - p) - pe) + a.lo;
  float h, l;
  fast_two_sum(x, r / (2.f * x), h, l);
  return mkdf(h, l);
}
__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.f ? df_neg(a) : a; }

// complex double-float
typedef cx<df> dfc;

template <>
__host__ __device__ __forceinline__ dfc czero<df>() {
  dfc z;
  z.re = mkdf(0.f, 0.f);
  z.im = mkdf(0.f, 0.f);
  return z;
}
__device__ __forceinline__ dfc dfc_of(zc a) {
  dfc z;
  z.re = df_of(a.re);
  z.im = df_of(a.im);
  return z;
}
__device__ __forceinline__ zc dfc_val(dfc a) { return mkc<double>(df_val(a.re), df_val(a.im)); }

// acc += a * b (complex), unnormalised; the CTA GEMM renormalises after each
// k-tile through cacc_renorm.
__device__ __forceinline__ void cfma(dfc &acc, dfc a, dfc b) {
  df_fma_lazy(acc.re, a.re, b.re);
  df_fma_lazy(acc.re, df_neg(a.im), b.im);
  df_fma_lazy(acc.im, a.re, b.im);
  df_fma_lazy(acc.im, a.im, b.re);
}
__device__ __forceinline__ void cacc_renorm(dfc &a) {
  df_renorm(a.re);
  df_renorm(a.im);
}

// Operand conversion for kernels templated on the accumulation type
// (double: native FP64; df: double-float on the FP32 pipe).
template <typename A>
__device__ __forceinline__ cx<A> acc_of(zc v);
template <>
__device__ __forceinline__ zc acc_of<double>(zc v) { return v; }
template <>
__device__ __forceinline__ dfc acc_of<df>(zc v) { return dfc_of(v); }
__device__ __forceinline__ zc acc_val(zc v) { return v; }
__device__ __forceinline__ zc acc_val(dfc v) { return dfc_val(v); }
