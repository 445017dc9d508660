// Complex arithmetic for the device code (FP64 and FP32 variants).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

template <typename T>
struct __align__(2 * sizeof(T)) cx {
  T re, im;
};

typedef cx<double> zc;
typedef cx<float> cc;

template <typename T>
__host__ __device__ __forceinline__ cx<T> mkc(T r, T i) {
  cx<T> z;
  z.re = r;
  z.im = i;
  return z;
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> czero() { return mkc<T>(T(0), T(0)); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mkc<T>(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mkc<T>(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mkc<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ cx<T> cjmul(cx<T> a, cx<T> b) {
  return mkc<T>(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> cconj(cx<T> a) { return mkc<T>(a.re, -a.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> cscale(T s, cx<T> a) { return mkc<T>(s * a.re, s * a.im); }
template <typename T>
__host__ __device__ __forceinline__ T cabs1(cx<T> a) { return fabs(a.re) + fabs(a.im); }
template <typename T>
__host__ __device__ __forceinline__ T cnorm2(cx<T> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b with four fused multiply-adds
template <typename T>
__device__ __forceinline__ void cfma(cx<T> &acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// 1 / a, scaled to avoid overflow of |a|^2 (Smith's method)
template <typename T>
__device__ __forceinline__ cx<T> cinv(cx<T> a) {
  if (fabs(a.re) >= fabs(a.im)) {
    T r = a.im / a.re;
    T d = a.re + a.im * r;
    return mkc<T>(T(1) / d, -r / d);
  } else {
    T r = a.re / a.im;
    T d = a.re * r + a.im;
    return mkc<T>(r / d, T(-1) / d);
  }
}
template <typename T>
__device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b) { return cmul(a, cinv(b)); }

template <typename T, typename S>
__host__ __device__ __forceinline__ cx<T> ccast(cx<S> a) { return mkc<T>(T(a.re), T(a.im)); }

// k = sqrt(E - En): positive real above threshold, i*sqrt(En - E) below.
__device__ __forceinline__ zc kz_branch(double E, double En) {
  double d = E - En;
  return d > 0.0 ? mkc<double>(sqrt(d), 0.0) : mkc<double>(0.0, sqrt(-d));
}
// e^{i k dz} for k on the branch above (|.| <= 1)
__device__ __forceinline__ zc phase_fwd(zc k, double dz) {
  double mag = exp(-k.im * dz);
  double s, c;
  sincos(k.re * dz, &s, &c);
  return mkc<double>(mag * c, mag * s);
}
