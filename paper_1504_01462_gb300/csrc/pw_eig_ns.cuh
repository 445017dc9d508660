// Complex non-Hermitian eigenproblems for one team of threads (one CTA on the
// GPU): Householder reduction to upper Hessenberg form, the implicitly shifted
// QR iteration to complex Schur form A = Z T Z^H, and reordering of the Schur
// form by swaps of neighbouring diagonal entries.  These are the textbook
// algorithms (Householder reflections; the single-shift QR iteration of
// Francis and Kublanovskaya with Wilkinson shifts and bulge chasing by
// Givens rotations; swapping of 1 x 1 Schur blocks by one rotation that zeros
// the (2,1) entry of the exchanged block), written for column-major FP64
// complex matrices in global memory.  Every function is called by all threads
// of the team and ends with the team synchronised.
#pragma once
#include <math.h>

#include "pw_cx.cuh"

namespace pw {
namespace ns {

// A team: thread `id` of `size`; `red` holds size + 8 doubles that every
// thread of the team can read and write (shared memory on the GPU).
struct Team {
  int id, size;
  double *red;
  __device__ void sync() const { __syncthreads(); }
  // the sum over the team of one value per thread, returned to every thread
  __device__ double sum(double v) const {
    red[id] = v;
    sync();
    if (id == 0) {
      double s = 0.0;
      for (int i = 0; i < size; ++i) s += red[i];
      red[size] = s;
    }
    sync();
    const double s = red[size];
    sync();
    return s;
  }
};

__device__ __forceinline__ double cabs_(zc a) { return hypot(a.re, a.im); }

// A rotation [[c, s], [-conj(s), c]] (c real) with
// [[c, s], [-conj(s), c]] [f; g] = [r; 0].
struct Rot {
  double c;
  zc s;
};
__device__ inline Rot make_rot(zc f, zc g) {
  const double fa = cabs_(f), ga = cabs_(g);
  Rot q;
  if (ga == 0.0) {
    q.c = 1.0;
    q.s = czero<double>();
  } else if (fa == 0.0) {
    q.c = 0.0;
    q.s = mkc<double>(g.re / ga, -g.im / ga);
  } else {
    const double nrm = hypot(fa, ga);
    q.c = fa / nrm;
    const zc ph = mkc<double>(f.re / fa, f.im / fa);   // f / |f|
    q.s = cmul(ph, mkc<double>(g.re / nrm, -g.im / nrm));
  }
  return q;
}

// rows i, i+1 of A (columns c0 .. c1-1) <- G [row i; row i+1]
__device__ inline void rot_rows(const Team &t, zc *A, int ld, int i, int c0, int c1, Rot q) {
  for (int j = c0 + t.id; j < c1; j += t.size) {
    zc &x = A[i + (size_t)j * ld], &y = A[i + 1 + (size_t)j * ld];
    const zc a = x, b = y;
    x = cadd(cscale(q.c, a), cmul(q.s, b));
    y = csub(cscale(q.c, b), cmul(cconj(q.s), a));
  }
}
// columns i, i+1 of A (rows r0 .. r1-1) <- [col i, col i+1] G^H
__device__ inline void rot_cols(const Team &t, zc *A, int ld, int i, int r0, int r1, Rot q) {
  zc *x = A + (size_t)i * ld, *y = A + (size_t)(i + 1) * ld;
  for (int r = r0 + t.id; r < r1; r += t.size) {
    const zc a = x[r], b = y[r];
    x[r] = cadd(cscale(q.c, a), cmul(cconj(q.s), b));
    y[r] = csub(cscale(q.c, b), cmul(q.s, a));
  }
}

// Householder reduction of A (N x N) to upper Hessenberg form H = Q^H A Q,
// with Z <- Z Q.  v: N scratch values visible to the team.
__device__ inline void hessenberg(const Team &t, zc *A, zc *Z, int N, zc *v) {
  for (int k = 0; k + 2 < N; ++k) {
    double nx = 0.0;
    for (int i = k + 1 + t.id; i < N; i += t.size) nx += cnorm2(A[i + (size_t)k * N]);
    nx = t.sum(nx);
    const zc x0 = A[k + 1 + (size_t)k * N];
    const double a0 = cabs_(x0);
    if (nx - a0 * a0 <= 1e-300) continue;   // the column is already reduced
    const double nr = sqrt(nx);
    const zc beta = a0 > 0.0 ? mkc<double>(-x0.re / a0 * nr, -x0.im / a0 * nr) : mkc<double>(-nr, 0.0);
    for (int i = k + 1 + t.id; i < N; i += t.size) v[i] = A[i + (size_t)k * N];
    t.sync();
    if (t.id == 0) v[k + 1] = csub(x0, beta);
    t.sync();
    const double vv = nx - a0 * a0 + cnorm2(v[k + 1]);
    const double tau = 2.0 / vv;
    // left: rows k+1.. of columns k.. (each thread one column)
    for (int j = k + t.id; j < N; j += t.size) {
      zc w = czero<double>();
      for (int i = k + 1; i < N; ++i) cfma(w, cconj(v[i]), A[i + (size_t)j * N]);
      w = cscale(tau, w);
      for (int i = k + 1; i < N; ++i) A[i + (size_t)j * N] = csub(A[i + (size_t)j * N], cmul(v[i], w));
    }
    t.sync();
    // right: columns k+1.. of every row of A and Z (each thread one row)
    for (int r = t.id; r < 2 * N; r += t.size) {
      zc *M = r < N ? A : Z;
      const int i = r < N ? r : r - N;
      zc w = czero<double>();
      for (int j = k + 1; j < N; ++j) cfma(w, M[i + (size_t)j * N], v[j]);
      w = cscale(tau, w);
      for (int j = k + 1; j < N; ++j) M[i + (size_t)j * N] = csub(M[i + (size_t)j * N], cmul(w, cconj(v[j])));
    }
    t.sync();
    for (int i = k + 2 + t.id; i < N; i += t.size) A[i + (size_t)k * N] = czero<double>();
    t.sync();
  }
}

// Complex Schur form of the upper Hessenberg H (N x N) by the implicitly
// shifted QR iteration: H <- Z0^H H Z0 upper triangular, Z <- Z Z0.  Returns
// false if an eigenvalue did not converge within 30 iterations.  rs: 4
// doubles visible to the team (the current rotation).
__device__ inline bool schur(const Team &t, zc *H, zc *Z, int N, double *rs) {
  const double eps = 2.220446049250313e-16;
  int hi = N - 1, iter = 0;
  while (hi > 0) {
    // deflation: the largest lo <= hi with H(lo, lo-1) negligible
    int lo = hi;
    while (lo > 0) {
      const zc sub = H[lo + (size_t)(lo - 1) * N];
      const double d = cabs1(H[lo + (size_t)lo * N]) + cabs1(H[lo - 1 + (size_t)(lo - 1) * N]);
      if (cabs1(sub) <= eps * d) break;
      --lo;
    }
    if (lo > 0) {
      t.sync();
      if (t.id == 0) H[lo + (size_t)(lo - 1) * N] = czero<double>();
      t.sync();
    }
    if (lo == hi) {
      --hi;
      iter = 0;
      continue;
    }
    if (++iter > 30) return false;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 nearer H(hi, hi);
    // exceptional shifts after 10 and 20 iterations without deflation
    const zc a = H[hi - 1 + (size_t)(hi - 1) * N], b = H[hi - 1 + (size_t)hi * N];
    const zc c = H[hi + (size_t)(hi - 1) * N], d = H[hi + (size_t)hi * N];
    zc mu;
    if (iter == 10 || iter == 20) {
      mu = cadd(d, mkc<double>(0.75 * cabs1(c), 0.0));
    } else {
      const zc h = mkc<double>(0.5 * (a.re - d.re), 0.5 * (a.im - d.im));
      const zc z = cadd(cmul(h, h), cmul(b, c));
      // principal square root of z
      const double s = sqrt(0.5 * (cabs_(z) + fabs(z.re)));
      zc disc = czero<double>();
      if (s > 0.0)
        disc = z.re >= 0.0 ? mkc<double>(s, z.im / (2.0 * s))
                           : mkc<double>(fabs(z.im) / (2.0 * s), z.im >= 0.0 ? s : -s);
      const zc m = mkc<double>(0.5 * (a.re + d.re), 0.5 * (a.im + d.im));
      const zc e1 = cadd(m, disc), e2 = csub(m, disc);
      mu = cabs1(csub(e1, d)) <= cabs1(csub(e2, d)) ? e1 : e2;
    }
    // the QR sweep over [lo, hi], chasing the bulge
    for (int k = lo; k < hi; ++k) {
      if (t.id == 0) {
        zc f, g;
        if (k == lo) {
          f = csub(H[lo + (size_t)lo * N], mu);
          g = H[lo + 1 + (size_t)lo * N];
        } else {
          f = H[k + (size_t)(k - 1) * N];
          g = H[k + 1 + (size_t)(k - 1) * N];
        }
        const Rot q = make_rot(f, g);
        rs[0] = q.c;
        rs[1] = q.s.re;
        rs[2] = q.s.im;
      }
      t.sync();
      Rot q;
      q.c = rs[0];
      q.s = mkc<double>(rs[1], rs[2]);
      rot_rows(t, H, N, k, k > lo ? k - 1 : lo, N, q);
      t.sync();
      rot_cols(t, H, N, k, 0, min(k + 2, hi) + 1, q);
      rot_cols(t, Z, N, k, 0, N, q);
      t.sync();
      if (k > lo && t.id == 0) H[k + 1 + (size_t)(k - 1) * N] = czero<double>();
      t.sync();
    }
  }
  return true;
}

// Exchanges the diagonal entries i and i+1 of the upper triangular T (N x N),
// T <- G T G^H, Z <- Z G^H.
__device__ inline void schur_swap(const Team &t, zc *T, zc *Z, int N, int i, double *rs) {
  if (t.id == 0) {
    const zc a = T[i + (size_t)i * N], b = T[i + 1 + (size_t)(i + 1) * N];
    const Rot q = make_rot(T[i + (size_t)(i + 1) * N], csub(b, a));
    rs[0] = q.c;
    rs[1] = q.s.re;
    rs[2] = q.s.im;
  }
  t.sync();
  Rot q;
  q.c = rs[0];
  q.s = mkc<double>(rs[1], rs[2]);
  const zc a = T[i + (size_t)i * N], b = T[i + 1 + (size_t)(i + 1) * N];
  t.sync();
  rot_rows(t, T, N, i, i, N, q);
  t.sync();
  rot_cols(t, T, N, i, 0, i + 2, q);
  rot_cols(t, Z, N, i, 0, N, q);
  t.sync();
  if (t.id == 0) {
    T[i + (size_t)i * N] = b;
    T[i + 1 + (size_t)(i + 1) * N] = a;
    T[i + 1 + (size_t)i * N] = czero<double>();
  }
  t.sync();
}

// Reorders the Schur form so that the diagonal entries with key 0 come first
// (a stable bubble of adjacent swaps); key(i) reads the entry's class from
// keys[i], which moves with its entry.  Returns the number with key 0.
__device__ inline int schur_select(const Team &t, zc *T, zc *Z, int N, int *keys, double *rs) {
  int cnt = 0;
  for (int i = 0; i < N; ++i) cnt += keys[i] == 0;
  int pos = 0;
  for (int i = 0; i < N; ++i) {
    if (keys[i] != 0) continue;
    for (int j = i; j > pos; --j) {
      schur_swap(t, T, Z, N, j - 1, rs);
      if (t.id == 0) {
        const int k = keys[j - 1];
        keys[j - 1] = keys[j];
        keys[j] = k;
      }
      t.sync();
    }
    ++pos;
  }
  return cnt;
}

}  // namespace ns
}  // namespace pw
