// Slice potentials, slice Hamiltonians, their eigenmodes and the interface
// overlaps: everything of the path that depends on k_par but not on E.
//
//   k_tables      V^p(dG) of Gaussian wells averaged over each slice (Sec. II A:
//                 the slice potential is taken z-independent inside a slice)
//   k_assemble_h  H_p(G,G') = |k+G|^2 delta + V^p(G-G')          (Eq. loc)
//   k_heev        eigenpairs (E_n^p, phi_n^p) of every H_p       (Eq. loc / A8):
//                 Householder tridiagonalisation, implicit QL, back-
//                 transformation; the mixed form runs the same steps in
//                 double-float as five launches (k_heev<df> reduction,
//                 k_ql_df, k_rot_apply, k_backtransform, k_eig_sort)
//   k_jacobi      a second, independent solver (cyclic two-sided Jacobi)
//   k_overlaps    O_p = U_p^H U_{p+1} = sum_s (M^{p+1}_{js})^* M^p_{ns}
//                 of App. A Eq. transfer
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <type_traits>

#include "pw_cta.cuh"
#include "pw_df.cuh"
#include "pw_internal.h"

namespace pw {

// ---------------------------------------------------------------------------
// Fourier tables.  One thread per (slice, dG).  For a well -v0 exp(-|r-R|^2/2s^2)
// the transverse-periodic Fourier coefficient is
//   -(2 pi s^2 / A) v0 exp(-s^2 |G|^2 / 2) exp(-i G.R_perp) x (z-weight),
// the z-weight being the slice average of exp(-(z-Z)^2/2s^2):
//   (s sqrt(pi/2) / dz) [erf((z_hi-Z)/(sqrt2 s)) - erf((z_lo-Z)/(sqrt2 s))]
// for a slice, and s sqrt(2 pi) / period for a z-periodic electrode.
// ---------------------------------------------------------------------------
__global__ void k_tables(TableArgs a) {
  const int tsz = (2 * a.Dm + 1) * (2 * a.Dn + 1);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (e >= tsz) return;
  const bool is_lead = (q == 0 || q == a.nq - 1);
  const int side = (q == 0) ? 0 : 1;
  if (is_lead ? a.explicit_lead[side] : a.explicit_slices) return;
  const int dm = e / (2 * a.Dn + 1) - a.Dm;
  const int dn = e % (2 * a.Dn + 1) - a.Dn;
  const double gx = dm * a.b1x + dn * a.b2x;
  const double gy = dm * a.b1y + dn * a.b2y;
  const double g2 = gx * gx + gy * gy;
  const double pref = -2.0 * M_PI / a.area;
  double re = 0.0, im = 0.0;
  if (is_lead) {
    const WellSet &w = a.lead[side];
    for (int i = 0; i < w.n; ++i) {
      const double s = w.sigma[i];
      const double amp = pref * s * s * w.v0[i] * exp(-0.5 * s * s * g2) *
                         (s * sqrt(2.0 * M_PI) / a.period[side]);
      double sn, cs;
      sincos(gx * w.xyz[2 * i] + gy * w.xyz[2 * i + 1], &sn, &cs);
      re += amp * cs;
      im -= amp * sn;
    }
  } else {
    const double zlo = a.z_edges[q - 1], zhi = a.z_edges[q];
    const WellSet &w = a.slices;
    for (int i = 0; i < w.n; ++i) {
      const double s = w.sigma[i];
      const double Z = w.xyz[3 * i + 2];
      const double wz = (s * sqrt(0.5 * M_PI) / (zhi - zlo)) *
                        (erf((zhi - Z) / (M_SQRT2 * s)) - erf((zlo - Z) / (M_SQRT2 * s)));
      const double amp = pref * s * s * w.v0[i] * exp(-0.5 * s * s * g2) * wz;
      double sn, cs;
      sincos(gx * w.xyz[3 * i] + gy * w.xyz[3 * i + 1], &sn, &cs);
      re += amp * cs;
      im -= amp * sn;
    }
  }
  a.tab[(size_t)q * tsz + e] = mkc<double>(re, im);
}

void launch_tables(const TableArgs &a, cudaStream_t s) {
  const int tsz = (2 * a.Dm + 1) * (2 * a.Dn + 1);
  dim3 grid((tsz + 255) / 256, a.nq);
  PW_TIMED(KK_TABLES, s, k_tables<<<grid, 256, 0, s>>>(a));
}

// ---------------------------------------------------------------------------
// Hamiltonians, column-major, one thread per element.
// ---------------------------------------------------------------------------
__global__ void k_assemble_h(zc *H, const zc *tab, const int *mn, const double *G, double kx,
                             double ky, int n, int Dm, int Dn) {
  const int q = blockIdx.y;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * n) return;
  const int i = e % n, j = e / n;
  const int tw = 2 * Dn + 1;
  const int dm = mn[2 * i] - mn[2 * j] + Dm;
  const int dn = mn[2 * i + 1] - mn[2 * j + 1] + Dn;
  zc v = tab[(size_t)q * (2 * Dm + 1) * tw + dm * tw + dn];
  if (i == j) {
    const double x = kx + G[2 * i], y = ky + G[2 * i + 1];
    v.re += x * x + y * y;
    v.im = 0.0;
  }
  H[(size_t)q * n * n + e] = v;
}

void launch_assemble_h(zc *H, const zc *tab, const int *mn, const double *G, double kx, double ky,
                       int n, int nq, int Dm, int Dn, cudaStream_t s) {
  dim3 grid((unsigned)(((size_t)n * n + 255) / 256), nq);
  PW_TIMED(KK_ASSEMBLE, s, k_assemble_h<<<grid, 256, 0, s>>>(H, tab, mn, G, kx, ky, n, Dm, Dn));
}

// ---------------------------------------------------------------------------
// Batched Hermitian eigensolver: cyclic two-sided Jacobi with a parallel
// (round-robin) ordering, one CTA per matrix, matrix in global memory.
//
// For a pair (p, q) with a_pq = |b| e^{i phi}, the unitary
//   J = [[c, s], [-s e^{-i phi}, c e^{-i phi}]],
//   theta = (a_qq - a_pp) / (2|b|), t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)),
//   c = 1 / sqrt(t^2 + 1), s = t c,
// makes (J^H A J)_pq = 0 with new diagonal a_pp - t|b|, a_qq + t|b|.  Each round
// applies n/2 disjoint rotations: columns of A and V first (A J, V J), then
// rows of A (J^H (A J)).  Sweeps continue until the largest |a_pq| met in a
// sweep is below conv_rel * max|A| (1e-12 in FP64; convergence is quadratic,
// so the last sweep leaves off-diagonals at rounding level).  Each round
// streams A and V through L2/HBM, so the kernel is bandwidth-bound.
// ---------------------------------------------------------------------------
constexpr int EIG_THREADS = 512;

__device__ __forceinline__ void atomic_max_pos(unsigned long long *addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__global__ void __launch_bounds__(EIG_THREADS)
    k_jacobi(cx<T> *A_all, cx<T> *V_all, size_t stride, int n, int init_identity, int max_sweeps,
             double conv_rel, int *sweeps_out, double *En_all, zc *U_all) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int mat = blockIdx.x;
  cx<T> *A = A_all + (size_t)mat * stride;
  cx<T> *V = V_all + (size_t)mat * stride;
  const int m = (n + 1) & ~1;
  const int np = m / 2;
  const int tid = threadIdx.x;
  T *sc = reinterpret_cast<T *>(smraw);   // c
  T *ss = sc + np;                         // s
  T *sdp = ss + np;                        // new a_pp
  T *sdq = sdp + np;                       // new a_qq
  cx<T> *sph = reinterpret_cast<cx<T> *>(smraw + (size_t)4 * np * sizeof(double));  // e^{-i phi}
  int *sp = reinterpret_cast<int *>(sph + np);
  int *sq = sp + np;
  int *sskip = sq + np;
  double *slam = reinterpret_cast<double *>(sskip + np + (np & 1));
  int *srank = reinterpret_cast<int *>(slam + n);
  __shared__ unsigned long long s_off;
  __shared__ unsigned long long s_amax;

  if (init_identity)
    for (size_t e = tid; e < (size_t)n * n; e += EIG_THREADS) {
      const int i = e % n, j = e / n;
      V[e] = mkc<T>(i == j ? T(1) : T(0), T(0));
    }
  if (tid == 0) s_amax = 0ull;
  __syncthreads();
  {
    double am = 0.0;
    for (size_t e = tid; e < (size_t)n * n; e += EIG_THREADS) am = fmax(am, (double)cabs1(A[e]));
    atomic_max_pos(&s_amax, am);
  }
  __syncthreads();
  const double amax = fmax(__longlong_as_double((long long)s_amax), 1e-300);
  const double rot_thresh = 1e-18 * amax;
  const double conv = conv_rel * amax;
  int converged = 0, sweep = 0;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_off = 0ull;
    __syncthreads();
    for (int r = 0; r < m - 1; ++r) {
      for (int k = tid; k < np; k += EIG_THREADS) {
        int p, q;
        if (k == 0) {
          p = m - 1;
          q = r;
        } else {
          p = (r + k) % (m - 1);
          q = (r - k + (m - 1)) % (m - 1);
        }
        if (p > q) { const int t = p; p = q; q = t; }
        sp[k] = p;
        sq[k] = q;
        int skip = 1;
        if (q < n) {
          const T app = A[p + (size_t)p * n].re, aqq = A[q + (size_t)q * n].re;
          const cx<T> apq = A[p + (size_t)q * n];
          const T mag = hypot(apq.re, apq.im);
          if (mag > T(0)) atomic_max_pos(&s_off, (double)mag);
          if ((double)mag > rot_thresh) {
            const T theta = (aqq - app) / (T(2) * mag);
            const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
            const T c = T(1) / sqrt(t * t + T(1));
            sc[k] = c;
            ss[k] = t * c;
            sph[k] = mkc<T>(apq.re / mag, -apq.im / mag);
            sdp[k] = app - t * mag;
            sdq[k] = aqq + t * mag;
            skip = 0;
          }
        }
        sskip[k] = skip;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (size_t e = tid; e < (size_t)np * n; e += EIG_THREADS) {
        const int k = e / n, i = e % n;
        if (sskip[k]) continue;
        const int p = sp[k], q = sq[k];
        const T c = sc[k], s = ss[k];
        const cx<T> ph = sph[k];
        {
          const cx<T> x = A[i + (size_t)p * n], y = cmul(ph, A[i + (size_t)q * n]);
          A[i + (size_t)p * n] = mkc<T>(c * x.re - s * y.re, c * x.im - s * y.im);
          A[i + (size_t)q * n] = mkc<T>(s * x.re + c * y.re, s * x.im + c * y.im);
        }
        {
          const cx<T> x = V[i + (size_t)p * n], y = cmul(ph, V[i + (size_t)q * n]);
          V[i + (size_t)p * n] = mkc<T>(c * x.re - s * y.re, c * x.im - s * y.im);
          V[i + (size_t)q * n] = mkc<T>(s * x.re + c * y.re, s * x.im + c * y.im);
        }
      }
      __syncthreads();
      // rows: A <- J^H A; the 2x2 blocks take their exact values
      for (size_t e = tid; e < (size_t)np * n; e += EIG_THREADS) {
        const int k = e / n, j = e % n;
        if (sskip[k]) continue;
        const int p = sp[k], q = sq[k];
        const T c = sc[k], s = ss[k];
        const cx<T> phc = cconj(sph[k]);
        if (j == p) {
          A[p + (size_t)p * n] = mkc<T>(sdp[k], T(0));
          A[q + (size_t)p * n] = czero<T>();
        } else if (j == q) {
          A[q + (size_t)q * n] = mkc<T>(sdq[k], T(0));
          A[p + (size_t)q * n] = czero<T>();
        } else {
          const cx<T> x = A[p + (size_t)j * n], y = cmul(phc, A[q + (size_t)j * n]);
          A[p + (size_t)j * n] = mkc<T>(c * x.re - s * y.re, c * x.im - s * y.im);
          A[q + (size_t)j * n] = mkc<T>(s * x.re + c * y.re, s * x.im + c * y.im);
        }
      }
      __syncthreads();
    }
    converged = __longlong_as_double((long long)s_off) <= conv;
    __syncthreads();
  }
  if (tid == 0) sweeps_out[mat] = converged ? sweep : -1;
  if (!En_all) return;
  // eigenvalues ascending (ties by index); eigenvector columns written to U
  double *En = En_all + (size_t)mat * n;
  zc *U = U_all + (size_t)mat * n * n;
  for (int i = tid; i < n; i += EIG_THREADS) slam[i] = (double)A[i + (size_t)i * n].re;
  __syncthreads();
  for (int i = tid; i < n; i += EIG_THREADS) {
    const double li = slam[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = slam[j];
      rank += (lj < li) || (lj == li && j < i);
    }
    En[rank] = li;
    srank[i] = rank;
  }
  __syncthreads();
  for (size_t e = tid; e < (size_t)n * n; e += EIG_THREADS) {
    const int i = e % n, j = e / n;
    U[i + (size_t)srank[j] * n] = ccast<double>(V[e]);
  }
}

template <typename T>
size_t jacobi_smem(int n) {
  const int np = ((n + 1) & ~1) / 2;
  return (size_t)4 * np * sizeof(double) + (size_t)np * sizeof(zc) + (size_t)(3 * np + 2) * sizeof(int) +
         (size_t)n * (sizeof(double) + sizeof(int)) + 64;
}

// ---------------------------------------------------------------------------
// Batched Hermitian eigensolver, tridiagonal route (FP64, one CTA per matrix):
//   1. Householder reduction Q^H A Q = T (T real symmetric tridiagonal).  For
//      column k, x = A[k+1:, k], alpha = x_0, beta = -sign(Re alpha) ||x||,
//      tau = (beta - alpha) / beta, v = (1, x_1.. / (alpha - beta)), so that
//      (I - tau v v^H)^H x = beta e_1; the trailing block is updated as
//      p = tau A v, c = Re(conj(tau) v^H p) / 2, w = p - c v,
//      A <- A - v w^H - w v^H.
//   2. Implicit QL with Wilkinson-type shifts on (d, e), rotations accumulated
//      into Z (each thread streams its rows; the rotation sequence of a QL
//      step is formed once in shared memory).  The QL step is the published
//      algorithm of H. Bowdler, R. S. Martin, C. Reinsch and J. H. Wilkinson,
//      "The QR and QL algorithms for symmetric matrices", Numer. Math. 11
//      (1968) 293-306 (tql2 in EISPACK): a shift from the leading 2 x 2 block
//      of the unreduced part, then plane rotations chasing the bulge from its
//      bottom up; written here from that description.
//   3. Back-transformation U = Q_0 Q_1 ... Q_{n-2} Z, then ascending sort.
// Memory traffic is O(n^3) bytes per matrix in total (the two-sided Jacobi
// streams the matrix every round), so this route is FP64-bound.
// ---------------------------------------------------------------------------
constexpr int HEEV_THREADS = 512;

// Arithmetic of the eigensolver's O(n^3) parts, native FP64 or double-float
// (pw_df.cuh).  Matrices stay 16-byte complex elements in global memory in
// either case (a double-float complex is two float pairs); the tridiagonal
// (d, e), the QL rotations' construction and every scalar of the Householder
// steps (norms, tau, 1/(alpha - beta)) are FP64 in both.
template <typename R>
struct HeevAr;

template <>
struct HeevAr<double> {
  typedef zc C;
  static __device__ __forceinline__ C from(zc z) { return z; }
  static __device__ __forceinline__ zc to(C z) { return z; }
  static __device__ __forceinline__ C zero() { return czero<double>(); }
  static __device__ __forceinline__ C one() { return mkc<double>(1.0, 0.0); }
  static __device__ __forceinline__ bool is_zero(C z) { return z.re == 0.0 && z.im == 0.0; }
  static __device__ __forceinline__ double norm2(C z) { return cnorm2(z); }
  static __device__ __forceinline__ C mul(C a, C b) { return cmul(a, b); }
  static __device__ __forceinline__ void fma(C &acc, C a, C b) { cfma(acc, a, b); }
  // acc += conj(a) b (the products and sums as fused multiply-adds, here and
  // below: one FP64 instruction per real product)
  static __device__ __forceinline__ void jfma(C &acc, C a, C b) {
    acc.re = ::fma(a.re, b.re, acc.re);
    acc.re = ::fma(a.im, b.im, acc.re);
    acc.im = ::fma(a.re, b.im, acc.im);
    acc.im = ::fma(-a.im, b.re, acc.im);
  }
  static __device__ __forceinline__ void renorm(C &) {}
  static __device__ __forceinline__ C add(C a, C b) { return cadd(a, b); }
  // a - c v
  static __device__ __forceinline__ C sub_scaled(C a, double c, C v) { return csub(a, cscale(c, v)); }
  // a - v conj(w_j) - w conj(v_j)
  static __device__ __forceinline__ C rank2(C a, C v, C wj, C w, C vj) {
    a.re = ::fma(-v.re, wj.re, a.re);
    a.re = ::fma(-v.im, wj.im, a.re);
    a.re = ::fma(-w.re, vj.re, a.re);
    a.re = ::fma(-w.im, vj.im, a.re);
    a.im = ::fma(-v.im, wj.re, a.im);
    a.im = ::fma(v.re, wj.im, a.im);
    a.im = ::fma(-w.im, vj.re, a.im);
    a.im = ::fma(w.re, vj.im, a.im);
    return a;
  }
  // a - v p
  static __device__ __forceinline__ C sub_mul(C a, C v, C p) {
    a.re = ::fma(-v.re, p.re, a.re);
    a.re = ::fma(v.im, p.im, a.re);
    a.im = ::fma(-v.re, p.im, a.im);
    a.im = ::fma(-v.im, p.re, a.im);
    return a;
  }
  typedef double Rot;
  static __device__ __forceinline__ Rot rot_of(double c) { return c; }
  // (s y + c x, c y - s x)
  static __device__ __forceinline__ void rot(C y, C x, Rot c, Rot s, C &hi, C &lo) {
    hi = mkc<double>(s * y.re + c * x.re, s * y.im + c * x.im);
    lo = mkc<double>(c * y.re - s * x.re, c * y.im - s * x.im);
  }
  static __device__ __forceinline__ C shfl_down(C z, int off) {
    return mkc<double>(__shfl_down_sync(0xffffffffu, z.re, off), __shfl_down_sync(0xffffffffu, z.im, off));
  }
};

template <>
struct HeevAr<df> {
  typedef dfc C;
  static __device__ __forceinline__ C from(zc z) { return dfc_of(z); }
  static __device__ __forceinline__ zc to(C z) { return dfc_val(z); }
  static __device__ __forceinline__ C zero() { return czero<df>(); }
  static __device__ __forceinline__ C one() {
    C z = czero<df>();
    z.re.hi = 1.f;
    return z;
  }
  static __device__ __forceinline__ bool is_zero(C z) { return z.re.hi == 0.f && z.im.hi == 0.f; }
  static __device__ __forceinline__ double norm2(C z) {
    const double r = df_val(z.re), i = df_val(z.im);
    return r * r + i * i;
  }
  static __device__ __forceinline__ df dmul(df a, df b) { return df_mul(a, b); }
  static __device__ __forceinline__ C mul(C a, C b) {
    C r = czero<df>();
    df_fma_lazy(r.re, a.re, b.re);
    df_fma_lazy(r.re, df_neg(a.im), b.im);
    df_fma_lazy(r.im, a.re, b.im);
    df_fma_lazy(r.im, a.im, b.re);
    cacc_renorm(r);
    return r;
  }
  static __device__ __forceinline__ void fma(C &acc, C a, C b) { cfma(acc, a, b); }
  static __device__ __forceinline__ void jfma(C &acc, C a, C b) {
    df_fma_lazy(acc.re, a.re, b.re);
    df_fma_lazy(acc.re, a.im, b.im);
    df_fma_lazy(acc.im, a.re, b.im);
    df_fma_lazy(acc.im, df_neg(a.im), b.re);
  }
  static __device__ __forceinline__ void renorm(C &a) { cacc_renorm(a); }
  static __device__ __forceinline__ C add(C a, C b) {
    C r;
    r.re = df_add(a.re, b.re);
    r.im = df_add(a.im, b.im);
    return r;
  }
  static __device__ __forceinline__ C sub_scaled(C a, double c, C v) {
    const df m = df_of(-c);
    df_fma_lazy(a.re, m, v.re);
    df_fma_lazy(a.im, m, v.im);
    cacc_renorm(a);
    return a;
  }
  static __device__ __forceinline__ C rank2(C a, C v, C wj, C w, C vj) {
    // re -= v.re wj.re + v.im wj.im + w.re vj.re + w.im vj.im
    df_fma_lazy(a.re, df_neg(v.re), wj.re);
    df_fma_lazy(a.re, df_neg(v.im), wj.im);
    df_fma_lazy(a.re, df_neg(w.re), vj.re);
    df_fma_lazy(a.re, df_neg(w.im), vj.im);
    // im -= v.im wj.re - v.re wj.im + w.im vj.re - w.re vj.im
    df_fma_lazy(a.im, df_neg(v.im), wj.re);
    df_fma_lazy(a.im, v.re, wj.im);
    df_fma_lazy(a.im, df_neg(w.im), vj.re);
    df_fma_lazy(a.im, w.re, vj.im);
    cacc_renorm(a);
    return a;
  }
  static __device__ __forceinline__ C sub_mul(C a, C v, C p) {
    df_fma_lazy(a.re, df_neg(v.re), p.re);
    df_fma_lazy(a.re, v.im, p.im);
    df_fma_lazy(a.im, df_neg(v.re), p.im);
    df_fma_lazy(a.im, df_neg(v.im), p.re);
    cacc_renorm(a);
    return a;
  }
  typedef df Rot;
  static __device__ __forceinline__ Rot rot_of(double c) { return df_of(c); }
  static __device__ __forceinline__ void rot(C y, C x, Rot c, Rot s, C &hi, C &lo) {
    hi = czero<df>();
    lo = czero<df>();
    df_fma_lazy(hi.re, s, y.re);
    df_fma_lazy(hi.re, c, x.re);
    df_fma_lazy(hi.im, s, y.im);
    df_fma_lazy(hi.im, c, x.im);
    df_fma_lazy(lo.re, c, y.re);
    df_fma_lazy(lo.re, df_neg(s), x.re);
    df_fma_lazy(lo.im, c, y.im);
    df_fma_lazy(lo.im, df_neg(s), x.im);
    cacc_renorm(hi);
    cacc_renorm(lo);
  }
  static __device__ __forceinline__ C shfl_down(C z, int off) {
    C r;
    r.re.hi = __shfl_down_sync(0xffffffffu, z.re.hi, off);
    r.re.lo = __shfl_down_sync(0xffffffffu, z.re.lo, off);
    r.im.hi = __shfl_down_sync(0xffffffffu, z.im.hi, off);
    r.im.lo = __shfl_down_sync(0xffffffffu, z.im.lo, off);
    return r;
  }
};

// Block sum of a complex value in the solver's arithmetic (returned as FP64).
template <typename R, int NTH>
__device__ zc block_csum(typename HeevAr<R>::C v, typename HeevAr<R>::C *scratch) {
  typedef HeevAr<R> Ar;
  for (int off = 16; off > 0; off >>= 1) v = Ar::add(v, Ar::shfl_down(v, off));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < NTH / 32 ? scratch[lane] : Ar::zero();
    for (int off = 16; off > 0; off >>= 1) v = Ar::add(v, Ar::shfl_down(v, off));
    if (lane == 0) scratch[32] = v;
  }
  __syncthreads();
  const zc r = Ar::to(scratch[32]);
  __syncthreads();
  return r;
}

// Workspace of the split double-float route (per matrix of a launch group):
// the tridiagonal (d, e), the Householder scalars, and the QL rotation stream
// (steps (m, lo), then the rotations i = m-1 .. lo of each step as
// (c_hi, c_lo, s_hi, s_lo)).
struct HeevWS {
  double *d, *e;        // n per matrix; d holds the eigenvalues after the QL kernel
  dfc *tau;             // n per matrix
  float4 *rot;          // rot_cap per matrix
  int2 *steps;          // step_cap per matrix
  int *nsteps;          // 1 per matrix
  int rot_cap, step_cap;
};

// ---- eigenvectors of the split route: Z = product of the recorded QL
// rotations, U = Q Z, then the ascending sort (three launches after k_ql_df).
//
// Rotation (s, i) of QL step s replaces columns (i, i+1) of every row z of Z by
// (c z_i - s z_{i+1}, s z_i + c z_{i+1}).  Rows are independent: one thread per
// row.  Step s+1 may rotate columns (i, i+1) as soon as step s has finished
// every rotation touching column i, i.e. its rotation i-1, so ROT_K consecutive
// steps run as a wavefront with a lag of two columns: at time c step k applies
// its rotation i = c + 2k, and the ROT_K rotations of one time touch disjoint
// column pairs inside the window [c, c + 2 ROT_K - 1], which lives in
// registers.  Each pass over the row therefore applies ROT_K steps while
// reading and writing every column once (the column-by-column form streams the
// whole of Z from memory once per step).  A step with no rotation at some time
// applies the identity (c = 1, s = 0, exact in double-float), so the body of a
// time is straight-line code.
constexpr int ROT_ROWS = 64;    // rows (threads) per CTA
constexpr int ROT_K = 16;       // QL steps per pass

// a b + c d in double-float (products formed exactly by FMA, one
// normalisation)
__device__ __forceinline__ df df_dot2(df a, df b, df c, df d) {
  const float p1 = a.hi * b.hi;
  float e1 = fmaf(a.hi, b.hi, -p1);
  e1 = fmaf(a.hi, b.lo, e1);
  e1 = fmaf(a.lo, b.hi, e1);
  const float p2 = c.hi * d.hi;
  float e2 = fmaf(c.hi, d.hi, -p2);
  e2 = fmaf(c.hi, d.lo, e2);
  e2 = fmaf(c.lo, d.hi, e2);
  float sh, sl;
  two_sum(p1, p2, sh, sl);
  sl += e1 + e2;
  float h, l;
  fast_two_sum(sh, sl, h, l);
  return mkdf(h, l);
}
// (y, x) <- (c y - s x, s y + c x)
__device__ __forceinline__ void rot_df(dfc &y, dfc &x, df c, df sn) {
  const df nsn = df_neg(sn);
  const dfc hi = {df_dot2(sn, y.re, c, x.re), df_dot2(sn, y.im, c, x.im)};
  const dfc lo = {df_dot2(c, y.re, nsn, x.re), df_dot2(c, y.im, nsn, x.im)};
  x = hi;
  y = lo;
}

// grid (ceil(n / ROT_ROWS), nmat); Z (n x n per matrix, column-major,
// double-float) is written from the identity.
__global__ void __launch_bounds__(ROT_ROWS) k_rot_apply(HeevWS ws, dfc *Z_all, int *status, int n) {
  constexpr int W2 = 2 * ROT_K;
  __shared__ int sm_m[ROT_K], sm_lo[ROT_K], sm_r0[ROT_K];
  const int mat = blockIdx.y;
  const int row = blockIdx.x * ROT_ROWS + threadIdx.x;
  const bool act = row < n;
  dfc *Z = Z_all + (size_t)mat * n * n;
  const int nst = min(max(ws.nsteps[mat], 0), ws.step_cap);
  const int2 *steps = ws.steps + (size_t)mat * ws.step_cap;
  const float4 *rot = ws.rot + (size_t)mat * ws.rot_cap;
  dfc zero = czero<df>(), one = zero;
  one.re.hi = 1.f;
  if (act)
    for (int j = 0; j < n; ++j) Z[row + (size_t)j * n] = j == row ? one : zero;
  int r0 = 0;          // thread 0: rotations of the steps before this pass
  bool bad = false;
  for (int s0 = 0; s0 < nst; s0 += ROT_K) {
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 0; k < ROT_K; ++k) {
        int m = 0, lo = 0;
        if (s0 + k < nst) {
          const int2 ml = steps[s0 + k];
          m = ml.x;
          lo = ml.y;
          // a step outside the matrix or the stream cannot come from k_ql_df;
          // it is recorded, not followed
          if (m >= n || lo < 0 || lo > m || r0 + (m - lo) > ws.rot_cap) {
            bad = true;
            m = lo = 0;
          }
        }
        sm_m[k] = m;
        sm_lo[k] = lo;
        sm_r0[k] = r0;
        r0 += m - lo;
      }
    }
    __syncthreads();
    int mk[ROT_K], lk[ROT_K], rk[ROT_K];
    int c_hi = -(1 << 30), c_lo = 1 << 30;
#pragma unroll
    for (int k = 0; k < ROT_K; ++k) {
      mk[k] = sm_m[k];
      lk[k] = sm_lo[k];
      rk[k] = sm_r0[k] + sm_m[k] - 1;   // stream index of rotation i: rk - i
      if (mk[k] > lk[k]) {
        c_hi = max(c_hi, mk[k] - 1 - 2 * k);
        c_lo = min(c_lo, lk[k] - 2 * k);
      }
    }
    if (!act || c_hi < c_lo) continue;
    // w[q] holds column c + q at time c; columns outside [0, n) are never
    // rotated (every rotated column lies in [lo_k, m_k] of its step)
    dfc w[W2];
#pragma unroll
    for (int q = 0; q < W2; ++q) {
      const int cc = c_hi + q;
      w[q] = cc >= 0 && cc < n ? Z[row + (size_t)cc * n] : zero;
    }
    dfc nxt = c_hi - 1 >= 0 ? Z[row + (size_t)(c_hi - 1) * n] : zero;
    for (int c = c_hi;; --c) {
#pragma unroll
      for (int k = 0; k < ROT_K; ++k) {
        const int i = c + 2 * k;
        const bool on = i >= lk[k] && i < mk[k];
        const float4 q = on ? rot[rk[k] - i] : make_float4(1.f, 0.f, 0.f, 0.f);
        rot_df(w[2 * k], w[2 * k + 1], mkdf(q.x, q.y), mkdf(q.z, q.w));
      }
      if (c == c_lo) break;
      // column c + W2 - 1 leaves the window, column c - 1 enters
      if (c + W2 - 1 < n) Z[row + (size_t)(c + W2 - 1) * n] = w[W2 - 1];
#pragma unroll
      for (int q = W2 - 1; q > 0; --q) w[q] = w[q - 1];
      w[0] = nxt;
      if (c - 2 >= 0) nxt = Z[row + (size_t)(c - 2) * n];
    }
#pragma unroll
    for (int q = 0; q < W2; ++q) {
      const int cc = c_lo + q;
      if (cc >= 0 && cc < n) Z[row + (size_t)cc * n] = w[q];
    }
  }
  if (bad) status[mat] = -1;
}

// U = Q Z by the stored Householder vectors (Q_{n-2} applied first): one warp
// per BT_COLS columns of Z, held in shared memory (each loaded Householder
// element serves all of them, and their reductions interleave); Householder
// vector k is column k of the reduced matrix A below the subdiagonal (unit
// leading element implied).  The result goes back to Z's columns (FP64
// complex in place of the double-float element, both 16 bytes).
constexpr int BT_WARPS = 8, BT_COLS = 1;
__global__ void __launch_bounds__(BT_WARPS * 32) k_backtransform(const dfc *A_all, dfc *Z_all, HeevWS ws, int n) {
  extern __shared__ __align__(16) unsigned char smraw[];
  typedef HeevAr<df> Ar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mat = blockIdx.y, j0 = (blockIdx.x * BT_WARPS + warp) * BT_COLS;
  if (j0 >= n) return;
  const int ncol = min(BT_COLS, n - j0);
  const size_t nn = (size_t)n * n;
  const dfc *A = A_all + mat * nn;
  dfc *Zc = Z_all + mat * nn + (size_t)j0 * n;
  dfc *z = reinterpret_cast<dfc *>(smraw) + (size_t)warp * BT_COLS * n;   // z[i + c n]
  const dfc *tau_m = ws.tau + (size_t)mat * n;
  for (int q = lane; q < ncol * n; q += 32) z[q] = Zc[q];
  for (int q = ncol * n + lane; q < BT_COLS * n; q += 32) z[q] = Ar::zero();   // a missing last column
  __syncwarp();
  for (int k = n - 2; k >= 0; --k) {
    const dfc tau = tau_m[k];
    if (Ar::is_zero(tau)) continue;
    const dfc *x = A + (size_t)k * n;   // v_r = x[r] for r > k + 1, v_{k+1} = 1
    dfc acc[BT_COLS];
#pragma unroll
    for (int c = 0; c < BT_COLS; ++c) acc[c] = Ar::zero();
    for (int r = k + 1 + lane; r < n; r += 32) {
      const dfc v = r == k + 1 ? Ar::one() : x[r];
#pragma unroll
      for (int c = 0; c < BT_COLS; ++c) Ar::jfma(acc[c], v, z[r + c * n]);
    }
    dfc p[BT_COLS];
#pragma unroll
    for (int c = 0; c < BT_COLS; ++c) {
      Ar::renorm(acc[c]);
      for (int off = 16; off > 0; off >>= 1) acc[c] = Ar::add(acc[c], Ar::shfl_down(acc[c], off));
      acc[c] = Ar::mul(tau, acc[c]);
      p[c] = {mkdf(__shfl_sync(0xffffffffu, acc[c].re.hi, 0), __shfl_sync(0xffffffffu, acc[c].re.lo, 0)),
              mkdf(__shfl_sync(0xffffffffu, acc[c].im.hi, 0), __shfl_sync(0xffffffffu, acc[c].im.lo, 0))};
    }
    for (int r = k + 1 + lane; r < n; r += 32) {
      const dfc v = r == k + 1 ? Ar::one() : x[r];
#pragma unroll
      for (int c = 0; c < BT_COLS; ++c) z[r + c * n] = Ar::sub_mul(z[r + c * n], v, p[c]);
    }
    __syncwarp();
  }
  zc *out = reinterpret_cast<zc *>(Zc);
  for (int q = lane; q < ncol * n; q += 32) out[q] = Ar::to(z[q]);
}

// Ascending eigenvalues (ties by index) and the matching columns into HU and
// En; the last launch of the split route, so it also completes the status.
__global__ void __launch_bounds__(256) k_eig_sort(const zc *U_all, zc *HU_all, double *En_all, const double *d_all,
                                                 int *status, int n) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mat = blockIdx.y, j = blockIdx.x * 8 + warp;
  if (blockIdx.x == 0 && threadIdx.x == 0 && status[mat] >= 0) status[mat] = 1;
  if (j >= n) return;
  const size_t nn = (size_t)n * n;
  const double *d = d_all + (size_t)mat * n;
  const double lj = d[j];
  int r = 0;
  for (int i = lane; i < n; i += 32) r += (d[i] < lj) || (d[i] == lj && i < j);
  for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
  r = __shfl_sync(0xffffffffu, r, 0);
  if (lane == 0) En_all[(size_t)mat * n + r] = lj;
  const zc *src = U_all + mat * nn + (size_t)j * n;
  zc *dst = HU_all + mat * nn + (size_t)r * n;
  for (int i = lane; i < n; i += 32) dst[i] = src[i];
}

// The QL recurrence of the split route in double-float on the FP32 pipe, one
// matrix per 32-thread block (thread 0 runs the scalar recurrence; GB300's
// FP64 pipe retires a scalar FP64 operation far slower than the FP32 pipe
// retires the ~10 FP32 operations of its double-float counterpart).  Same
// implicit QL as part 0 (Bowdler, Martin, Reinsch and Wilkinson, 1968: shift
// from the leading 2 x 2 block, rotations from the bottom of the unreduced
// block up); the deflation test uses the
// double-float resolution (4e-15 relative).  Writes the eigenvalues into
// ws.d, the step list and the rotations; status -1 when an eigenvalue needs
// more than 60 iterations or the stream exceeds its capacity.
__device__ __forceinline__ df hypot_df(df a, df b) {
  const float big = fmaxf(fabsf(a.hi), fabsf(b.hi));
  if (big == 0.f) return mkdf(0.f, 0.f);
  // scale small arguments by an exact power of two so that the squares stay normal
  const float sc = big < 1e-15f ? 18446744073709551616.f : 1.f;   // 2^64
  const df as = df_mul_f(a, sc), bs = df_mul_f(b, sc);
  const df r = df_sqrt(df_add(df_mul(as, as), df_mul(bs, bs)));
  return sc == 1.f ? r : df_mul_f(r, 1.f / sc);
}

__global__ void __launch_bounds__(32) k_ql_df(HeevWS ws, int *status, int n) {
  extern __shared__ __align__(16) unsigned char smraw[];
  df *dd = reinterpret_cast<df *>(smraw);
  df *ee = dd + n;
  const int mat = blockIdx.x;
  double *gd = ws.d + (size_t)mat * n;
  const double *ge = ws.e + (size_t)mat * n;
  for (int i = threadIdx.x; i < n; i += 32) {
    dd[i] = df_of(gd[i]);
    ee[i] = df_of(ge[i]);
  }
  __syncwarp();
  if (threadIdx.x != 0) return;
  float4 *rot = ws.rot + (size_t)mat * ws.rot_cap;
  int2 *steps = ws.steps + (size_t)mat * ws.step_cap;
  const float eps = 4e-15f;
  int nrot = 0, nst = 0;
  bool failed = false;
  for (int l = 0; l < n && !failed; ++l) {
    int iter = 0;
    for (;;) {
      int m = l;
      for (; m < n - 1; ++m) {
        const float s2 = fabsf(dd[m].hi) + fabsf(dd[m + 1].hi);
        if (fabsf(ee[m].hi) <= eps * s2) break;
      }
      if (m == l) break;
      if (++iter > 60 || nst >= ws.step_cap || nrot + (m - l) > ws.rot_cap) {
        failed = true;
        break;
      }
      df g = df_div(df_sub(dd[l + 1], dd[l]), df_mul_f(ee[l], 2.f));
      df r = hypot_df(g, df_from_float(1.f));
      g = df_add(df_sub(dd[m], dd[l]), df_div(ee[l], g.hi >= 0.f ? df_add(g, r) : df_sub(g, r)));
      df sn = df_from_float(1.f), c = df_from_float(1.f), p = df_from_float(0.f);
      int lo = l;
      bool under = false;
      for (int i = m - 1; i >= l; --i) {
        const df f = df_mul(sn, ee[i]), b = df_mul(c, ee[i]);
        r = hypot_df(f, g);
        ee[i + 1] = r;
        if (r.hi == 0.f) {
          dd[i + 1] = df_sub(dd[i + 1], p);
          ee[m] = df_from_float(0.f);
          under = true;
          lo = i + 1;
          break;
        }
        const df inv = df_div(df_from_float(1.f), r);
        sn = df_mul(f, inv);
        c = df_mul(g, inv);
        g = df_sub(dd[i + 1], p);
        r = df_add(df_mul(df_sub(dd[i], g), sn), df_mul_f(df_mul(c, b), 2.f));
        p = df_mul(sn, r);
        dd[i + 1] = df_add(g, p);
        g = df_sub(df_mul(c, r), b);
        rot[nrot++] = make_float4(c.hi, c.lo, sn.hi, sn.lo);
      }
      if (!under) {
        dd[l] = df_sub(dd[l], p);
        ee[l] = g;
        ee[m] = df_from_float(0.f);
      }
      steps[nst++] = make_int2(m, lo);
    }
  }
  for (int i = 0; i < n; ++i) gd[i] = df_val(dd[i]);
  ws.nsteps[mat] = nst;
  status[mat] = failed ? -1 : 0;
}

// part 0: the whole solver in one kernel (thread 0 runs the QL recurrence);
// part 1: Householder reduction only, (d, e, tau) to the workspace (the
// split route continues with k_ql_df, k_rot_apply, k_backtransform and
// k_eig_sort).
template <typename R>
__global__ void __launch_bounds__(HEEV_THREADS, 2) k_heev(zc *HU_all, zc *Z_all, double *En_all,
                                                       int *status, int n, int part, HeevWS ws,
                                                       int remap_last) {
  typedef HeevAr<R> Ar;
  typedef typename Ar::C C;
  typedef typename Ar::Rot Rot;
  constexpr int NTH = HEEV_THREADS;
  extern __shared__ __align__(16) unsigned char smraw[];
  // remap_last >= 0: the grid's last CTA takes matrix remap_last instead
  const int mat = (remap_last >= 0 && blockIdx.x == gridDim.x - 1) ? remap_last : (int)blockIdx.x;
  const int tid = threadIdx.x;
  const size_t nn = (size_t)n * n;
  zc *A64 = HU_all + mat * nn;
  C *A = reinterpret_cast<C *>(A64);          // the matrix in the solver's format, in place
  C *Z = reinterpret_cast<C *>(Z_all + mat * nn);
  double *En = En_all + (size_t)mat * n;
  C *v = reinterpret_cast<C *>(smraw);
  C *pw_ = v + n;
  C *taus = pw_ + n;
  C *vnx = taus + n;                    // the next step's reflector
  C *pn = vnx + n;                      // A22 times it (the fused pass)
  C *cred = pn + n;                     // 33 complex: block reductions
  double *d = reinterpret_cast<double *>(cred + 33);
  double *e = d + n;
  double *cs = e + n;                   // 2n: the rotations of two QL steps
  double *sn = cs + 2 * n;
  Rot *csr = reinterpret_cast<Rot *>(sn + 2 * n);
  Rot *snr = csr + 2 * n;
  int *ctl = reinterpret_cast<int *>(snr + 2 * n);   // two QL steps' control words; [8] failed
  int *rank = ctl + 16;
  {
    // the carve above must fit the launch's dynamic shared memory
    unsigned dyn = 0;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const size_t need = (size_t)(reinterpret_cast<unsigned char *>(rank + n) - smraw);
    if (need > dyn) {
      if (tid == 0) {
        printf("k_heev: needs %llu bytes of shared memory, launched with %u\n", (unsigned long long)need, dyn);
        status[mat] = -2;
      }
      return;
    }
  }
  if (tid == 0) ctl[8] = 0;
  if constexpr (!std::is_same<R, double>::value) {
    // to the solver's format, element by element in place
    for (size_t q = tid; q < nn; q += NTH) {
      const zc z = A64[q];
      A[q] = Ar::from(z);
    }
    __syncthreads();
  }

  // ---- 1. Householder tridiagonalisation
  // Step k reflects column k (below the diagonal) with v_k, tau_k, forms
  // w_k = p - (Re(conj(tau) v^H p)/2) v with p = tau A22 v, and updates the
  // trailing matrix A22 <- A22 - v w^H - w v^H.  The update is fused with the
  // next step's product: column 0 of A22 is updated first, step k+1's
  // reflector is formed from it, and one pass over A22[1:, 1:] both updates
  // each element and accumulates A22[1:, 1:] v_{k+1} -- one read and one write
  // of the trailing matrix per step instead of two reads and a write.
  // Row 0 of A22 beyond its diagonal is never read again and is left as is.
  C *vc = v, *vn = vnx;   // reflector of this step, of the next
  // the reflector of column k from x = A[k+1:, k]: v (stored below the
  // diagonal too), d[k], e[k], taus[k]; returns tau (FP64)
  auto reflect = [&](int k, C *vv) -> zc {
    const int m = n - k - 1;
    C *x = A + (k + 1) + (size_t)k * n;
    C part = Ar::zero();
    for (int i = 1 + tid; i < m; i += NTH) Ar::jfma(part, x[i], x[i]);
    Ar::renorm(part);
    const double xn2 = block_csum<R, NTH>(part, cred).re;
    const zc alpha = Ar::to(x[0]);
    zc tau;
    double beta;
    if (xn2 == 0.0 && alpha.im == 0.0) {
      tau = czero<double>();
      beta = alpha.re;
    } else {
      beta = -copysign(sqrt(cnorm2(alpha) + xn2), alpha.re);
      tau = mkc<double>((beta - alpha.re) / beta, -alpha.im / beta);
    }
    const bool skip = tau.re == 0.0 && tau.im == 0.0;
    const C scl = Ar::from(skip ? czero<double>() : cinv(mkc<double>(alpha.re - beta, alpha.im)));
    for (int i = tid; i < m; i += NTH) {
      const C vi = i == 0 ? Ar::one() : Ar::mul(x[i], scl);
      vv[i] = vi;
      if (i > 0) x[i] = vi;   // kept for the back-transformation
    }
    if (tid == 0) {
      d[k] = Ar::to(A[k + (size_t)k * n]).re;
      e[k] = beta;
      taus[k] = Ar::from(tau);
    }
    __syncthreads();
    return tau;
  };
  zc tau = reflect(0, vc);
  bool have_p = false;   // pn holds A22 v of this step (without tau)
  for (int k = 0; k + 1 < n; ++k) {
    const int m = n - k - 1;
    const bool skip = tau.re == 0.0 && tau.im == 0.0;
    C *A22 = A + (k + 1) + (size_t)(k + 1) * n;
    if (skip) {
      if (k + 2 < n) tau = reflect(k + 1, vc);
      have_p = false;
      continue;
    }
    const C tauc = Ar::from(tau);
    // p = tau A22 v
    if (have_p) {
      for (int i = tid; i < m; i += NTH) pw_[i] = Ar::mul(tauc, pn[i]);
    } else {
      for (int i = tid; i < m; i += NTH) {
        C acc = Ar::zero();
        for (int j = 0; j < m; ++j) {
          Ar::fma(acc, A22[i + (size_t)j * n], vc[j]);
          if ((j & 31) == 31) Ar::renorm(acc);
        }
        Ar::renorm(acc);
        pw_[i] = Ar::mul(tauc, acc);
      }
    }
    __syncthreads();
    C vp = Ar::zero();
    for (int i = tid; i < m; i += NTH) Ar::jfma(vp, vc[i], pw_[i]);
    Ar::renorm(vp);
    const zc vhp = block_csum<R, NTH>(vp, cred);
    const double c = 0.5 * (tau.re * vhp.re + tau.im * vhp.im);   // Re(conj(tau) v^H p)
    for (int i = tid; i < m; i += NTH) pw_[i] = Ar::sub_scaled(pw_[i], c, vc[i]);
    __syncthreads();
    // column 0 of A22 first: the next reflector comes from it
    for (int i = tid; i < m; i += NTH) A22[i] = Ar::rank2(A22[i], vc[i], pw_[0], pw_[i], vc[0]);
    __syncthreads();
    if (k + 2 >= n) break;   // A22 was 1 x 1
    const zc tau2 = reflect(k + 1, vn);
    const bool fuse = !(tau2.re == 0.0 && tau2.im == 0.0);
    // A22[1:, 1:] updated, and (fuse) pn = A22[1:, 1:] v_{k+1}, one row per thread
    for (int r = 1 + tid; r < m; r += NTH) {
      C acc = Ar::zero();
      const C vr = vc[r], wr = pw_[r];
      for (int j = 1; j < m; ++j) {
        C *aij = A22 + r + (size_t)j * n;
        const C a2 = Ar::rank2(*aij, vr, pw_[j], wr, vc[j]);
        *aij = a2;
        if (fuse) {
          Ar::fma(acc, a2, vn[j - 1]);
          if ((j & 31) == 0) Ar::renorm(acc);
        }
      }
      Ar::renorm(acc);
      pn[r - 1] = acc;
    }
    __syncthreads();
    C *t = vc;
    vc = vn;
    vn = t;
    tau = tau2;
    have_p = fuse;
  }
  if (tid == 0) {
    d[n - 1] = Ar::to(A[(n - 1) + (size_t)(n - 1) * n]).re;
    e[n - 1] = 0.0;
  }
  if constexpr (!std::is_same<R, double>::value) {
    if (part == 1) {
      __syncthreads();
      for (int i = tid; i < n; i += NTH) {
        ws.d[(size_t)mat * n + i] = d[i];
        ws.e[(size_t)mat * n + i] = e[i];
        ws.tau[(size_t)mat * n + i] = taus[i];
      }
      return;
    }
  }
  // The tridiagonal is real (e_k = beta_k), so are its eigenvectors: in FP64
  // they accumulate as a real n x n matrix in the first half of Z's storage
  // (half the arithmetic and traffic of the rotations) and become complex
  // before the back-transformation.
  constexpr bool real_z = std::is_same<R, double>::value;
  double *Zr = reinterpret_cast<double *>(Z);
  for (size_t q = tid; q < nn; q += NTH) {
    const int i = q % n, j = q / n;
    if constexpr (real_z) Zr[q] = i == j ? 1.0 : 0.0;
    else Z[q] = i == j ? Ar::one() : Ar::zero();
  }
  __syncthreads();

  // ---- 2. implicit QL on the tridiagonal (d, e), FP64
  // Thread 0 runs the recurrence one QL step ahead of the others: while
  // threads 32 .. NTH-1 apply step k's rotations to the rows of Z, thread 0
  // forms step k+1's (the recurrence reads and writes only d and e, never Z),
  // into the other half of the double-buffered rotation arrays and control
  // words.  gen(b) writes the next step into buffer b: ctl[4b] = m,
  // ctl[4b+1] = lo (rotations i = m-1 .. lo were formed), ctl[4b+3] = 1 when
  // every eigenvalue has converged.
  const double eps = 2.220446049250313e-16;
  int ql_l = 0, ql_iter = 0;   // thread 0's position in the recurrence
  auto gen = [&](int b) {
    int *cb = ctl + 4 * b;
    double *csb = cs + (size_t)b * n, *snb = sn + (size_t)b * n;
    Rot *csrb = csr + (size_t)b * n, *snrb = snr + (size_t)b * n;
    for (;;) {
      if (ql_l >= n) {
        cb[3] = 1;
        return;
      }
      const int l = ql_l;
      int m = l;
      for (; m < n - 1; ++m) {
        const double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) {   // d[l] has converged
        ++ql_l;
        ql_iter = 0;
        continue;
      }
      if (++ql_iter > 60) {   // recorded as a failure; the next eigenvalue follows
        ctl[8] = 1;
        ++ql_l;
        ql_iter = 0;
        continue;
      }
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      int lo = l;
      bool under = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = s * e[i], b2 = c * e[i];
        // r = |(f, g)|, s = f / r, c = g / r through one reciprocal square
        // root (f and g are of the size of the matrix entries here)
        const double q = fma(f, f, g * g);
        if (q == 0.0) {
          e[i + 1] = 0.0;
          d[i + 1] -= p;
          e[m] = 0.0;
          under = true;
          lo = i + 1;
          break;
        }
        const double ir = rsqrt(q);
        r = q * ir;
        e[i + 1] = r;
        s = f * ir;
        c = g * ir;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b2;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b2;
        csb[i] = c;
        snb[i] = s;
        csrb[i] = Ar::rot_of(c);
        snrb[i] = Ar::rot_of(s);
      }
      if (!under) {
        d[l] -= p;
        e[l] = g;
        e[m] = 0.0;
      }
      cb[0] = m;
      cb[1] = lo;
      cb[3] = 0;
      return;
    }
  };
  if (tid == 0) gen(0);
  __syncthreads();
  for (int step = 0;; ++step) {
    const int b = step & 1;
    const int m = ctl[4 * b], lo = ctl[4 * b + 1], fin = ctl[4 * b + 3];
    if (fin) break;
    if (m < 0 || m >= n || lo < 0 || lo > m) {   // cannot happen; recorded, not followed
      if (tid == 0) {
        printf("k_heev: QL step out of range (matrix %d, m %d, lo %d)\n", mat, m, lo);
        ctl[8] = 1;
      }
      break;
    }
    if (tid == 0) {
      gen(b ^ 1);
    } else if (tid >= 32 && lo < m) {
      const double *csb = cs + (size_t)b * n, *snb = sn + (size_t)b * n;
      const Rot *csrb = csr + (size_t)b * n, *snrb = snr + (size_t)b * n;
      for (int row = tid - 32; row < n; row += NTH - 32) {
        if constexpr (real_z) {
          double x = Zr[row + (size_t)m * n];
          for (int i = m - 1; i >= lo; --i) {
            const double y = Zr[row + (size_t)i * n], c = csb[i], s = snb[i];
            Zr[row + (size_t)(i + 1) * n] = fma(s, y, c * x);
            x = fma(c, y, -s * x);
          }
          Zr[row + (size_t)lo * n] = x;
        } else {
          C x = Z[row + (size_t)m * n];
          for (int i = m - 1; i >= lo; --i) {
            const C y = Z[row + (size_t)i * n];
            C hi, lo_;
            Ar::rot(y, x, csrb[i], snrb[i], hi, lo_);
            Z[row + (size_t)(i + 1) * n] = hi;
            x = lo_;
          }
          Z[row + (size_t)lo * n] = x;
        }
      }
    }
    __syncthreads();
  }

  if constexpr (real_z) {
    // real Z to complex in place, highest block of NTH entries first: block b
    // writes doubles [2 b NTH, 2 (b+1) NTH), above every entry that a lower
    // block has still to read
    for (long long b = ((long long)nn - 1) / NTH; b >= 0; --b) {
      const size_t q = (size_t)b * NTH + tid;
      const double val = q < nn ? Zr[q] : 0.0;
      __syncthreads();
      if (q < nn) {
        Zr[2 * q] = val;
        Zr[2 * q + 1] = 0.0;
      }
      __syncthreads();
    }
  }

  // ---- 3. back-transformation U = Q Z (Q_{n-2} first)
  const int warp = tid >> 5, lane = tid & 31;
  for (int k = n - 2; k >= 0; --k) {
    const C tau = taus[k];
    if (Ar::is_zero(tau)) continue;
    const int m = n - k - 1;
    const C *x = A + (k + 1) + (size_t)k * n;
    for (int i = tid; i < m; i += NTH) v[i] = i == 0 ? Ar::one() : x[i];
    __syncthreads();
    C *Zk = Z + (k + 1);
    for (int j = warp; j < n; j += NTH / 32) {
      C acc = Ar::zero();
      for (int i = lane; i < m; i += 32) Ar::jfma(acc, v[i], Zk[i + (size_t)j * n]);
      Ar::renorm(acc);
      for (int off = 16; off > 0; off >>= 1) acc = Ar::add(acc, Ar::shfl_down(acc, off));
      if (lane == 0) pw_[j] = Ar::mul(tau, acc);
    }
    __syncthreads();
    for (size_t q = tid; q < (size_t)m * n; q += NTH) {
      const int i = q % m, j = q / m;
      Zk[i + (size_t)j * n] = Ar::sub_mul(Zk[i + (size_t)j * n], v[i], pw_[j]);
    }
    __syncthreads();
  }

  // ---- 4. ascending order (ties by index), back to FP64 storage
  for (int i = tid; i < n; i += NTH) {
    const double li = d[i];
    int r = 0;
    for (int j = 0; j < n; ++j) r += (d[j] < li) || (d[j] == li && j < i);
    rank[i] = r;
    En[r] = li;
  }
  __syncthreads();
  for (size_t q = tid; q < nn; q += NTH) {
    const int i = q % n, j = q / n;
    A64[i + (size_t)rank[j] * n] = Ar::to(Z[q]);
  }
  if (tid == 0) status[mat] = ctl[8] ? -1 : 1;
}

size_t heev_smem(int n) {
  return (size_t)5 * n * sizeof(zc) + 33 * sizeof(zc) + (size_t)6 * n * sizeof(double) +
         (size_t)4 * n * sizeof(double) + (16 + (size_t)n) * sizeof(int) + 64;
}

// Workspace of the split double-float route for nmat matrices of order n.
namespace {
inline size_t ws_align(size_t b) { return (b + 255) & ~(size_t)255; }
inline int heev_rot_cap(int n) { return 3 * n * n + 64; }
inline int heev_step_cap(int n) { return 8 * n + 64; }
}  // namespace

size_t heev_ws_bytes(int n, int nmat) {
  if (n <= 0 || nmat <= 0) return 0;
  const size_t m = (size_t)nmat;
  return ws_align(m * n * sizeof(double)) * 2 + ws_align(m * n * sizeof(dfc)) +
         ws_align(m * heev_rot_cap(n) * sizeof(float4)) + ws_align(m * heev_step_cap(n) * sizeof(int2)) +
         ws_align(m * sizeof(int));
}

// HU: in H, out U; V: scratch of the same size; status: positive on success,
// negative when an eigenvalue did not converge.  double_float: the O(n^3)
// parts in double-float arithmetic on the FP32 pipe (the mixed form); with a
// workspace (ws, ws_bytes >= heev_ws_bytes(n, 1)) the QL recurrence runs in
// double-float too, split into three launches per group of matrices
// (reduction, QL stream, vectors); without one, in FP64 inside k_heev.
int heev_resident_per_sm(int n) {
  const size_t smem = heev_smem(n);
  cudaFuncSetAttribute(k_heev<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_heev<double>, HEEV_THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

void launch_eig(zc *HU, zc *V, double *En, int *status, int n, int nmat, cudaStream_t s, bool double_float,
                void *ws, size_t ws_bytes, bool tail, int remap_last) {
  if (nmat <= 0) return;
  const size_t smem = heev_smem(n);
  const size_t nn = (size_t)n * n;
  HeevWS w{};
  if (double_float) {
    cudaFuncSetAttribute(k_heev<df>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int group = 0;
    if (ws && nmat > 0) {
      group = nmat;
      while (group > 0 && heev_ws_bytes(n, group) > ws_bytes) group = std::max(0, group - std::max(1, group / 8));
    }
    if (group <= 0) {
      PW_TIMED(KK_HEEV, s, k_heev<df><<<nmat, HEEV_THREADS, smem, s>>>(HU, V, En, status, n, 0, w, -1));
      return;
    }
    const size_t g = (size_t)group;
    const size_t bt_smem = (size_t)BT_WARPS * BT_COLS * n * sizeof(dfc);
    cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_smem);
    unsigned char *p = static_cast<unsigned char *>(ws);
    w.d = reinterpret_cast<double *>(p);
    p += ws_align(g * n * sizeof(double));
    w.e = reinterpret_cast<double *>(p);
    p += ws_align(g * n * sizeof(double));
    w.tau = reinterpret_cast<dfc *>(p);
    p += ws_align(g * n * sizeof(dfc));
    w.rot = reinterpret_cast<float4 *>(p);
    p += ws_align(g * heev_rot_cap(n) * sizeof(float4));
    w.steps = reinterpret_cast<int2 *>(p);
    p += ws_align(g * heev_step_cap(n) * sizeof(int2));
    w.nsteps = reinterpret_cast<int *>(p);
    w.rot_cap = heev_rot_cap(n);
    w.step_cap = heev_step_cap(n);
    auto shifted = [&](int k) {   // the workspace of matrices k .. of a group
      HeevWS x = w;
      x.d += (size_t)k * n;
      x.e += (size_t)k * n;
      x.tau += (size_t)k * n;
      x.rot += (size_t)k * w.rot_cap;
      x.steps += (size_t)k * w.step_cap;
      x.nsteps += k;
      return x;
    };
    // QL, rotations, back-transformation and sort of matrices m .. m+c-1
    auto chain = [&](int m, int c, const HeevWS &wk, cudaStream_t st) {
      zc *H = HU + (size_t)m * nn;
      zc *Z = V + (size_t)m * nn;
      PW_TIMED(KK_QL, st, k_ql_df<<<c, 32, 2 * (size_t)n * sizeof(df), st>>>(wk, status + m, n));
      PW_TIMED(KK_ROT, st,
               k_rot_apply<<<dim3((n + ROT_ROWS - 1) / ROT_ROWS, c), ROT_ROWS, 0, st>>>(
                   wk, reinterpret_cast<dfc *>(Z), status + m, n));
      PW_TIMED(KK_BACKT, st,
               k_backtransform<<<dim3((n + BT_WARPS * BT_COLS - 1) / (BT_WARPS * BT_COLS), c), BT_WARPS * 32,
                                 bt_smem, st>>>(reinterpret_cast<const dfc *>(H), reinterpret_cast<dfc *>(Z), wk, n));
      PW_TIMED(KK_SORT, st,
               k_eig_sort<<<dim3((n + 7) / 8, c), 256, 0, st>>>(Z, H, En + (size_t)m * n, wk.d, status + m, n));
    };
    // The reduction runs two CTAs per SM.  When a group has more matrices than
    // that, the ones beyond the first full wave go through their own chain on
    // a second stream: the first wave's single-thread QL recurrences (a nearly
    // idle GPU otherwise) overlap the reduction of the rest, and the rest's QL
    // overlaps the first wave's vector kernels.
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int wave = 2 * std::max(sms, 1);
    for (int m0 = 0; m0 < nmat; m0 += group) {
      const int cnt = std::min(group, nmat - m0);
      const int nA = cnt > wave ? wave : cnt;
      cudaStream_t s2 = nullptr;
      cudaEvent_t fork = nullptr, join = nullptr;
      if (nA < cnt && (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();   // no second stream: one chain over the group
        if (s2) cudaStreamDestroy(s2);
        if (fork) cudaEventDestroy(fork);
        s2 = nullptr;
      }
      const int a_cnt = s2 ? nA : cnt;
      if (s2) {
        cudaEventRecord(fork, s);
        cudaStreamWaitEvent(s2, fork, 0);
      }
      PW_TIMED(KK_HEEV, s,
               k_heev<df><<<a_cnt, HEEV_THREADS, smem, s>>>(HU + (size_t)m0 * nn, V + (size_t)m0 * nn,
                                                            En + (size_t)m0 * n, status + m0, n, 1, w, -1));
      if (s2) {
        const int mb = m0 + nA, cb = cnt - nA;
        const HeevWS wb = shifted(nA);
        PW_TIMED(KK_HEEV, s2,
                 k_heev<df><<<cb, HEEV_THREADS, smem, s2>>>(HU + (size_t)mb * nn, V + (size_t)mb * nn,
                                                            En + (size_t)mb * n, status + mb, n, 1, wb, -1));
        chain(mb, cb, wb, s2);
        cudaEventRecord(join, s2);
      }
      chain(m0, a_cnt, w, s);
      if (s2) {
        cudaStreamWaitEvent(s, join, 0);
        cudaEventDestroy(fork);
        cudaEventDestroy(join);
        cudaStreamDestroy(s2);
      }
    }
  } else {
    cudaFuncSetAttribute(k_heev<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    PW_TIMED(tail ? KK_HEEV_TAIL : KK_HEEV, s,
             k_heev<double><<<nmat, HEEV_THREADS, smem, s>>>(HU, V, En, status, n, 0, w, remap_last));
  }
}

// The Jacobi route (same interface), kept as an independent second solver.
void launch_eig_jacobi(zc *HU, zc *V, double *En, int *status, int n, int nmat, cudaStream_t s) {
  const size_t sm64 = jacobi_smem<double>(n);
  cudaFuncSetAttribute(k_jacobi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm64);
  k_jacobi<double><<<nmat, EIG_THREADS, sm64, s>>>(HU, V, (size_t)n * n, n, 1, 40, 1e-12, status,
                                                    En, HU);
}

// ---------------------------------------------------------------------------
// Overlaps O_p = U_p^H U_{p+1}: one CTA per interface.
// ---------------------------------------------------------------------------
// A: the accumulation type (double, or double-float for the mixed form).
// OVL_SPLIT CTAs share one interface's product, striding over its output
// tiles, so that the grid is several waves deep and its last wave small.
constexpr int OVL_SPLIT = 4;
template <typename A>
__global__ void __launch_bounds__(NT) k_overlaps(const zc *U, zc *O, int n, int nq, int g0) {
  extern __shared__ unsigned char smraw[];
  cx<A> *sm = reinterpret_cast<cx<A> *>(smraw);
  const int g = g0 + blockIdx.x / OVL_SPLIT, part = blockIdx.x % OVL_SPLIT;
  const int slot = g / (nq - 1), p = g % (nq - 1);
  const zc *Up = U + ((size_t)slot * nq + p) * n * n;
  const zc *Uq = Up + (size_t)n * n;
  zc *Op = O + ((size_t)slot * (nq - 1) + p) * n * n;
  cta_gemm_t<A, Tile<A, NT>::BM, Tile<A, NT>::BN, Tile<A, NT>::BK, 4, NT>(
      n, n, n, [=](int i, int l) { return acc_of<A>(cconj(Up[l + (size_t)i * n])); },
      [=](int l, int j) { return acc_of<A>(Uq[l + (size_t)j * n]); },
      [=](int i, int j, cx<A> acc) { Op[i + (size_t)j * n] = acc_val(acc); }, sm, part, OVL_SPLIT);
}

// FP32 copies of the overlaps (same column-major layout).
// (with O32lo: the FP32 remainders O - O32, so that O32 + O32lo is O as a
// double-float, 48 bits)
__global__ void __launch_bounds__(NT) k_o32(const zc *O, cc *O32, cc *O32lo, size_t count) {
  for (size_t e = (size_t)blockIdx.x * NT + threadIdx.x; e < count; e += (size_t)gridDim.x * NT) {
    const zc o = O[e];
    const cc h = ccast<float>(o);
    O32[e] = h;
    if (O32lo) O32lo[e] = mkc<float>((float)(o.re - (double)h.re), (float)(o.im - (double)h.im));
  }
}

// FP32 transposed copies (32 x 32 tiles through shared memory, coalesced on
// both sides); grid (tiles, count).
__global__ void __launch_bounds__(NT) k_o32t(const zc *O, cc *Ot, int n) {
  __shared__ cc tile[32][33];
  const size_t nn = (size_t)n * n;
  const zc *src = O + (size_t)blockIdx.y * nn;
  cc *dst = Ot + (size_t)blockIdx.y * nn;
  const int tn = (n + 31) / 32;
  const int i0 = (blockIdx.x % tn) * 32, j0 = (blockIdx.x / tn) * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8
  for (int r = ty; r < 32; r += NT / 32) {
    const int i = i0 + tx, j = j0 + r;
    if (i < n && j < n) tile[r][tx] = ccast<float>(src[i + (size_t)j * n]);   // (i, j) -> tile[j - j0][i - i0]
  }
  __syncthreads();
  for (int r = ty; r < 32; r += NT / 32) {
    const int j = j0 + tx, i = i0 + r;
    if (i < n && j < n) dst[j + (size_t)i * n] = tile[tx][r];   // Ot[j + i n] = O[i + j n]
  }
}

void launch_overlaps_fp32(const zc *O, cc *O32, cc *O32t, cc *O32lo, int n, int count, cudaStream_t s) {
  const size_t nn = (size_t)n * n, total = (size_t)count * nn;
  const size_t blocks = (total + NT - 1) / NT;
  PW_TIMED(KK_O32, s, k_o32<<<(unsigned)(blocks < 4096 ? blocks : 4096), NT, 0, s>>>(O, O32, O32lo, total));
  if (!O32t) return;
  const int tn = (n + 31) / 32;
  for (int c0 = 0; c0 < count; c0 += 65535) {   // grid.y limit
    const int c = count - c0 < 65535 ? count - c0 : 65535;
    PW_TIMED(KK_O32T, s, k_o32t<<<dim3(tn * tn, c), NT, 0, s>>>(O + c0 * nn, O32t + c0 * nn, n));
  }
}

void launch_overlaps(const zc *U, zc *O, int n, int nq, int nslots, cudaStream_t s, bool double_float, int g0,
                     int g1) {
  const size_t smem = gemm_smem_elems<double>() * sizeof(zc);
  const int total = nslots * (nq - 1);
  if (g1 < 0 || g1 > total) g1 = total;
  if (g0 < 0) g0 = 0;
  if (g0 >= g1) return;
  const unsigned grid = (unsigned)(g1 - g0) * OVL_SPLIT;
  if (double_float) PW_TIMED(KK_OVERLAPS, s, k_overlaps<df><<<grid, NT, smem, s>>>(U, O, n, nq, g0));
  else PW_TIMED(KK_OVERLAPS, s, k_overlaps<double><<<grid, NT, smem, s>>>(U, O, n, nq, g0));
}

}  // namespace pw
