// Interface scattering matrices (pw_slice_smatrix) and single star products
// (pw_compose), one CTA per point; the algebra of the junction sweep.
//
// Interface p joins slice p (wavenumbers k^p) and slice p+1 (k^{p+1},
// thickness dz_{p+1}, dz = 0 for the right electrode).  With
//   P = (O + K_p^{-1} O K_{p+1}) / 2,  Q = (O - K_p^{-1} O K_{p+1}) / 2,
//   E+ = diag(exp(i k^{p+1} dz_{p+1}))         (|E+| <= 1, never the growing exp),
// App. A Eq. transfer reads I11 = P E-, I12 = Q E+, I21 = Q E-, I22 = P E+ and
// Eq. scatter becomes
//   S11 = E+ P^{-1},  S12 = -E+ P^{-1} Q E+,  S21 = Q P^{-1},  S22 = (P - Q P^{-1} Q) E+.
//
// Sweep (pw_sweep_batched.cu).  The junction's S(0,N+1) is the left-to-right chain of star
// products (Eq. recurrence) S(0,p+1) = S(0,p) * S(p,p+1).  Only two blocks of
// the accumulated product are needed for t: R = S12(0,p) (n x n) and
// Tacc = S11(0,p) restricted to the incident (open left) columns.  Inserting
// the interface blocks above into Eq. recurrence and using
// (I - R S21(p,p+1)) P = P - R Q gives, with W = P - R Q and Y = R P - Q,
//   S11(0,p+1) = E+ W^{-1} Tacc,     S12(0,p+1) = E+ W^{-1} Y E+,
// i.e. one GEMM R [Q | P] and one LU solve W [Z_Y | Z_T] = [Y | Tacc] per
// interface.  The algebra is exact; tests compare against the oracle, which
// forms every S(p,p+1) and applies Eq. recurrence literally.
#include <math.h>

#include "pw_cta.cuh"
#include "pw_internal.h"

namespace pw {

template <typename T>
struct SweepSmem {
  cx<T> *gemm;   // gemm_smem_elems + NB*NB
  cx<T> *kinvL;  // 1 / k^p
  cx<T> *kR;     // k^{p+1}
  cx<T> *ep;     // E+
  T *sval;
  int *sidx;
  int *flag;
};

template <typename T, int NTH = NT>
__device__ SweepSmem<T> carve(unsigned char *raw, int n) {
  SweepSmem<T> s;
  cx<T> *c = reinterpret_cast<cx<T> *>(raw);
  s.gemm = c;
  c += gemm_smem_elems<T, NTH>() + Tile<T, NTH>::NB * Tile<T, NTH>::NB;
  s.kinvL = c;
  c += n;
  s.kR = c;
  c += n;
  s.ep = c;
  c += n;
  s.sval = reinterpret_cast<T *>(c);
  s.sidx = reinterpret_cast<int *>(s.sval + 32);
  s.flag = s.sidx + 32;
  return s;
}

template <typename T, int NTH = NT>
__host__ __device__ size_t carve_bytes(int n) {
  return (gemm_smem_elems<T, NTH>() + Tile<T, NTH>::NB * Tile<T, NTH>::NB + 3 * (size_t)n) *
             sizeof(cx<T>) + 32 * sizeof(T) + 64 * sizeof(int) + 16;
}

// k vectors of the interface p -> smem (computed in FP64, stored in T)
template <typename T>
__device__ void interface_vectors(const double *Ep, const double *Eq, double E, double dz, int n,
                                  SweepSmem<T> &s) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const zc kl = kz_branch(E, Ep[i]);
    const zc kr = kz_branch(E, Eq[i]);
    s.kinvL[i] = ccast<T>(cinv(kl));
    s.kR[i] = ccast<T>(kr);
    s.ep[i] = ccast<T>(phase_fwd(kr, dz));
  }
  __syncthreads();
}

// P_lj (sel = +1) or Q_lj (sel = -1) of the interface from O and the k vectors
template <typename T>
__device__ __forceinline__ cx<T> pq_elem(const zc *O, int n, int l, int j, const SweepSmem<T> &s,
                                         T sel) {
  const cx<T> o = ccast<T>(O[l + (size_t)j * n]);
  const cx<T> r = cmul(s.kR[j], s.kinvL[l]);
  const cx<T> f = mkc<T>(T(0.5) * (T(1) + sel * r.re), T(0.5) * sel * r.im);
  return cmul(o, f);
}

// ---------------------------------------------------------------------------
// Explicit interface S(p,p+1) (Eq. scatter), FP64.  work: n x 3n per CTA.
// CTA b handles point b at interface iface (by_iface = 0), or point 0 at
// interface iface + b (by_iface = 1); its four blocks go to S + b * sstride.
// mixed = 1 writes the mixed element of Eq. recurrence2 instead: the transfer
// blocks I11 = P E-, I12 = Q E+ (Eq. transfer, E- = diag(e^{-ik^{p+1}dz}))
// in place of S11, S12, with S21 and S22 as in Eq. scatter.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_slice_smatrix(const PointDesc *pts, const double *En,
                                                      const zc *Oall, const double *dz, zc *work,
                                                      int *pivall, int *status, zc *S, int n, int N,
                                                      int iface0, int mixed, size_t sstride, int by_iface) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int b = blockIdx.x;
  const int pt = by_iface ? 0 : b, iface = by_iface ? iface0 + b : iface0;
  const PointDesc d = pts[pt];
  const int tid = threadIdx.x;
  SweepSmem<double> s = carve<double>(smraw, n);
  if (tid == 0) *s.flag = 0;
  const double *Ep = En + ((size_t)d.kset * (N + 2) + iface) * n;
  const zc *O = Oall + ((size_t)d.kset * (N + 1) + iface) * n * n;
  zc *M = work + (size_t)b * n * 3 * n;
  int *piv = pivall + (size_t)b * n;
  const double dzq = dz[iface + 1];
  interface_vectors<double>(Ep, Ep + n, d.E, dzq, n, s);
  // [P | I | Q]
  for (size_t e = tid; e < (size_t)n * 3 * n; e += NT) {
    const int i = e % n, j = e / n;
    zc v;
    if (j < n) v = pq_elem<double>(O, n, i, j, s, 1.0);
    else if (j < 2 * n) v = mkc<double>(i == j - n ? 1.0 : 0.0, 0.0);
    else v = pq_elem<double>(O, n, i, j - 2 * n, s, -1.0);
    M[e] = v;
  }
  __syncthreads();
  cta_lu_solve<double>(M, n, n, 3 * n, piv, s.gemm, s.sval, s.sidx, s.flag);
  // X1 = P^{-1} at columns [n, 2n), X2 = P^{-1} Q at [2n, 3n)
  zc *S11 = S + (size_t)b * sstride;
  zc *S12 = S11 + (size_t)n * n;
  zc *S21 = S12 + (size_t)n * n;
  zc *S22 = S21 + (size_t)n * n;
  for (size_t e = tid; e < (size_t)n * n; e += NT) {
    const int i = e % n, j = e / n;
    if (mixed) {
      S11[e] = cmul(pq_elem<double>(O, n, i, j, s, 1.0), phase_fwd(s.kR[j], -dzq));
      S12[e] = cmul(pq_elem<double>(O, n, i, j, s, -1.0), s.ep[j]);
    } else {
      S11[e] = cmul(s.ep[i], M[i + (size_t)(n + j) * n]);
      const zc x2 = cmul(cmul(s.ep[i], M[i + (size_t)(2 * n + j) * n]), s.ep[j]);
      S12[e] = mkc<double>(-x2.re, -x2.im);
    }
  }
  __syncthreads();
  const SweepSmem<double> sc = s;
  // [S21 | S22'] = Q [X1 | X2];  S22 = (P - Q X2) E+
  cta_gemm<double>(
      n, 2 * n, n, [=](int i, int l) { return pq_elem<double>(O, n, i, l, sc, -1.0); },
      [=](int l, int j) { return M[l + (size_t)(n + j) * n]; },
      [=](int i, int j, zc acc) {
        if (j < n) S21[i + (size_t)j * n] = acc;
        else {
          const int c = j - n;
          S22[i + (size_t)c * n] = cmul(csub(pq_elem<double>(O, n, i, c, sc, 1.0), acc), sc.ep[c]);
        }
      },
      s.gemm);
  if (tid == 0 && *s.flag) status[b] = 1;
}

cudaError_t launch_slice_smatrix(const PointDesc *pts, const double *En, const zc *O, const double *dz,
                                 zc *work, int *piv, int *status, zc *S, int n, int N, int iface,
                                 int npts, cudaStream_t st, int mixed, size_t sstride, int by_iface) {
  const size_t smem = carve_bytes<double>(n);
  cudaError_t e = cudaFuncSetAttribute(k_slice_smatrix, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (sstride == 0) sstride = (size_t)4 * n * n;
  k_slice_smatrix<<<npts, NT, smem, st>>>(pts, En, O, dz, work, piv, status, S, n, N, iface, mixed, sstride,
                                          by_iface);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Star product (Eq. recurrence), FP64.  X = I - a12 b21; with
// [Z1 | Z2] = X^{-1} [a11 | a12 b22]:
//   S11 = b11 Z1, S12 = b12 + b11 Z2, S21 = a21 + a22 b21 Z1,
//   S22 = a22 b22 + a22 b21 Z2.
// work per point: n x 4n ([X | Z1 | Z2] then a22 b21).
// ---------------------------------------------------------------------------
// CTA pt combines Sa + pt * Strides.a with Sb + pt * Strides.b into Sab + pt * Strides.c.
__global__ void __launch_bounds__(NT) k_compose(const zc *Sa, const zc *Sb, zc *Sab, zc *work,
                                                int *pivall, int *status, int n, Strides str) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const int tid = threadIdx.x;
  SweepSmem<double> s = carve<double>(smraw, 0);
  if (tid == 0) *s.flag = 0;
  const size_t nn = (size_t)n * n;
  const zc *a11 = Sa + (size_t)pt * str.a, *a12 = a11 + nn, *a21 = a12 + nn, *a22 = a21 + nn;
  const zc *b11 = Sb + (size_t)pt * str.b, *b12 = b11 + nn, *b21 = b12 + nn, *b22 = b21 + nn;
  zc *o11 = Sab + (size_t)pt * str.c, *o12 = o11 + nn, *o21 = o12 + nn, *o22 = o21 + nn;
  zc *M = work + (size_t)pt * 4 * nn;
  zc *Tmp = M + 3 * nn;
  int *piv = pivall + (size_t)pt * n;
  // X = I - a12 b21
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return a12[i + (size_t)l * n]; },
      [=](int l, int j) { return b21[l + (size_t)j * n]; },
      [=](int i, int j, zc acc) { M[i + (size_t)j * n] = csub(mkc<double>(i == j ? 1.0 : 0.0, 0.0), acc); },
      s.gemm);
  // [a11 | a12 b22]
  for (size_t e = tid; e < nn; e += NT) M[nn + e] = a11[e];
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return a12[i + (size_t)l * n]; },
      [=](int l, int j) { return b22[l + (size_t)j * n]; },
      [=](int i, int j, zc acc) { M[2 * nn + i + (size_t)j * n] = acc; }, s.gemm);
  cta_lu_solve<double>(M, n, n, 3 * n, piv, s.gemm, s.sval, s.sidx, s.flag);
  // b11 [Z1 | Z2]
  cta_gemm<double>(
      n, 2 * n, n, [=](int i, int l) { return b11[i + (size_t)l * n]; },
      [=](int l, int j) { return M[nn + l + (size_t)j * n]; },
      [=](int i, int j, zc acc) {
        if (j < n) o11[i + (size_t)j * n] = acc;
        else o12[i + (size_t)(j - n) * n] = cadd(b12[i + (size_t)(j - n) * n], acc);
      },
      s.gemm);
  // Tmp = a22 b21
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return a22[i + (size_t)l * n]; },
      [=](int l, int j) { return b21[l + (size_t)j * n]; },
      [=](int i, int j, zc acc) { Tmp[i + (size_t)j * n] = acc; }, s.gemm);
  // Tmp [Z1 | Z2]
  cta_gemm<double>(
      n, 2 * n, n, [=](int i, int l) { return Tmp[i + (size_t)l * n]; },
      [=](int l, int j) { return M[nn + l + (size_t)j * n]; },
      [=](int i, int j, zc acc) {
        if (j < n) o21[i + (size_t)j * n] = cadd(a21[i + (size_t)j * n], acc);
        else o22[i + (size_t)(j - n) * n] = acc;
      },
      s.gemm);
  // S22 += a22 b22
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return a22[i + (size_t)l * n]; },
      [=](int l, int j) { return b22[l + (size_t)j * n]; },
      [=](int i, int j, zc acc) { o22[i + (size_t)j * n] = cadd(o22[i + (size_t)j * n], acc); },
      s.gemm);
  if (tid == 0 && *s.flag) status[pt] = 1;
}

cudaError_t launch_compose(const zc *Sa, const zc *Sb, zc *Sab, zc *work, int *piv, int *status,
                           int n, int npts, cudaStream_t st, Strides str) {
  const size_t smem = carve_bytes<double>(0);
  cudaError_t e =
      cudaFuncSetAttribute(k_compose, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (!str.a) str = Strides{(size_t)4 * n * n, (size_t)4 * n * n, (size_t)4 * n * n};
  k_compose<<<npts, NT, smem, st>>>(Sa, Sb, Sab, work, piv, status, n, str);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Layer doubling with Eq. recurrence2 (App. A), FP64.  A mixed element holds
// (I11, I12, S21, S22) of a stretch of slices, four n x n column-major blocks
// in that order.  One step, with X = I11(m,n) + I12(m,n) S21(n,k) and the
// element a of (m,n), b of (n,k):
//   I11 = X b11,  I12 = X b12 + a12 b22,  V = a22 b21 X^{-1},
//   S21 = a21 + V,  S22 = a22 b22 - V a12 b22.
// V comes from the LU solve X^T V^T = (a22 b21)^T.  work per CTA: n x 4n
// ([X^T | (a22 b21)^T] solved in place, X, a12 b22).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_compose_mixed(const zc *Ta, const zc *Tb, zc *Tab, zc *work,
                                                      int *pivall, int *status, int n, Strides str) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const int tid = threadIdx.x;
  SweepSmem<double> s = carve<double>(smraw, 0);
  if (tid == 0) *s.flag = 0;
  const size_t nn = (size_t)n * n;
  const zc *a11 = Ta + (size_t)pt * str.a, *a12 = a11 + nn, *a21 = a12 + nn, *a22 = a21 + nn;
  const zc *b11 = Tb + (size_t)pt * str.b, *b12 = b11 + nn, *b21 = b12 + nn, *b22 = b21 + nn;
  zc *o11 = Tab + (size_t)pt * str.c, *o12 = o11 + nn, *o21 = o12 + nn, *o22 = o21 + nn;
  zc *M = work + (size_t)pt * 4 * nn;   // [X^T | V^T] (n x 2n)
  zc *X = M + 2 * nn;
  zc *W = M + 3 * nn;                   // a12 b22
  int *piv = pivall + (size_t)pt * n;
  // X = a11 + a12 b21, kept as is and transposed
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return a12[i + (size_t)l * n]; },
      [=](int l, int j) { return b21[l + (size_t)j * n]; },
      [=](int i, int j, zc acc) {
        const zc x = cadd(a11[i + (size_t)j * n], acc);
        X[i + (size_t)j * n] = x;
        M[j + (size_t)i * n] = x;
      },
      s.gemm);
  // (a22 b21)^T
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return a22[i + (size_t)l * n]; },
      [=](int l, int j) { return b21[l + (size_t)j * n]; },
      [=](int i, int j, zc acc) { M[nn + j + (size_t)i * n] = acc; }, s.gemm);
  // W = a12 b22
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return a12[i + (size_t)l * n]; },
      [=](int l, int j) { return b22[l + (size_t)j * n]; },
      [=](int i, int j, zc acc) { W[i + (size_t)j * n] = acc; }, s.gemm);
  cta_lu_solve<double>(M, n, n, 2 * n, piv, s.gemm, s.sval, s.sidx, s.flag);
  // [I11 | I12] = X [b11 | b12] (+ W)
  cta_gemm<double>(
      n, 2 * n, n, [=](int i, int l) { return X[i + (size_t)l * n]; },
      [=](int l, int j) { return j < n ? b11[l + (size_t)j * n] : b12[l + (size_t)(j - n) * n]; },
      [=](int i, int j, zc acc) {
        if (j < n) o11[i + (size_t)j * n] = acc;
        else o12[i + (size_t)(j - n) * n] = cadd(acc, W[i + (size_t)(j - n) * n]);
      },
      s.gemm);
  // S21 = a21 + V (V(i, j) = M[nn + j + i n])
  for (size_t e = tid; e < nn; e += NT) {
    const int i = e % n, j = e / n;
    o21[e] = cadd(a21[e], M[nn + j + (size_t)i * n]);
  }
  // S22 = a22 b22 - V W
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return a22[i + (size_t)l * n]; },
      [=](int l, int j) { return b22[l + (size_t)j * n]; },
      [=](int i, int j, zc acc) { o22[i + (size_t)j * n] = acc; }, s.gemm);
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return M[nn + l + (size_t)i * n]; },
      [=](int l, int j) { return W[l + (size_t)j * n]; },
      [=](int i, int j, zc acc) { o22[i + (size_t)j * n] = csub(o22[i + (size_t)j * n], acc); }, s.gemm);
  if (tid == 0 && *s.flag) status[pt] = 1;
}

cudaError_t launch_compose_mixed(const zc *Ta, const zc *Tb, zc *Tab, zc *work, int *piv, int *status, int n,
                                 int npairs, cudaStream_t st, Strides str) {
  const size_t smem = carve_bytes<double>(0);
  cudaError_t e =
      cudaFuncSetAttribute(k_compose_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_compose_mixed<<<npairs, NT, smem, st>>>(Ta, Tb, Tab, work, piv, status, n, str);
  return cudaGetLastError();
}

// Eq. scatter on mixed elements, block b at T + b * stride, in place:
// S11 = I11^{-1}, S12 = -I11^{-1} I12 (LU solve I11 [S11 | Z] = [1 | I12]);
// S21, S22 stay.  work per CTA: n x 3n.
__global__ void __launch_bounds__(NT) k_mixed_to_s(zc *T, size_t stride, zc *work, int *pivall, int *status,
                                                   int n) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int b = blockIdx.x, tid = threadIdx.x;
  SweepSmem<double> s = carve<double>(smraw, 0);
  if (tid == 0) *s.flag = 0;
  const size_t nn = (size_t)n * n;
  zc *t11 = T + (size_t)b * stride, *t12 = t11 + nn;
  zc *M = work + (size_t)b * 3 * nn;
  for (size_t e = tid; e < nn; e += NT) {
    const int i = e % n, j = e / n;
    M[e] = t11[e];
    M[nn + e] = mkc<double>(i == j ? 1.0 : 0.0, 0.0);
    M[2 * nn + e] = t12[e];
  }
  __syncthreads();
  cta_lu_solve<double>(M, n, n, 3 * n, pivall + (size_t)b * n, s.gemm, s.sval, s.sidx, s.flag);
  for (size_t e = tid; e < nn; e += NT) {
    t11[e] = M[nn + e];
    const zc z = M[2 * nn + e];
    t12[e] = mkc<double>(-z.re, -z.im);
  }
  if (tid == 0 && *s.flag) status[b] = 1;
}

cudaError_t launch_mixed_to_s(zc *T, size_t stride, zc *work, int *piv, int *status, int n, int nblocks,
                              cudaStream_t st) {
  const size_t smem = carve_bytes<double>(0);
  cudaError_t e = cudaFuncSetAttribute(k_mixed_to_s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_mixed_to_s<<<nblocks, NT, smem, st>>>(T, stride, work, piv, status, n);
  return cudaGetLastError();
}

// The switching measure of Eq. recurrence2: out[b] = the 1-norm (largest
// absolute column sum) of the first block (I11) of T + b * stride.
__global__ void __launch_bounds__(NT) k_i11_norm(const zc *T, size_t stride, int n, double *out) {
  __shared__ double red[NT / 32];
  const zc *t = T + (size_t)blockIdx.x * stride;
  double m = 0.0;
  for (int j = threadIdx.x; j < n; j += NT) {
    double c = 0.0;
    for (int i = 0; i < n; ++i) c += hypot(t[i + (size_t)j * n].re, t[i + (size_t)j * n].im);
    m = fmax(m, c);
  }
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < NT / 32; ++w) r = fmax(r, red[w]);
    out[blockIdx.x] = r;
  }
}

cudaError_t launch_i11_norm(const zc *T, size_t stride, int n, int nblocks, double *out, cudaStream_t st) {
  k_i11_norm<<<nblocks, NT, 0, st>>>(T, stride, n, out);
  return cudaGetLastError();
}

// t and T from S11 of the whole junction (App. C, Sec. II B): with the
// electrodes' eigenvalues ascending, the open channels are the first nL (left)
// and nR (right); t_ij = sqrt(k_i^R / k_j^L) S11_ij, T = sum |t_ij|^2.
__global__ void __launch_bounds__(NT) k_t_from_s(const zc *S11, const double *EnL, const double *EnR, double E,
                                                 int n, int nL, int nR, double *T_out) {
  __shared__ double red[NT / 32];
  double acc = 0.0;
  for (int e = threadIdx.x; e < nL * nR; e += NT) {
    const int i = e % nR, j = e / nR;
    const zc s = S11[i + (size_t)j * n];
    acc += (s.re * s.re + s.im * s.im) * sqrt(E - EnR[i]) / sqrt(E - EnL[j]);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < NT / 32; ++w) r += red[w];
    *T_out = r;
  }
}

cudaError_t launch_t_from_s(const zc *S11, const double *EnL, const double *EnR, double E, int n, int nL, int nR,
                            double *T_out, cudaStream_t st) {
  k_t_from_s<<<1, NT, 0, st>>>(S11, EnL, EnR, E, n, nL, nR, T_out);
  return cudaGetLastError();
}

}  // namespace pw
