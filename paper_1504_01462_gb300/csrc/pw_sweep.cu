// The E-dependent hot path: interface scattering matrices and their star
// products, one CTA per (E, k_par) point.
//
// Interface p joins slice p (wavenumbers k^p) and slice p+1 (k^{p+1},
// thickness dz_{p+1}, dz = 0 for the right electrode).  With
//   P = (O + K_p^{-1} O K_{p+1}) / 2,  Q = (O - K_p^{-1} O K_{p+1}) / 2,
//   E+ = diag(exp(i k^{p+1} dz_{p+1}))         (|E+| <= 1, never the growing exp),
// App. A Eq. transfer reads I11 = P E-, I12 = Q E+, I21 = Q E-, I22 = P E+ and
// Eq. scatter becomes
//   S11 = E+ P^{-1},  S12 = -E+ P^{-1} Q E+,  S21 = Q P^{-1},  S22 = (P - Q P^{-1} Q) E+.
//
// Sweep (k_sweep).  The junction's S(0,N+1) is the left-to-right chain of star
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
template <typename T, int NTH>
__global__ void __launch_bounds__(NTH) k_sweep(SweepArgs a, int p) {
  constexpr int NT = NTH;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const PointDesc d = a.pts[pt];
  const int n = a.n, N = a.N, nc = a.nc;
  const int ncols = 2 * n + nc;
  const int tid = threadIdx.x;
  if (d.skip) {
    if (p == N && tid == 0) {
      a.T[d.out] = __longlong_as_double(0x7ff8000000000000ll);
      if (a.nopen) { a.nopen[2 * d.out] = d.nL; a.nopen[2 * d.out + 1] = d.nR; }
      if (a.err) a.err[d.out] = 0.0;
    }
    return;
  }
  if (a.status[pt] != 0) {
    if (p == N && tid == 0) {
      a.T[d.out] = __longlong_as_double(0x7ff8000000000000ll);
      if (a.nopen) { a.nopen[2 * d.out] = d.nL; a.nopen[2 * d.out + 1] = d.nR; }
    }
    return;
  }
  SweepSmem<T> s = carve<T, NTH>(smraw, n);
  if (tid == 0) *s.flag = 0;
  const double *Ep = a.En + ((size_t)d.kset * (N + 2) + p) * n;
  const double *Eq = Ep + n;
  const zc *O = a.O + ((size_t)d.kset * (N + 1) + p) * n * n;
  cx<T> *R = reinterpret_cast<cx<T> *>(a.R) + (size_t)pt * n * n;
  cx<T> *M = reinterpret_cast<cx<T> *>(a.M) + (size_t)pt * n * ncols;
  int *piv = a.piv + (size_t)pt * n;
  interface_vectors<T>(Ep, Eq, d.E, a.dz[p + 1], n, s);

  if (p == 0) {
    // S(0,0) = I: R = 0, Tacc = the open left columns of I  ->  W = P, Y = -Q
    for (size_t e = tid; e < (size_t)n * ncols; e += NT) {
      const int i = e % n, j = e / n;
      cx<T> v;
      if (j < n) v = pq_elem<T>(O, n, i, j, s, T(1));
      else if (j < 2 * n) { v = pq_elem<T>(O, n, i, j - n, s, T(-1)); v.re = -v.re; v.im = -v.im; }
      else { const int c = j - 2 * n; v = mkc<T>((i == c && c < d.nL) ? T(1) : T(0), T(0)); }
      M[e] = v;
    }
    __syncthreads();
  } else {
    // [W | Y] = [P | -Q] + [-R Q | R P]
    const SweepSmem<T> sc = s;
    cta_gemm<T, NTH>(
        n, 2 * n, n, [=](int i, int l) { return R[i + (size_t)l * n]; },
        [=](int l, int j) {
          return j < n ? pq_elem<T>(O, n, l, j, sc, T(-1)) : pq_elem<T>(O, n, l, j - n, sc, T(1));
        },
        [=](int i, int j, cx<T> acc) {
          if (j < n) M[i + (size_t)j * n] = csub(pq_elem<T>(O, n, i, j, sc, T(1)), acc);
          else M[i + (size_t)j * n] = csub(acc, pq_elem<T>(O, n, i, j - n, sc, T(-1)));
        },
        s.gemm);
  }
  // W [Z_Y | Z_T] = [Y | Tacc]
  cta_lu_solve<T, NTH>(M, n, n, ncols, piv, s.gemm, s.sval, s.sidx, s.flag);
  // keep Z_Y, u = Z_T and the LU factors of W for the refinement passes
  if (a.Zst) {
    cx<T> *Zs = reinterpret_cast<cx<T> *>(a.Zst) + ((size_t)pt * (N + 1) + p) * n * n;
    cx<T> *Us = reinterpret_cast<cx<T> *>(a.Ust) + ((size_t)pt * (N + 1) + p) * n * nc;
    cx<T> *Ls = reinterpret_cast<cx<T> *>(a.LUst) + ((size_t)pt * (N + 1) + p) * n * n;
    int *Ps = a.PIVst + ((size_t)pt * (N + 1) + p) * n;
    for (size_t e = tid; e < (size_t)n * n; e += NT) {
      Zs[e] = M[(size_t)n * n + e];
      Ls[e] = M[e];
    }
    for (size_t e = tid; e < (size_t)n * nc; e += NT) Us[e] = M[(size_t)2 * n * n + e];
    for (int e = tid; e < n; e += NT) Ps[e] = piv[e];
  }
  // R <- E+ Z_Y E+,  Tacc <- E+ Z_T
  for (size_t e = tid; e < (size_t)n * n; e += NT) {
    const int i = e % n, j = e / n;
    R[e] = cmul(cmul(s.ep[i], M[i + (size_t)(n + j) * n]), s.ep[j]);
  }
  for (size_t e = tid; e < (size_t)n * nc; e += NT) {
    const int i = e % n, c = e / n;
    cx<T> &v = M[i + (size_t)(2 * n + c) * n];
    v = cmul(s.ep[i], v);
  }
  __syncthreads();
  if (tid == 0 && *s.flag) a.status[pt] = 1;
  if (p < N) return;

  // ---- t_ij = sqrt(k_i^R / k_j^L) S11_ij on open channels, T = sum |t_ij|^2
  const double *EL = a.En + ((size_t)d.kset * (N + 2)) * n;
  const double *ER = EL + (size_t)(N + 1) * n;
  double acc = 0.0;
  for (int e = tid; e < d.nR * d.nL; e += NT) {
    const int i = e % d.nR, j = e / d.nR;
    const double f = sqrt(sqrt(d.E - ER[i]) / sqrt(d.E - EL[j]));
    const cx<T> v = M[i + (size_t)(2 * n + j) * n];
    const zc tv = mkc<double>(f * double(v.re), f * double(v.im));
    acc += tv.re * tv.re + tv.im * tv.im;
    if (a.t) a.t[(size_t)d.out * n * n + i + (size_t)j * n] = tv;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  __shared__ double red[NT / 32];
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double tsum = 0.0;
    for (int w = 0; w < NT / 32; ++w) tsum += red[w];
    a.T[d.out] = (*s.flag || a.status[pt]) ? __longlong_as_double(0x7ff8000000000000ll) : tsum;
    if (a.nopen) { a.nopen[2 * d.out] = d.nL; a.nopen[2 * d.out + 1] = d.nR; }
    if (a.err) a.err[d.out] = 0.0;
  }
}

// The FP64 sweep is bound by the FP64 pipe at 256 threads per point; the FP32
// sweep is latency-bound and runs 512 threads (16 warps) per point.
constexpr int SWEEP_NT64 = 256, SWEEP_NT32 = 512;

size_t sweep_smem_bytes(int n, int precision) {
  return precision == PW_FP64 ? carve_bytes<double, SWEEP_NT64>(n) : carve_bytes<float, SWEEP_NT32>(n);
}

cudaError_t launch_sweep(const SweepArgs &a, int npts, int p, int precision, cudaStream_t s) {
  const size_t smem = sweep_smem_bytes(a.n, precision);
  cudaError_t e;
  if (precision == PW_FP64) {
    e = cudaFuncSetAttribute(k_sweep<double, SWEEP_NT64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_sweep<double, SWEEP_NT64><<<npts, SWEEP_NT64, smem, s>>>(a, p);
  } else {
    e = cudaFuncSetAttribute(k_sweep<float, SWEEP_NT32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_sweep<float, SWEEP_NT32><<<npts, SWEEP_NT32, smem, s>>>(a, p);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Explicit interface S(p,p+1) (Eq. scatter), FP64.  work: n x 3n per point.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_slice_smatrix(const PointDesc *pts, const double *En,
                                                      const zc *Oall, const double *dz, zc *work,
                                                      int *pivall, int *status, zc *S, int n, int N,
                                                      int iface) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const PointDesc d = pts[pt];
  const int tid = threadIdx.x;
  SweepSmem<double> s = carve<double>(smraw, n);
  if (tid == 0) *s.flag = 0;
  const double *Ep = En + ((size_t)d.kset * (N + 2) + iface) * n;
  const zc *O = Oall + ((size_t)d.kset * (N + 1) + iface) * n * n;
  zc *M = work + (size_t)pt * n * 3 * n;
  int *piv = pivall + (size_t)pt * n;
  interface_vectors<double>(Ep, Ep + n, d.E, dz[iface + 1], n, s);
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
  zc *S11 = S + (size_t)pt * 4 * n * n;
  zc *S12 = S11 + (size_t)n * n;
  zc *S21 = S12 + (size_t)n * n;
  zc *S22 = S21 + (size_t)n * n;
  for (size_t e = tid; e < (size_t)n * n; e += NT) {
    const int i = e % n, j = e / n;
    S11[e] = cmul(s.ep[i], M[i + (size_t)(n + j) * n]);
    const zc x2 = cmul(cmul(s.ep[i], M[i + (size_t)(2 * n + j) * n]), s.ep[j]);
    S12[e] = mkc<double>(-x2.re, -x2.im);
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
  if (tid == 0 && *s.flag) status[pt] = 1;
}

cudaError_t launch_slice_smatrix(const PointDesc *pts, const double *En, const zc *O, const double *dz,
                                 zc *work, int *piv, int *status, zc *S, int n, int N, int iface,
                                 int npts, cudaStream_t st) {
  const size_t smem = carve_bytes<double>(n);
  cudaError_t e = cudaFuncSetAttribute(k_slice_smatrix, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_slice_smatrix<<<npts, NT, smem, st>>>(pts, En, O, dz, work, piv, status, S, n, N, iface);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Star product (Eq. recurrence), FP64.  X = I - a12 b21; with
// [Z1 | Z2] = X^{-1} [a11 | a12 b22]:
//   S11 = b11 Z1, S12 = b12 + b11 Z2, S21 = a21 + a22 b21 Z1,
//   S22 = a22 b22 + a22 b21 Z2.
// work per point: n x 4n ([X | Z1 | Z2] then a22 b21).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_compose(const zc *Sa, const zc *Sb, zc *Sab, zc *work,
                                                int *pivall, int *status, int n) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const int tid = threadIdx.x;
  SweepSmem<double> s = carve<double>(smraw, 0);
  if (tid == 0) *s.flag = 0;
  const size_t nn = (size_t)n * n;
  const zc *a11 = Sa + (size_t)pt * 4 * nn, *a12 = a11 + nn, *a21 = a12 + nn, *a22 = a21 + nn;
  const zc *b11 = Sb + (size_t)pt * 4 * nn, *b12 = b11 + nn, *b21 = b12 + nn, *b22 = b21 + nn;
  zc *o11 = Sab + (size_t)pt * 4 * nn, *o12 = o11 + nn, *o21 = o12 + nn, *o22 = o21 + nn;
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
                           int n, int npts, cudaStream_t st) {
  const size_t smem = carve_bytes<double>(0);
  cudaError_t e =
      cudaFuncSetAttribute(k_compose, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_compose<<<npts, NT, smem, st>>>(Sa, Sb, Sab, work, piv, status, n);
  return cudaGetLastError();
}

}  // namespace pw
