// Separable nonlocal terms on the GPU, FP64 (Eqs. kse0, ksep, nloc, gsol_p0,
// calm_0; the M X = D system of Eq. trans, without electrode-crossing
// projectors).  The projectors are Bloch sums of Gaussians,
//     W_alpha(r) = exp(-|r - tau_alpha|^2 / 2 s_alpha^2)  for z_lo <= z <= z_hi,
// whose plane-wave coefficients separate into amp_alpha(G) prof_alpha(z) with
//     amp_alpha(G) = (2 pi s^2 / A) e^{-|k+G|^2 s^2 / 2} e^{-i (k+G).tau_perp},
//     prof_alpha(z) = e^{-(z - tau_z)^2 / 2 s^2} on [z_lo, z_hi], 0 elsewhere.
// In slice p (modes U_p, wavenumbers k) the projector's mode-space values are
// w_alpha(z) = v_alpha prof_alpha(z), v_alpha = U_p^H amp_alpha, and the
// particular solution of f'' + k^2 f = w with the outgoing Green's function
// e^{ik|u|} / 2ik has the edge values
//     fa = v Ia / 2ik,  fb = v Ib / 2ik,
//     Ia = int prof e^{ik(z - z_a)} dz,  Ib = int prof e^{ik(z_b - z)} dz
// over the slice [z_a, z_b].  By linearity the scattering state is
// psi = psi_0 + sum_alpha C_alpha psi_alpha: psi_0 the local state (the
// incident columns of the sweep), psi_alpha the response to the unit source
// of projector alpha with no incident wave.  In mode space the interface
// equations of App. A gain f_p = (Q fa_q - fb_p) C and g_p = P fa_q C, so the
// sweep carries each source as a right-hand-side column that takes
// Y fa_q + fb_p before the interface solve (Y = R P - Q), and the backward
// pass adds P fa_q to b_p.  Eq. calm_0, C = D A sum_p <W|psi>_p, is then an
// m x m system per incident channel:
//     (I - A D (S + P)) C = A D R,
//     S_ba = sum_p HA_b . a_p^(a) + HB_b . b_p^(a),  R_bj the same for psi_0,
//     HA_b = conj(v_b) Ia_b,  HB_b = conj(v_b) Ib_b,
//     P_ba = sum_p sum_modes conj(v_b) v_a J_ba / 2ik,  J_ba = int int prof_b(z) e^{ik|z - z'|} prof_a(z'),
// and t = flux factors x (a_{N+1}^(0) + sum_alpha a_{N+1}^(alpha) C_alpha).
// The z integrals use Gauss-Legendre rules over each slice (the inner
// integral of J split at the outer node, where the Green's function has its
// kink).
#include <math.h>

#include "pw_internal.h"

namespace pw {
namespace {

constexpr int NLT = 256;
constexpr int NL_MAXM = kNlMaxProj;
constexpr int NL_MAXL = kNlMaxOpen;

// e^{i k u} for the branch of kz_branch (|.| <= 1 for u >= 0)
__device__ __forceinline__ zc cexpi(zc k, double u) {
  const double mag = exp(-k.im * u);
  double sn, cs;
  sincos(k.re * u, &sn, &cs);
  return mkc<double>(mag * cs, mag * sn);
}

__device__ __forceinline__ double profile(const double *pr, double z) {
  // pr: tau_z, sigma, z_lo, z_hi
  if (z < pr[2] || z > pr[3]) return 0.0;
  const double u = (z - pr[0]) / pr[1];
  return exp(-0.5 * u * u);
}

__device__ __forceinline__ zc warp_sum(zc v) {
  for (int off = 16; off > 0; off >>= 1) {
    v.re += __shfl_down_sync(0xffffffffu, v.re, off);
    v.im += __shfl_down_sync(0xffffffffu, v.im, off);
  }
  return v;
}

}  // namespace

// V[p-1][alpha][j] = sum_G conj(U_p(G, j)) amp_alpha(G) for the device slices
// p = 1..N of one k-set slot; grid (N, m), one warp per mode (coalesced over G).
// proj: per projector tau_x, tau_y, tau_z, sigma, z_lo, z_hi.
__global__ void __launch_bounds__(NLT) k_nl_project(const zc *U, zc *V, const double *G, double kx, double ky,
                                                    const double *proj, double area, int n, int m) {
  extern __shared__ __align__(16) unsigned char smraw[];
  zc *amp = reinterpret_cast<zc *>(smraw);
  const int p = blockIdx.x + 1, al = blockIdx.y;
  const double *pr = proj + 6 * al;
  const double s = pr[3];
  for (int g = threadIdx.x; g < n; g += NLT) {
    const double qx = kx + G[2 * g], qy = ky + G[2 * g + 1];
    const double mag = (2.0 * M_PI * s * s / area) * exp(-0.5 * (qx * qx + qy * qy) * s * s);
    double sn, cs;
    sincos(qx * pr[0] + qy * pr[1], &sn, &cs);
    amp[g] = mkc<double>(mag * cs, -mag * sn);
  }
  __syncthreads();
  const zc *Up = U + (size_t)p * n * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < n; j += NLT / 32) {
    zc acc = czero<double>();
    for (int g = lane; g < n; g += 32) cfma(acc, cconj(Up[g + (size_t)j * n]), amp[g]);
    acc = warp_sum(acc);
    if (lane == 0) V[((size_t)(p - 1) * m + al) * n + j] = acc;
  }
}

// Per point and device slice: FA, FB, HA, HB (n values per projector) and PP
// (m x m).  grid (N, points); one thread per mode.
__global__ void __launch_bounds__(NLT) k_nl_slice_terms(NonlocalArgs a) {
  __shared__ double red[NL_MAXM * NL_MAXM * 2];
  const int p = blockIdx.x + 1, pt = blockIdx.y;
  const PointDesc d = a.pts[pt];
  const int n = a.n, m = a.m, Q = a.q;
  for (int e = threadIdx.x; e < 2 * m * m; e += NLT) red[e] = 0.0;
  __syncthreads();
  const double za = a.zedge[p - 1], zb = a.zedge[p], h = 0.5 * (zb - za);
  const double *Ep = a.En + ((size_t)d.en_off + p) * n;
  const zc *V = a.V + ((size_t)d.kset * a.ks_N + (p - 1)) * m * n;
  const size_t base = ((size_t)d.x_off + p) * m;
  zc pp[NL_MAXM * NL_MAXM];
  for (int e = 0; e < m * m; ++e) pp[e] = czero<double>();
  for (int j = threadIdx.x; j < n; j += NLT) {
    const zc k = kz_branch(d.E, Ep[j]);
    const zc i2k = cinv(mkc<double>(-2.0 * k.im, 2.0 * k.re));   // 1 / (2ik)
    for (int al = 0; al < m; ++al) {
      const double *pr = a.proj + 6 * al + 2;   // tau_z, sigma, z_lo, z_hi
      zc Ia = czero<double>(), Ib = czero<double>();
      for (int i = 0; i < Q; ++i) {
        const double z = za + h * (a.gl[i] + 1.0), wz = h * a.gl[Q + i] * profile(pr, z);
        const zc ea = cexpi(k, z - za), eb = cexpi(k, zb - z);
        Ia.re += wz * ea.re;
        Ia.im += wz * ea.im;
        Ib.re += wz * eb.re;
        Ib.im += wz * eb.im;
      }
      const zc v = V[(size_t)al * n + j];
      a.FA[(base + al) * n + j] = cmul(cmul(v, Ia), i2k);
      a.FB[(base + al) * n + j] = cmul(cmul(v, Ib), i2k);
      a.HA[(base + al) * n + j] = cmul(cconj(v), Ia);
      a.HB[(base + al) * n + j] = cmul(cconj(v), Ib);
      // F(z_i) = int prof_al(z') e^{ik|z_i - z'|} dz' at the outer nodes, split at z_i;
      // J_b,al = sum_i w_i prof_b(z_i) F(z_i)
      zc J[NL_MAXM];
      for (int b = 0; b < m; ++b) J[b] = czero<double>();
      for (int i = 0; i < Q; ++i) {
        const double zi = za + h * (a.gl[i] + 1.0), wi = h * a.gl[Q + i];
        const double hl = 0.5 * (zi - za), hr = 0.5 * (zb - zi);
        zc F = czero<double>();
        for (int l = 0; l < Q; ++l) {
          const double zl = za + hl * (a.gl[l] + 1.0), wl = hl * a.gl[Q + l] * profile(pr, zl);
          const double zr = zi + hr * (a.gl[l] + 1.0), wr = hr * a.gl[Q + l] * profile(pr, zr);
          const zc el = cexpi(k, zi - zl), er = cexpi(k, zr - zi);
          F.re += wl * el.re + wr * er.re;
          F.im += wl * el.im + wr * er.im;
        }
        for (int b = 0; b < m; ++b) {
          const double pb = wi * profile(a.proj + 6 * b + 2, zi);
          J[b].re += pb * F.re;
          J[b].im += pb * F.im;
        }
      }
      for (int b = 0; b < m; ++b) {
        const zc vb = V[(size_t)b * n + j];
        cfma(pp[b * m + al], cmul(cconj(vb), v), cmul(J[b], i2k));
      }
    }
  }
  // block sums of pp
  const int lane = threadIdx.x & 31;
  for (int e = 0; e < m * m; ++e) {
    const zc v = warp_sum(pp[e]);
    if (lane == 0) {
      atomicAdd(&red[2 * e], v.re);
      atomicAdd(&red[2 * e + 1], v.im);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += NLT)
    a.PP[((size_t)d.x_off + p) * m * m + e] = mkc<double>(red[2 * e], red[2 * e + 1]);
}

// One interface step's source columns: Tacc[:, c0 + alpha] += Y fa_q + fb_p
// (FP64 sweep; Y = R P - Q is the middle block of M); grid (points, m).
__global__ void __launch_bounds__(NLT) k_nl_sources(SweepArgs a, int p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  zc *fa = reinterpret_cast<zc *>(smraw);
  const int pt = blockIdx.x, al = blockIdx.y;
  const PointDesc d = a.pts[pt];
  if (d.skip || a.status[pt] || p > d.N) return;
  const int n = a.n, ncols = 2 * n + a.nc, q = p + 1;
  zc *M = reinterpret_cast<zc *>(a.M) + (size_t)pt * n * ncols;
  const bool have_a = q <= d.N, have_b = p >= 1;   // no particular solutions in the electrodes
  for (int i = threadIdx.x; i < n; i += NLT)
    fa[i] = have_a ? a.nl_fa[(((size_t)d.x_off + q) * a.nl_m + al) * n + i] : czero<double>();
  __syncthreads();
  zc *col = M + (size_t)(2 * n + a.nl_c0 + al) * n;
  for (int i = threadIdx.x; i < n; i += NLT) {
    zc acc = have_b ? a.nl_fb[(((size_t)d.x_off + p) * a.nl_m + al) * n + i] : czero<double>();
    if (have_a)
      for (int l = 0; l < n; ++l) cfma(acc, M[i + (size_t)(n + l) * n], fa[l]);
    col[i] = cadd(col[i], acc);
  }
}

// Eq. calm_0 and t for every point: one CTA per point.
__global__ void __launch_bounds__(NLT) k_nl_solve(NonlocalArgs a) {
  __shared__ double red[2 * NL_MAXM * (NL_MAXM + NL_MAXL)];
  __shared__ zc Mm[NL_MAXM * NL_MAXM], X[NL_MAXM * NL_MAXL];
  __shared__ double tred[NLT / 32];
  __shared__ int sing;
  const int pt = blockIdx.x;
  const PointDesc d = a.pts[pt];
  const int n = a.n, N = d.N, m = a.m, nc = a.nc, nL = d.nL, nR = d.nR;
  if (d.skip || a.status[pt]) {
    if (threadIdx.x == 0) a.T[d.out] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  // columns: incident j < nL, sources c0 + alpha
  const int ncl = nL + m;
  for (int e = threadIdx.x; e < 2 * m * ncl; e += NLT) red[e] = 0.0;
  __syncthreads();
  auto colof = [&](int c) { return c < nL ? c : a.c0 + (c - nL); };
  const int lane = threadIdx.x & 31;
  for (int b = 0; b < m; ++b)
    for (int c = 0; c < ncl; ++c) {
      const int cc_ = colof(c);
      zc acc = czero<double>();
      for (size_t e = threadIdx.x; e < (size_t)N * n; e += NLT) {
        const int p = 1 + (int)(e / n), j = (int)(e % n);
        const size_t sl = (size_t)d.x_off + p;
        const zc ha = a.HA[(sl * m + b) * n + j], hb = a.HB[(sl * m + b) * n + j];
        cfma(acc, ha, a.Xa[sl * n * nc + j + (size_t)cc_ * n]);
        cfma(acc, hb, a.Xb[sl * n * nc + j + (size_t)cc_ * n]);
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        atomicAdd(&red[2 * (b * ncl + c)], acc.re);
        atomicAdd(&red[2 * (b * ncl + c) + 1], acc.im);
      }
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Mm = I - A D (S + sum_p PP),  X = A D R
    zc SP[NL_MAXM * NL_MAXM];
    for (int b = 0; b < m; ++b)
      for (int al = 0; al < m; ++al) {
        zc v = mkc<double>(red[2 * (b * ncl + nL + al)], red[2 * (b * ncl + nL + al) + 1]);
        for (int p = 1; p <= N; ++p) v = cadd(v, a.PP[((size_t)d.x_off + p) * m * m + b * m + al]);
        SP[b * m + al] = v;
      }
    for (int b = 0; b < m; ++b) {
      for (int al = 0; al < m; ++al) {
        zc v = czero<double>();
        for (int g = 0; g < m; ++g) cfma(v, a.D[b * m + g], SP[g * m + al]);
        Mm[b * m + al] = mkc<double>((b == al ? 1.0 : 0.0) - a.area * v.re, -a.area * v.im);
      }
      for (int j = 0; j < nL; ++j) {
        zc v = czero<double>();
        for (int g = 0; g < m; ++g)
          cfma(v, a.D[b * m + g], mkc<double>(red[2 * (g * ncl + j)], red[2 * (g * ncl + j) + 1]));
        X[b * nL + j] = mkc<double>(a.area * v.re, a.area * v.im);
      }
    }
    // Gaussian elimination with partial pivoting (m <= NL_MAXM)
    int bad = 0;
    for (int c = 0; c < m && !bad; ++c) {
      int piv = c;
      for (int r = c + 1; r < m; ++r)
        if (cabs1(Mm[r * m + c]) > cabs1(Mm[piv * m + c])) piv = r;
      if (cabs1(Mm[piv * m + c]) == 0.0) { bad = 1; break; }
      if (piv != c) {
        for (int e = 0; e < m; ++e) { const zc t = Mm[c * m + e]; Mm[c * m + e] = Mm[piv * m + e]; Mm[piv * m + e] = t; }
        for (int e = 0; e < nL; ++e) { const zc t = X[c * nL + e]; X[c * nL + e] = X[piv * nL + e]; X[piv * nL + e] = t; }
      }
      const zc inv = cinv(Mm[c * m + c]);
      for (int r = c + 1; r < m; ++r) {
        const zc f = cmul(Mm[r * m + c], inv);
        for (int e = c; e < m; ++e) Mm[r * m + e] = csub(Mm[r * m + e], cmul(f, Mm[c * m + e]));
        for (int e = 0; e < nL; ++e) X[r * nL + e] = csub(X[r * nL + e], cmul(f, X[c * nL + e]));
      }
    }
    for (int c = m - 1; c >= 0 && !bad; --c) {
      const zc inv = cinv(Mm[c * m + c]);
      for (int e = 0; e < nL; ++e) {
        zc v = X[c * nL + e];
        for (int r = c + 1; r < m; ++r) v = csub(v, cmul(Mm[c * m + r], X[r * nL + e]));
        X[c * nL + e] = cmul(v, inv);
      }
    }
    sing = bad;
    if (a.C && !bad)
      for (int al = 0; al < m; ++al)
        for (int j = 0; j < nL; ++j) a.C[((size_t)d.out * m + al) * n + j] = X[al * nL + j];
  }
  __syncthreads();
  if (sing) {
    if (threadIdx.x == 0) a.T[d.out] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  // t_ij = sqrt(k_i^R / k_j^L) (a^(0)_{N+1} + sum_alpha a^(alpha)_{N+1} C_alpha)_ij on open channels
  const double *EL = a.En + (size_t)d.en_off * n;
  const double *ER = a.En + ((size_t)d.en_off + N + 1) * n;
  const zc *A1 = a.Xa + ((size_t)d.x_off + N + 1) * n * nc;
  double acc = 0.0;
  for (int e = threadIdx.x; e < nR * nL; e += NLT) {
    const int i = e % nR, j = e / nR;
    zc x = A1[i + (size_t)j * n];
    for (int al = 0; al < m; ++al) cfma(x, A1[i + (size_t)(a.c0 + al) * n], X[al * nL + j]);
    const double f = sqrt(d.E - ER[i]) / sqrt(d.E - EL[j]);
    acc += f * (x.re * x.re + x.im * x.im);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) tred[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NLT / 32; ++w) s += tred[w];
    a.T[d.out] = s;
  }
}

cudaError_t launch_nl_project(const zc *U, zc *V, const int *, const double *G, double kx, double ky,
                              const double *proj, double area, int n, int N, int m, cudaStream_t s) {
  if (N < 1 || m < 1) return cudaSuccess;
  k_nl_project<<<dim3(N, m), NLT, (size_t)n * sizeof(zc), s>>>(U, V, G, kx, ky, proj, area, n, m);
  return cudaGetLastError();
}

cudaError_t launch_nl_slice_terms(const NonlocalArgs &a, int npts, cudaStream_t s) {
  if (a.N < 1 || npts < 1) return cudaSuccess;
  k_nl_slice_terms<<<dim3(a.N, npts), NLT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_nl_solve(const NonlocalArgs &a, int npts, cudaStream_t s) {
  if (npts < 1) return cudaSuccess;
  k_nl_solve<<<npts, NLT, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_nl_sources(const SweepArgs &a, int npts, int p, cudaStream_t s) {
  k_nl_sources<<<dim3(npts, a.nl_m), NLT, (size_t)a.n * sizeof(zc), s>>>(a, p);
  return cudaGetLastError();
}

}  // namespace pw
