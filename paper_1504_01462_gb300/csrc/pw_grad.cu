// Adjoint of the transmission with respect to the device wells' depths
// (pw_grad), FP64.
//
// For the slice ODE c'' = (H(z) - E) c the Wronskian d^T c' - d'^T c of a
// solution c of H and a solution d of the transposed problem H^T is constant
// in z; perturbing H by dH gives, for the scattering state c_j incident from
// the left electrode in channel j and the transposed problem's state d_i
// incident from the right electrode in channel i,
//     int d_i^T dH c_j dz = 2 i k_i^R dt_ij,
// hence with T = sum_ij (k_i^R / k_j^L) |t_ij|^2
//     dT = sum_ij Im(conj(t_ij) int d_i^T dH c_j dz) / k_j^L.
// Inside device slice p both states are sums of the slice's modes,
//     c = U_p (e^{iK(z - z_{p-1})} a_p + e^{-iK(z - z_p)} b_p),
//     d = conj(U_p) (e^{iK(z - z_{p-1})} a'_p + e^{-iK(z - z_p)} b'_p),
// so the z-integral is closed-form:  dT = Im sum_mn (U_p^H dH_p U_p)_mn Gamma_p,mn,
//     Gamma_p = J1 o (A' W A^T + B' W B^T) + J2 o (A' W B^T + B' W A^T),
//     W_ij = conj(t_ij) / k_j^L,  J1_mn = int_0^dz e^{i(k_m+k_n)s} ds,
//     J2_mn = int_0^dz e^{i k_m s} e^{i k_n (dz - s)} ds.
// Summing Gamma_p over the points of one k_par, transforming it once to the
// plane-wave basis (conj(U_p) Gamma_p U_p^T) and folding it onto G - G' gives
// dT/dV0_w = Im sum_p sum_dG dV^p(dG)/dV0_w g_p(dG) in closed form.
//
// The amplitudes a_p, b_p come from the stored sweep (Z_p, u_p) and a backward
// pass; the transposed problem seen from the right electrode is the same
// sweep on the z-mirrored slices with transposed overlaps.
#include <math.h>

#include "pw_cta.cuh"
#include "pw_internal.h"

namespace pw {

namespace {

constexpr int GT = 256;

__device__ __forceinline__ int gslice(const GradArgs &g, int q) { return g.mirror ? g.N + 1 - q : q; }

__device__ __forceinline__ size_t xblk(const GradArgs &g, int pt, int q) {
  return ((size_t)pt * (g.N + 2) + q) * (size_t)g.n * g.nc;
}

}  // namespace

// Backward pass at interface p (p = N .. 0) of a stored FP64 sweep:
//   a_q = Z_p (e_q b_q) + u_p,   b_p = Q_p a_q + P_p e_q b_q   (q = p + 1)
__global__ void __launch_bounds__(GT) k_grad_backward(GradArgs g, int p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const PointDesc d = g.pts[pt];
  if (d.skip || g.status[pt]) return;
  const int n = g.n, nc = g.nc, N = g.N, q = p + 1;
  zc *gsm = reinterpret_cast<zc *>(smraw);
  zc *kinv = gsm + skinny_smem_elems<double>();
  zc *kr = kinv + n;
  zc *er = kr + n;
  const double *Ep = g.En + ((size_t)d.kset * (N + 2) + gslice(g, p)) * n;
  const double *Eq = g.En + ((size_t)d.kset * (N + 2) + gslice(g, q)) * n;
  const double dz = g.dz[gslice(g, q)];
  for (int i = threadIdx.x; i < n; i += GT) {
    const zc kl = kz_branch(d.E, Ep[i]);
    const zc kq = kz_branch(d.E, Eq[i]);
    kinv[i] = cinv(kl);
    kr[i] = kq;
    er[i] = phase_fwd(kq, dz);
  }
  __syncthreads();
  const zc *O = g.O + ((size_t)d.kset * (N + 1) + (g.mirror ? N - p : p)) * n * n;
  const bool tr = g.mirror != 0;
  // the stores of interface p (a point's slot st_off + p: every interface, or
  // the interfaces of the segment being recomputed)
  const zc *Z = g.Zst + (size_t)(d.st_off + p) * n * n;
  const zc *U = g.Ust + (size_t)(d.st_off + p) * n * nc;
  zc *carry = g.carry + (size_t)pt * n * nc;
  zc *tmp = g.tmp + (size_t)pt * 2 * n * nc;
  for (int e = threadIdx.x; e < n * nc; e += GT) {
    const int i = e % n, c = e / n;
    const zc b = (q <= N) ? carry[e] : czero<double>();
    tmp[n + i + (size_t)c * 2 * n] = cmul(er[i], b);
  }
  __syncthreads();
  zc *Xa = g.Xa + xblk(g, pt, q);
  zc *Xb = g.Xb + xblk(g, pt, p);
  cta_gemm_skinny<double>(
      n, nc, n, [=](int i, int l) { return Z[i + (size_t)l * n]; },
      [=](int l, int j) { return tmp[n + l + (size_t)j * 2 * n]; },
      [=](int i, int j, zc acc) {
        const zc a = cadd(acc, U[i + (size_t)j * n]);
        tmp[i + (size_t)j * 2 * n] = a;
        Xa[i + (size_t)j * n] = a;
      },
      gsm);
  // separable nonlocal terms: the source columns' b_p carries P_p fa_q, the
  // particular solution of slice q at its left edge (none in the right electrode)
  if (g.nl_m > 0 && q <= N) {
    __syncthreads();
    for (int e = threadIdx.x; e < n * g.nl_m; e += GT) {
      const int i = e % n, al = e / n;
      zc &x = tmp[n + i + (size_t)(g.nl_c0 + al) * 2 * n];
      x = cadd(x, g.nl_fa[(((size_t)d.x_off + q) * g.nl_m + al) * n + i]);
    }
    __syncthreads();
  }
  auto pq = [=](int l, int j, double sel) {
    const zc o = tr ? O[j + (size_t)l * n] : O[l + (size_t)j * n];
    const zc r = cmul(kr[j], kinv[l]);
    return cmul(o, mkc<double>(0.5 * (1.0 + sel * r.re), 0.5 * sel * r.im));
  };
  cta_gemm_skinny<double>(
      n, nc, 2 * n, [=](int i, int l) { return l < n ? pq(i, l, -1.0) : pq(i, l - n, 1.0); },
      [=](int l, int j) { return tmp[l + (size_t)j * 2 * n]; },
      [=](int i, int j, zc acc) {
        carry[i + (size_t)j * n] = acc;
        Xb[i + (size_t)j * n] = acc;
      },
      gsm);
}

// x = 0 except the incident a_0 (identity on the first nL channels)
__global__ void k_grad_init(GradArgs g) {
  const int pt = blockIdx.x;
  const PointDesc d = g.pts[pt];
  zc *A0 = g.Xa + xblk(g, pt, 0);
  for (int e = threadIdx.x; e < g.n * g.nc; e += blockDim.x) {
    const int i = e % g.n, c = e / g.n;
    A0[e] = mkc<double>((i == c && c < d.nL) ? 1.0 : 0.0, 0.0);
  }
}

// Gamma_p (tile of the n x n eigenbasis matrix) summed over the batch's points
// of k-set `slot`, for the device slices p0 .. p0 + gridDim.y - 1 (a chunk;
// Gam holds one n x n matrix per slice of the chunk); grid (tiles, slices).
__global__ void __launch_bounds__(GT) k_grad_gamma(GammaArgs h, int slot, int p0) {
  const int p = p0 + blockIdx.y;   // device slice p0 .. (1-based)
  const int n = h.n, N = h.N, nc = h.nc;
  const int tiles_i = (n + 15) / 16;
  const int i0 = (blockIdx.x % tiles_i) * 16, j0 = (blockIdx.x / tiles_i) * 16;
  const int ti = threadIdx.x % 16, tj = threadIdx.x / 16;
  const int m = i0 + ti, nn_ = j0 + tj;   // element (m, nn_) of Gamma_p
  __shared__ zc sP1[16][16], sP2[16][16], sA[16][16], sB[16][16];
  __shared__ zc skm[16], skn[16], sem[16], sen[16];
  zc acc = czero<double>();
  const double dz = h.dz[p];
  for (int pt = 0; pt < h.npts; ++pt) {
    const PointDesc d = h.pts[pt];
    if (d.kset != slot || d.skip || h.status[pt] || h.status_m[pt] || d.nL == 0 || d.nR == 0) continue;
    const double w = h.weight ? h.weight[pt] : 1.0;
    const double *Ep = h.En + ((size_t)d.kset * (N + 2) + p) * n;
    const double *EL = h.En + ((size_t)d.kset * (N + 2)) * n;
    __syncthreads();
    if (threadIdx.x < 16) {
      const int r = threadIdx.x;
      if (i0 + r < n) {
        const zc k = kz_branch(d.E, Ep[i0 + r]);
        skm[r] = k;
        sem[r] = phase_fwd(k, dz);
      }
      if (j0 + r < n) {
        const zc k = kz_branch(d.E, Ep[j0 + r]);
        skn[r] = k;
        sen[r] = phase_fwd(k, dz);
      }
    }
    // original amplitudes a_p, b_p (channels j < nL) and the transposed problem's
    // a'_p = b^m_{N+1-p}, b'_p = a^m_{N+1-p} (channels i < nR)
    const zc *A = h.Xa + ((size_t)pt * (N + 2) + p) * (size_t)n * nc;
    const zc *B = h.Xb + ((size_t)pt * (N + 2) + p) * (size_t)n * nc;
    const zc *Am = h.Xb_m + ((size_t)pt * (N + 2) + (N + 1 - p)) * (size_t)n * nc;   // a'
    const zc *Bm = h.Xa_m + ((size_t)pt * (N + 2) + (N + 1 - p)) * (size_t)n * nc;   // b'
    const zc *t = h.Xa + ((size_t)pt * (N + 2) + N + 1) * (size_t)n * nc;            // a_{N+1}
    const int nL = d.nL, nR = d.nR;
    zc part = czero<double>();
    for (int c0 = 0; c0 < nL; c0 += 16) {
      // P1 = A' W, P2 = B' W for rows i0.. and channels c0..c0+15 (W = conj(t)/kL)
      __syncthreads();
      {
        const int r = ti, c = tj;   // sP1[r][c]: row i0+r, left channel c0+c
        zc p1 = czero<double>(), p2 = czero<double>();
        if (i0 + r < n && c0 + c < nL) {
          const double kL = sqrt(d.E - EL[c0 + c]);
          for (int i = 0; i < nR; ++i) {
            const zc tc = cconj(t[i + (size_t)(c0 + c) * n]);
            const zc wv = mkc<double>(tc.re / kL, tc.im / kL);
            cfma(p1, Am[(i0 + r) + (size_t)i * n], wv);
            cfma(p2, Bm[(i0 + r) + (size_t)i * n], wv);
          }
        }
        sP1[r][c] = p1;
        sP2[r][c] = p2;
        // A, B rows j0.. (the column index of Gamma), channels c0..
        const int rr = ti, cc2 = tj;
        sA[rr][cc2] = (j0 + rr < n && c0 + cc2 < nL) ? A[(j0 + rr) + (size_t)(c0 + cc2) * n] : czero<double>();
        sB[rr][cc2] = (j0 + rr < n && c0 + cc2 < nL) ? B[(j0 + rr) + (size_t)(c0 + cc2) * n] : czero<double>();
      }
      __syncthreads();
      if (m < n && nn_ < n) {
        zc s1 = czero<double>(), s2 = czero<double>();
        for (int c = 0; c < 16 && c0 + c < nL; ++c) {
          cfma(s1, sP1[ti][c], sA[tj][c]);
          cfma(s1, sP2[ti][c], sB[tj][c]);
          cfma(s2, sP1[ti][c], sB[tj][c]);
          cfma(s2, sP2[ti][c], sA[tj][c]);
        }
        // J1 = (e_m e_n - 1) / (i (k_m + k_n)),  J2 = (e_m - e_n) / (i (k_m - k_n))
        const zc km = skm[ti], kn = skn[tj], em = sem[ti], en = sen[tj];
        const zc ks = cadd(km, kn), kd = csub(km, kn);
        zc J1, J2;
        if (cabs1(ks) * dz < 1e-8) J1 = mkc<double>(dz, 0.0);
        else J1 = cdiv(csub(cmul(em, en), mkc<double>(1.0, 0.0)), mkc<double>(-ks.im, ks.re));
        if (cabs1(kd) * dz < 1e-8) J2 = cscale(dz, em);
        else J2 = cdiv(csub(em, en), mkc<double>(-kd.im, kd.re));
        cfma(part, s1, J1);
        cfma(part, s2, J2);
      }
    }
    acc.re += w * part.re;
    acc.im += w * part.im;
  }
  if (m < n && nn_ < n) {
    zc &G = h.Gam[(size_t)(p - p0) * n * n + m + (size_t)nn_ * n];
    G = cadd(G, acc);
  }
}

// g_p(dG) += sum over (i, j) with G_i - G_j = dG of (conj(U_p) Gamma_p U_p^T)_ij;
// one CTA per device slice p0 .. p0 + gridDim.x - 1 of k-set `slot` (the
// chunk held in Gam).  T1: n x n scratch per slice of the chunk.
__global__ void __launch_bounds__(GT) k_grad_fold(GammaArgs h, int slot, int p0, const zc *U_all, zc *T1_all,
                                                  const int *mn, int Dm, int Dn) {
  extern __shared__ __align__(16) unsigned char smraw[];
  zc *gsm = reinterpret_cast<zc *>(smraw);
  const int p = p0 + blockIdx.x, n = h.n, N = h.N;
  const size_t nn = (size_t)n * n;
  const zc *U = U_all + ((size_t)slot * (N + 2) + p) * nn;
  const zc *Gm = h.Gam + (size_t)(p - p0) * nn;
  zc *T1 = T1_all + (size_t)(p - p0) * nn;
  zc *gtab = h.gtab + (size_t)(p - 1) * (2 * Dm + 1) * (2 * Dn + 1);
  // T1 = conj(U) Gamma
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return cconj(U[i + (size_t)l * n]); },
      [=](int l, int j) { return Gm[l + (size_t)j * n]; },
      [=](int i, int j, zc acc) { T1[i + (size_t)j * n] = acc; }, gsm);
  // (T1 U^T)_ij folded onto G_i - G_j
  const int tw = 2 * Dn + 1;
  cta_gemm<double>(
      n, n, n, [=](int i, int l) { return T1[i + (size_t)l * n]; },
      [=](int l, int j) { return U[j + (size_t)l * n]; },
      [=](int i, int j, zc acc) {
        const int dm = mn[2 * i] - mn[2 * j] + Dm, dn = mn[2 * i + 1] - mn[2 * j + 1] + Dn;
        double *dst = reinterpret_cast<double *>(gtab + (size_t)dm * tw + dn);
        atomicAdd(dst, acc.re);
        atomicAdd(dst + 1, acc.im);
      },
      gsm);
}

// dT/dV0_w = Im sum_p sum_dG dV^p(dG)/dV0_w g_p(dG); one CTA per device well.
// With `rate` (2 per well) also the derivative for well w moving transversally
// at that rate: its table picks up -i dG.rate, so
// dshift_w = Im sum (-i dG.rate) v0_w dV^p/dV0_w g_p = -sum (dG.rate) Re(v0_w dV g).
__global__ void __launch_bounds__(GT) k_grad_wells(GammaArgs h, WellSet w, const double *z_edges,
                                                   double b1x, double b1y, double b2x, double b2y,
                                                   double area, int Dm, int Dn, double *dV0,
                                                   const double *rate, double *dshift) {
  const int iw = blockIdx.x, N = h.N;
  const int tw = 2 * Dn + 1, tsz = (2 * Dm + 1) * tw;
  const double s = w.sigma[iw], X = w.xyz[3 * iw], Y = w.xyz[3 * iw + 1], Zw = w.xyz[3 * iw + 2];
  const double rx = rate ? rate[2 * iw] : 0.0, ry = rate ? rate[2 * iw + 1] : 0.0;
  const double v0 = w.v0[iw];
  double acc = 0.0, accs = 0.0;
  for (int p = 1; p <= N; ++p) {
    const double zlo = z_edges[p - 1], zhi = z_edges[p];
    const double wz = (s * sqrt(0.5 * M_PI) / (zhi - zlo)) *
                      (erf((zhi - Zw) / (M_SQRT2 * s)) - erf((zlo - Zw) / (M_SQRT2 * s)));
    const zc *gt = h.gtab + (size_t)(p - 1) * tsz;
    for (int e = threadIdx.x; e < tsz; e += GT) {
      const int dm = e / tw - Dm, dn = e % tw - Dn;
      const double gx = dm * b1x + dn * b2x, gy = dm * b1y + dn * b2y;
      const double amp = -2.0 * M_PI * s * s / area * exp(-0.5 * s * s * (gx * gx + gy * gy)) * wz;
      double sn, cs;
      sincos(gx * X + gy * Y, &sn, &cs);
      const zc dv = mkc<double>(amp * cs, -amp * sn);
      const zc gv = gt[e];
      acc += dv.re * gv.im + dv.im * gv.re;   // Im(dv * g)
      accs -= (gx * rx + gy * ry) * v0 * (dv.re * gv.re - dv.im * gv.im);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    acc += __shfl_down_sync(0xffffffffu, acc, off);
    accs += __shfl_down_sync(0xffffffffu, accs, off);
  }
  __shared__ double red[2][GT / 32];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = acc;
    red[1][threadIdx.x >> 5] = accs;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, ts = 0.0;
    for (int i = 0; i < GT / 32; ++i) {
      t += red[0][i];
      ts += red[1][i];
    }
    if (dV0) dV0[iw] = t;
    if (dshift) dshift[iw] = ts;
  }
}

// Electrode-translation term, one CTA per point.  With the two states' values
// and z-derivatives on the contact planes (left: z = 0 from the electrode's
// amplitudes of slice 0; right: z = z_N from those of slice N+1),
//     c = U (a + b),  c' = i U K (a - b),  d = conj(U) (a' + b'),  d' = i conj(U) K (a' - b'),
// an electrode moved by delta contributes X = -/+ i (d^T Gd c' - d'^T Gd c)
// (Gd = diag(G.delta), minus on the left) in place of the slice integral, and
// dT = Im sum_ij W_ij X_ij, W_ij = conj(t_ij) / k_j^L.  out[pt] is that sum
// for the electrodes' rates (rL, rR).  scr: 4 n nc per point.
__global__ void __launch_bounds__(GT) k_grad_leads(GammaArgs h, const zc *U_all, const double *Gv, zc *scr,
                                                   double rLx, double rLy, double rRx, double rRy,
                                                   double *out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const PointDesc d = h.pts[pt];
  const int n = h.n, N = h.N, nc = h.nc;
  if (d.skip || h.status[pt] || h.status_m[pt] || d.nL == 0 || d.nR == 0) {
    if (threadIdx.x == 0) out[pt] = 0.0;
    return;
  }
  zc *ks = reinterpret_cast<zc *>(smraw);
  double *ikL = reinterpret_cast<double *>(ks + n);
  __shared__ double red[GT / 32];
  const int nL = d.nL, nR = d.nR;
  const size_t nn = (size_t)n * n, vec = (size_t)n * nc;
  const double *EL = h.En + ((size_t)d.kset * (N + 2)) * n;
  for (int j = threadIdx.x; j < nL; j += GT) ikL[j] = 1.0 / sqrt(d.E - EL[j]);
  auto amp = [&](const zc *base, int q) { return base + ((size_t)pt * (N + 2) + q) * vec; };
  const zc *t = amp(h.Xa, N + 1);
  zc *C = scr + (size_t)pt * 4 * vec, *Cp = C + vec, *D = Cp + vec, *Dp = D + vec;
  double total = 0.0;
  for (int side = 0; side < 2; ++side) {
    const double rx = side ? rRx : rLx, ry = side ? rRy : rLy;
    if (rx == 0.0 && ry == 0.0) continue;
    const int q = side ? N + 1 : 0;
    const zc *U = U_all + ((size_t)d.kset * (N + 2) + q) * nn;
    const double *Eq = h.En + ((size_t)d.kset * (N + 2) + q) * n;
    const zc *A = amp(h.Xa, q), *B = amp(h.Xb, q);
    const zc *Ap = amp(h.Xb_m, N + 1 - q), *Bp = amp(h.Xa_m, N + 1 - q);   // a', b' of slice q
    __syncthreads();
    for (int m = threadIdx.x; m < n; m += GT) ks[m] = kz_branch(d.E, Eq[m]);
    __syncthreads();
    for (int e = threadIdx.x; e < n * (nL + nR); e += GT) {
      const int g = e % n, col = e / n;
      const bool isc = col < nL;
      const int j = isc ? col : col - nL;
      const zc *X1 = isc ? A : Ap, *X2 = isc ? B : Bp;
      zc v = czero<double>(), dv = czero<double>();
      for (int m = 0; m < n; ++m) {
        const zc u = isc ? U[g + (size_t)m * n] : cconj(U[g + (size_t)m * n]);
        const zc x1 = X1[m + (size_t)j * n], x2 = X2[m + (size_t)j * n];
        cfma(v, u, cadd(x1, x2));
        cfma(dv, u, cmul(ks[m], csub(x1, x2)));
      }
      const zc idv = mkc<double>(-dv.im, dv.re);   // i * dv
      if (isc) {
        C[g + (size_t)j * n] = v;
        Cp[g + (size_t)j * n] = idv;
      } else {
        D[g + (size_t)j * n] = v;
        Dp[g + (size_t)j * n] = idv;
      }
    }
    __syncthreads();
    zc sx = czero<double>(), sy = czero<double>();
    for (int g = threadIdx.x; g < n; g += GT) {
      zc acc = czero<double>();
      for (int j = 0; j < nL; ++j) {
        const zc cp = Cp[g + (size_t)j * n], c = C[g + (size_t)j * n];
        zc wd = czero<double>(), wdp = czero<double>();   // sum_i W_ij d_gi, sum_i W_ij d'_gi
        for (int i = 0; i < nR; ++i) {
          const zc tc = cconj(t[i + (size_t)j * n]);
          const zc wv = mkc<double>(tc.re * ikL[j], tc.im * ikL[j]);
          cfma(wd, wv, D[g + (size_t)i * n]);
          cfma(wdp, wv, Dp[g + (size_t)i * n]);
        }
        cfma(acc, wd, cp);
        acc = csub(acc, cmul(wdp, c));
      }
      sx = cadd(sx, cscale(Gv[2 * g], acc));
      sy = cadd(sy, cscale(Gv[2 * g + 1], acc));
    }
    // Im(-/+ i s) = -/+ Re(s)
    const double sign = side ? 1.0 : -1.0;
    total += sign * (rx * sx.re + ry * sy.re);
  }
  for (int off = 16; off > 0; off >>= 1) total += __shfl_down_sync(0xffffffffu, total, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = total;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < GT / 32; ++i) s += red[i];
    out[pt] = s;
  }
}

cudaError_t launch_grad_backward(const GradArgs &g, int npts, cudaStream_t s, int p_hi, int p_lo, bool init) {
  const size_t smem = skinny_smem_elems<double>() * sizeof(zc) + 3 * (size_t)g.n * sizeof(zc);
  cudaError_t e = cudaFuncSetAttribute(k_grad_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e) return e;
  if (init) {
    const size_t vec = (size_t)npts * g.n * g.nc * sizeof(zc);
    if ((e = cudaMemsetAsync(g.Xa, 0, vec * (g.N + 2), s)) || (e = cudaMemsetAsync(g.Xb, 0, vec * (g.N + 2), s)) ||
        (e = cudaMemsetAsync(g.carry, 0, vec, s)))
      return e;
    k_grad_init<<<npts, GT, 0, s>>>(g);
  }
  for (int p = p_hi; p >= p_lo; --p) k_grad_backward<<<npts, GT, smem, s>>>(g, p);
  return cudaGetLastError();
}

cudaError_t launch_grad_gamma(const GammaArgs &h, int slot, int p0, int cnt, cudaStream_t s) {
  const int tiles = ((h.n + 15) / 16) * ((h.n + 15) / 16);
  k_grad_gamma<<<dim3(tiles, cnt), GT, 0, s>>>(h, slot, p0);
  return cudaGetLastError();
}

cudaError_t launch_grad_fold(const GammaArgs &h, int slot, int p0, int cnt, const zc *U, zc *T1, const int *mn,
                             int Dm, int Dn, cudaStream_t s) {
  const size_t smem = gemm_smem_elems<double>() * sizeof(zc);
  k_grad_fold<<<cnt, GT, smem, s>>>(h, slot, p0, U, T1, mn, Dm, Dn);
  return cudaGetLastError();
}

cudaError_t launch_grad_wells(const GammaArgs &h, const WellSet &w, const double *z_edges, const double *b,
                              double area, int Dm, int Dn, double *dV0, const double *rate, double *dshift,
                              cudaStream_t s) {
  if (w.n <= 0) return cudaSuccess;
  k_grad_wells<<<w.n, GT, 0, s>>>(h, w, z_edges, b[0], b[1], b[2], b[3], area, Dm, Dn, dV0, rate, dshift);
  return cudaGetLastError();
}

cudaError_t launch_grad_leads(const GammaArgs &h, const zc *U_all, const double *G, zc *scr,
                              const double rate[2][2], double *out, cudaStream_t s) {
  const size_t smem = (size_t)h.n * (sizeof(zc) + sizeof(double));
  k_grad_leads<<<h.npts, GT, smem, s>>>(h, U_all, G, scr, rate[0][0], rate[0][1], rate[1][0], rate[1][1], out);
  return cudaGetLastError();
}

}  // namespace pw
