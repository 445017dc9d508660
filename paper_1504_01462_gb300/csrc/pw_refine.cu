// Mixed-precision form: FP64 iterative refinement of the whole junction
// system around the FP32 star-product sweep.
//
// Unknowns per point: the amplitudes a_q (forward waves, referenced at the
// left edge of slice q) and b_q (backward waves, referenced at its right edge)
// of every slice q = 0..N+1, with a_0 = the incident open channels and
// b_{N+1} = 0 fixed.  App. A Eq. transfer, written with E+ factors only,
// gives at every interface p (slices p | q = p+1)
//     F_p:  e_p a_p - P_p a_q - Q_p e_q b_q = f_p
//     B_p:  b_p     - Q_p a_q - P_p e_q b_q = g_p          (f = g = 0),
// e_q = exp(i k^q dz_q).  The forward sweep is block elimination of this
// system: with e_p a_p = R_p b_p + c_p,
//     a_q = Z_p e_q b_q + u_p,  Z_p = W_p^{-1} (R_p P - Q),
//     u_p = W_p^{-1} (c_p + R_p g_p - f_p),  W_p = P - R_p Q,
//     R_q = e_q Z_p e_q,  c_q = e_q u_p,
// and a backward pass recovers every amplitude:
//     a_q = Z_p e_q b_q + u_p,   b_p = Q_p a_q + P_p e_q b_q + g_p.
// Refinement: x <- x + M^{-1} (d - L x) with the residual d - L x evaluated in
// FP64 from FP64 overlaps and wavenumbers, and M^{-1} the FP32 sweep (Z_p and
// the LU factors of W_p kept from the first sweep, R_p = e_p Z_{p-1} e_p).
#include <math.h>

#include <algorithm>
#include <vector>

#include "pw_cta.cuh"
#include "pw_df.cuh"
#include "pw_internal.h"
#include "pw_tc.cuh"

namespace pw {

namespace {

struct KV {   // per-interface vectors, FP64, in shared memory (the residual)
  zc *kinvL, *kR, *eL, *eR;
};

__device__ KV carve_kv(unsigned char *raw, size_t off, int n) {
  KV v;
  zc *c = reinterpret_cast<zc *>(raw + off);
  v.kinvL = c;
  v.kR = c + n;
  v.eL = c + 2 * n;
  v.eR = c + 3 * n;
  return v;
}

__device__ void load_kv(const RefineArgs &a, const PointDesc &d, int p, KV &v) {
  const int n = a.n;
  const double *Ep = a.En + ((size_t)d.en_off + p) * n;
  const double *Eq = Ep + n;
  const double *dz = a.dz + d.dz_off;
  for (int i = threadIdx.x; i < n; i += NT) {
    const zc kl = kz_branch(d.E, Ep[i]);
    const zc kr = kz_branch(d.E, Eq[i]);
    v.kinvL[i] = cinv(kl);
    v.kR[i] = kr;
    v.eL[i] = phase_fwd(kl, dz[p]);
    v.eR[i] = phase_fwd(kr, dz[p + 1]);
  }
  __syncthreads();
}

__device__ __forceinline__ size_t blk(const RefineArgs &a, const PointDesc &d, int q) {
  return ((size_t)d.x_off + q) * (size_t)a.n * a.nc;
}
__device__ __forceinline__ size_t iblk(const RefineArgs &a, const PointDesc &d, int p) {
  return ((size_t)d.st_off + p) * (size_t)a.n * a.nc;
}
__device__ __forceinline__ const zc *overlap(const RefineArgs &a, const PointDesc &d, int p) {
  return a.O + ((size_t)d.o_off + p) * (size_t)a.n * a.n;
}

}  // namespace

// ---------------------------------------------------------------------------
// x = 0 except the incident a_0 (identity on the open left channels)
__global__ void k_refine_init(RefineArgs a) {
  const int pt = blockIdx.x;
  const PointDesc d = a.pts[pt];
  zc *A0 = a.Xa + blk(a, d, 0);
  for (int e = threadIdx.x; e < a.n * a.nc; e += blockDim.x) {
    const int i = e % a.n, c = e / a.n;
    A0[e] = mkc<double>((i == c && c < d.nL) ? 1.0 : 0.0, 0.0);
  }
}

// ---------------------------------------------------------------------------
// The FP32 preconditioner passes, several CTAs per point (row blocks of
// SKINNY_BM rows): grid (row blocks, points).
//   backward (p = N .. 0):  da_q = Z_p (e_q db_q) + u_p,  db_p = Q_p da_q + P_p e_q db_q (+ g_p),
//                           accumulated into Xa[q], Xb[p]; db_p is carried to interface p-1;
//   forward  (p = 0 .. N):  u_p = W_p^{-1} (c_p + R_p g_p - f_p),  R_p = e_p Z_{p-1} e_p,
//                           c_{p+1} = e_q u_p, with W_p's LU factors kept by the first sweep
//                           (an O(n^2 n_c) replay); u_p replaces the stored one for the next
//                           backward pass, and at p = N the carry is the correction of a_{N+1}.
namespace {

// 1/k^p, k^{p+1}, e^{i k^p dz_p}, e^{i k^{p+1} dz_{p+1}} in FP32 (null = not needed);
// E - E_n is formed in FP64 before the FP32 root, so thresholds keep their branch.
__device__ void load_kv32(const RefineArgs &a, const PointDesc &d, int p, cc *kinvL, cc *kR, cc *eL, cc *eR) {
  const int n = a.n;
  const double *Ep = a.En + ((size_t)d.en_off + p) * n;
  const double *Eq = Ep + n;
  const float dzl = (float)a.dz[d.dz_off + p], dzr = (float)a.dz[d.dz_off + p + 1];
  auto kz32 = [](double diff) {
    const float m = sqrtf((float)fabs(diff));
    return diff > 0.0 ? mkc<float>(m, 0.f) : mkc<float>(0.f, m);
  };
  auto ph32 = [](cc k, float dz) {
    const float mag = expf(-k.im * dz);
    float sn, cs;
    sincosf(k.re * dz, &sn, &cs);
    return mkc<float>(mag * cs, mag * sn);
  };
  for (int i = threadIdx.x; i < n; i += NT) {
    const cc kl = kz32(d.E - Ep[i]), kr = kz32(d.E - Eq[i]);
    if (kinvL) kinvL[i] = cinv(kl);
    if (kR) kR[i] = kr;
    if (eL) eL[i] = ph32(kl, dzl);
    if (eR) eR[i] = ph32(kr, dzr);
  }
  __syncthreads();
}

__device__ __forceinline__ bool refine_skip(const RefineArgs &a, const PointDesc &d, int pt, int p) {
  return d.skip || a.status[pt] || p > d.N;
}

}  // namespace

// Backward pass, part 1 at interface p (rows i0 .. i0+SKINNY_BM of this CTA):
//   da_q = Z_p (e_q db_q) + u_p  -> tmp[0:n] (rows), Xa[q];  e_q db_q -> tmp[n:2n] (rows)
__global__ void __launch_bounds__(NT) k_refine_bwd_a(RefineArgs a, int p, int with_src) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.y, i0 = blockIdx.x * SKINNY_BM;
  const PointDesc d = a.pts[pt];
  if (refine_skip(a, d, pt, p) || i0 >= a.n) return;
  const int n = a.n, nc = a.nc, N = d.N, q = p + 1;
  const int rows = min(SKINNY_BM, n - i0);
  cc *gsm = reinterpret_cast<cc *>(smraw);
  cc *eR = gsm + skinny_smem_elems<float>();
  cc *kR = eR + n;
  load_kv32(a, d, p, nullptr, a.Bw ? kR : nullptr, nullptr, eR);
  const zc *carry = a.carry + (size_t)pt * n * nc;   // db_q (db_{N+1} = 0)
  const bool has_b = q <= N;
  auto edb = [=](int l, int j) {
    return has_b ? cmul(eR[l], ccast<float>(carry[l + (size_t)j * n])) : czero<float>();
  };
  const cc *Z = a.Zst + ((size_t)d.st_off + p) * n * n;
  const cc *U = a.Ust + ((size_t)d.st_off + p) * n * nc;
  cc *tmp = a.tmp + (size_t)pt * 2 * n * nc;         // [da_q ; e_q db_q] as a 2n x nc block
  for (int e = threadIdx.x; e < rows * nc; e += NT) {
    const int i = i0 + e % rows, c = e / rows;
    tmp[n + i + (size_t)c * 2 * n] = edb(i, c);
  }
  zc *Xa = a.Xa + blk(a, d, q);
  const bool add = q <= N || !with_src;   // a correction of a_{N+1} was added by the forward pass
  cta_gemm_skinny<float>(
      rows, nc, n, [=](int i, int l) { return Z[i0 + i + (size_t)l * n]; },
      [=](int l, int j) { return edb(l, j); },
      [=](int i, int j, cc acc) {
        const cc da = cadd(acc, U[i0 + i + (size_t)j * n]);
        tmp[i0 + i + (size_t)j * 2 * n] = da;
        if (add) {
          zc &x = Xa[i0 + i + (size_t)j * n];
          x = cadd(x, ccast<double>(da));
        }
        if (a.Bw) {
          // operands of the batched backward product (k_refine_bwd_mm):
          // u = da + e db, w = K_q (e db - da)
          const cc e = tmp[n + i0 + i + (size_t)j * 2 * n];
          cc *Bw = a.Bw + (size_t)pt * 2 * nc * n;
          Bw[i0 + i + (size_t)j * n] = cadd(da, e);
          Bw[i0 + i + (size_t)(nc + j) * n] = cmul(kR[i0 + i], csub(e, da));
        }
      },
      gsm);
}

// Backward pass, part 2 when every point shares its overlaps: with
// Q = (O - K_p^{-1} O K_q)/2 and P = (O + K_p^{-1} O K_q)/2,
//   db_p = Q da_q + P e db_q = (O u + K_p^{-1} O w)/2,  u = da + e db, w = K_q (e db - da),
// so one product O [u_1 w_1 u_2 w_2 ...] on the tensor cores (TF32 hi/lo split,
// FP32 level like the rest of the preconditioner) serves every point;
// k_refine_bwd_c combines it.  Grid (64 x 128 tiles of n x 2 nc npts).
__global__ void __launch_bounds__(tc::CG_THREADS) k_refine_bwd_mm(RefineArgs a, int p, int npts) {
  extern __shared__ __align__(128) unsigned char smtc[];
  unsigned char *smraw = smtc;
  const int n = a.n, ncol = 2 * a.nc * npts;
  const int tiles_m = (n + tc::CG_M / 2 - 1) / (tc::CG_M / 2);
  const int r0 = (blockIdx.x % tiles_m) * (tc::CG_M / 2), c0 = (blockIdx.x / tiles_m) * tc::CG_N;
  const cc *O = a.O32 + ((size_t)a.pts[0].o_off + p) * n * n;
  const cc *B = a.Bw;
  cc *Y = a.Yw;
  const bool ok = tc::cgemm_tile<true, false>(
      n, ncol, n, r0, c0, [=](int i, int l) { return O[i + (size_t)l * n]; },
      [=](int l, int j) { return B[l + (size_t)j * n]; }, [=](int, int) { return czero<float>(); },
      [=](int i, int j, cc acc, cc) { Y[i + (size_t)j * n] = acc; }, smraw);
  if (!ok && threadIdx.x == 0)
    for (int pt = 0; pt < npts; ++pt) a.status[pt] = 2;
}

__global__ void __launch_bounds__(NT) k_refine_bwd_c(RefineArgs a, int p, int with_src) {
  __shared__ cc kinvL[1024];
  const int pt = blockIdx.y, i0 = blockIdx.x * SKINNY_BM;
  const PointDesc d = a.pts[pt];
  if (refine_skip(a, d, pt, p) || i0 >= a.n) return;
  const int n = a.n, nc = a.nc;
  const int rows = min(SKINNY_BM, n - i0);
  load_kv32(a, d, p, kinvL, nullptr, nullptr, nullptr);
  const cc *Y = a.Yw + (size_t)pt * 2 * nc * n;
  zc *carry = a.carry + (size_t)pt * n * nc;
  zc *Xb = a.Xb + blk(a, d, p);
  const zc *G = a.Gr + iblk(a, d, p);
  for (int e = threadIdx.x; e < rows * nc; e += NT) {
    const int i = i0 + e % rows, c = e / rows;
    const cc y1 = Y[i + (size_t)c * n], y2 = cmul(kinvL[i], Y[i + (size_t)(nc + c) * n]);
    zc db = mkc<double>(0.5 * ((double)y1.re + (double)y2.re), 0.5 * ((double)y1.im + (double)y2.im));
    if (with_src) db = cadd(db, G[i + (size_t)c * n]);
    carry[i + (size_t)c * n] = db;
    zc &x = Xb[i + (size_t)c * n];
    x = cadd(x, db);
  }
}

// Backward pass, part 2: db_p = [Q | P] [da_q ; e_q db_q] (+ g_p) for this CTA's
// rows -> carry (db_p, carried to interface p-1), Xb[p].
__global__ void __launch_bounds__(NT) k_refine_bwd_b(RefineArgs a, int p, int with_src) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.y, i0 = blockIdx.x * SKINNY_BM;
  const PointDesc d = a.pts[pt];
  if (refine_skip(a, d, pt, p) || i0 >= a.n) return;
  const int n = a.n, nc = a.nc;
  const int rows = min(SKINNY_BM, n - i0);
  cc *gsm = reinterpret_cast<cc *>(smraw);
  cc *kinvL = gsm + skinny_smem_elems<float>();
  cc *kR = kinvL + n;
  load_kv32(a, d, p, kinvL, kR, nullptr, nullptr);
  const cc *O32 = a.O32 ? a.O32 + ((size_t)d.o_off + p) * (size_t)n * n : nullptr;
  const zc *O = overlap(a, d, p);
  const cc *tmp = a.tmp + (size_t)pt * 2 * n * nc;
  zc *carry = a.carry + (size_t)pt * n * nc;
  zc *Xb = a.Xb + blk(a, d, p);
  const zc *G = a.Gr + iblk(a, d, p);
  auto pq = [=](int l, int j, float sel) {
    const cc o = O32 ? O32[l + (size_t)j * n] : ccast<float>(O[l + (size_t)j * n]);
    const cc r = cmul(kR[j], kinvL[l]);
    return cmul(o, mkc<float>(0.5f * (1.0f + sel * r.re), 0.5f * sel * r.im));
  };
  cta_gemm_skinny<float>(
      rows, nc, 2 * n,
      [=](int i, int l) { return l < n ? pq(i0 + i, l, -1.0f) : pq(i0 + i, l - n, 1.0f); },
      [=](int l, int j) { return tmp[l + (size_t)j * 2 * n]; },
      [=](int i, int j, cc acc) {
        zc db = ccast<double>(acc);
        if (with_src) db = cadd(db, G[i0 + i + (size_t)j * n]);
        carry[i0 + i + (size_t)j * n] = db;
        zc &x = Xb[i0 + i + (size_t)j * n];
        x = cadd(x, db);
      },
      gsm);
}

// Forward correction, part 1 (p > 0): rhs = c_p + R_p g_p - f_p for this CTA's
// rows, R_p = e_p Z_{p-1} e_p.
__global__ void __launch_bounds__(NT) k_refine_fwd_a(RefineArgs a, int p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.y, i0 = blockIdx.x * SKINNY_BM;
  const PointDesc d = a.pts[pt];
  if (refine_skip(a, d, pt, p) || i0 >= a.n) return;
  const int n = a.n, nc = a.nc;
  const int rows = min(SKINNY_BM, n - i0);
  cc *gsm = reinterpret_cast<cc *>(smraw);
  cc *eL = gsm + skinny_smem_elems<float>();
  load_kv32(a, d, p, nullptr, nullptr, eL, nullptr);
  const cc *Zprev = a.Zst + ((size_t)d.st_off + p - 1) * n * n;
  cc *rhs = a.M + (size_t)pt * n * (n + nc);   // n x nc scratch
  const zc *carry = a.carry + (size_t)pt * n * nc;
  const zc *F = a.Fr + iblk(a, d, p);
  const zc *G = a.Gr + iblk(a, d, p);
  cta_gemm_skinny<float>(
      rows, nc, n, [=](int i, int l) { return cmul(cmul(eL[i0 + i], Zprev[i0 + i + (size_t)l * n]), eL[l]); },
      [=](int l, int j) { return ccast<float>(G[l + (size_t)j * n]); },
      [=](int i, int j, cc acc) {
        const size_t e = i0 + i + (size_t)j * n;
        rhs[e] = ccast<float>(csub(cadd(carry[e], ccast<double>(acc)), F[e]));
      },
      gsm);
}

// Forward correction, part 2 (one CTA per point): u_p = W_p^{-1} rhs by the
// stored LU factors, c_{p+1} = e_q u_p; at the point's last interface the
// correction of a_{N+1} is added and its relative size recorded.
__global__ void __launch_bounds__(NT) k_refine_fwd_b(RefineArgs a, int p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const PointDesc d = a.pts[pt];
  if (refine_skip(a, d, pt, p)) return;
  const int n = a.n, nc = a.nc, N = d.N;
  cc *gsm = reinterpret_cast<cc *>(smraw);
  cc *eR = gsm + skinny_smem_elems<float>() + Tile<float>::NB * Tile<float>::NB;
  load_kv32(a, d, p, nullptr, nullptr, nullptr, eR);
  const cc *LU = a.LUst + ((size_t)d.st_off + p) * n * n;
  const int *piv = a.PIVst + ((size_t)d.st_off + p) * n;
  cc *Ust = a.Ust + ((size_t)d.st_off + p) * n * nc;
  cc *rhs = a.M + (size_t)pt * n * (n + nc);
  zc *carry = a.carry + (size_t)pt * n * nc;
  if (p == 0) {
    const zc *F = a.Fr + iblk(a, d, p);
    for (int e = threadIdx.x; e < n * nc; e += NT) rhs[e] = ccast<float>(csub(carry[e], F[e]));
    __syncthreads();
  }
  cta_lu_replay<float>(LU, n, piv, rhs, n, nc, gsm, a.lapack_piv != 0);
  for (int e = threadIdx.x; e < n * nc; e += NT) {
    const int i = e % n;
    const cc u = rhs[e];
    Ust[e] = u;
    carry[e] = ccast<double>(cmul(eR[i], u));
  }
  __syncthreads();
  if (p == N) {
    // add the correction of a_{N+1}; record its size relative to a_{N+1}
    zc *X = a.Xa + blk(a, d, N + 1);
    double dn = 0.0, xn = 0.0;
    for (int e = threadIdx.x; e < n * nc; e += NT) {
      const zc dx = carry[e];
      const zc x = cadd(X[e], dx);
      X[e] = x;
      dn += cnorm2(dx);
      xn += cnorm2(x);
    }
    for (int off = 16; off > 0; off >>= 1) {
      dn += __shfl_down_sync(0xffffffffu, dn, off);
      xn += __shfl_down_sync(0xffffffffu, xn, off);
    }
    __shared__ double red[2][NT / 32];
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = dn; red[1][threadIdx.x >> 5] = xn; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sd = 0.0, sx = 0.0;
      for (int w = 0; w < NT / 32; ++w) { sd += red[0][w]; sx += red[1][w]; }
      a.corr_prev[pt] = a.corr[pt];
      a.corr[pt] = sx > 0.0 ? sqrt(sd / sx) : 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 residual of every interface equation (one CTA per (interface, point)):
//   y1 = O (a_q + e_q b_q),  y2 = O K_q (a_q - e_q b_q),
//   f_p = -(e_p a_p - (y1 + K_p^{-1} y2)/2),  g_p = -(b_p - (y1 - K_p^{-1} y2)/2).
__global__ void __launch_bounds__(NT) k_refine_residual(RefineArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int p = blockIdx.x, pt = blockIdx.y;
  const PointDesc d = a.pts[pt];
  if (d.skip || a.status[pt] || p > d.N) return;
  const int n = a.n, nc = a.nc, N = d.N, q = p + 1;
  zc *gsm = reinterpret_cast<zc *>(smraw);
  KV v = carve_kv(smraw, skinny_smem_elems<double>() * sizeof(zc), n);
  load_kv(a, d, p, v);
  const zc *O = overlap(a, d, p);
  const size_t ooff = ((size_t)d.o_off + p) * (size_t)n * n;
  const cc *Ohi = (a.O32 && a.O32lo) ? a.O32 + ooff : nullptr;
  const cc *Olo = Ohi ? a.O32lo + ooff : nullptr;
  const zc *ap = a.Xa + blk(a, d, p);
  const zc *bp = a.Xb + blk(a, d, p);
  const zc *aq = a.Xa + blk(a, d, q);
  const zc *bq = a.Xb + blk(a, d, q);
  zc *F = a.Fr + iblk(a, d, p);
  zc *G = a.Gr + iblk(a, d, p);
  const KV vc = v;
  const bool has_bq = q <= N;
  // the O y products in double-float (48-bit) arithmetic on the FP32 pipe
  cta_gemm_skinny<df>(
      n, 2 * nc, n,
      [=](int i, int l) {
        const size_t e = i + (size_t)l * n;
        if (Ohi) {   // the double-float O from its two FP32 planes (no FP64 arithmetic)
          const cc h = Ohi[e], lo = Olo[e];
          dfc z;
          z.re = mkdf(h.re, lo.re);
          z.im = mkdf(h.im, lo.im);
          return z;
        }
        return dfc_of(O[e]);
      },
      [=](int l, int j) {
        const int c = j < nc ? j : j - nc;
        const zc A = aq[l + (size_t)c * n];
        const zc eb = has_bq ? cmul(vc.eR[l], bq[l + (size_t)c * n]) : czero<double>();
        return dfc_of(j < nc ? cadd(A, eb) : cmul(vc.kR[l], csub(A, eb)));
      },
      [=](int i, int j, dfc acc) {
        if (j < nc) F[i + (size_t)j * n] = dfc_val(acc);
        else G[i + (size_t)(j - nc) * n] = dfc_val(acc);
      },
      reinterpret_cast<dfc *>(gsm));
  for (int e = threadIdx.x; e < n * nc; e += NT) {
    const int i = e % n;
    const zc y1 = F[e], y2 = cmul(vc.kinvL[i], G[e]);
    const zc fwd = mkc<double>(0.5 * (y1.re + y2.re), 0.5 * (y1.im + y2.im));
    const zc bwd = mkc<double>(0.5 * (y1.re - y2.re), 0.5 * (y1.im - y2.im));
    F[e] = csub(fwd, cmul(vc.eL[i], ap[e]));
    G[e] = csub(bwd, bp[e]);
  }
}

// ---------------------------------------------------------------------------
// t and T from the refined a_{N+1}.  The estimate of the relative error of T
// left after the last pass is the relative change of T that pass made, times
// the contraction c_i / c_{i-1} it showed (c = relative size of the
// correction of a_{N+1}; 1 after a single pass).
__global__ void __launch_bounds__(NT) k_refine_finish(RefineArgs a) {
  const int pt = blockIdx.x;
  const PointDesc d = a.pts[pt];
  const int n = a.n, nc = a.nc, N = d.N, tid = threadIdx.x;
  if (d.skip || a.status[pt]) {
    if (tid == 0) {
      a.T[d.out] = __longlong_as_double(0x7ff8000000000000ll);
      if (a.nopen) { a.nopen[2 * d.out] = d.nL; a.nopen[2 * d.out + 1] = d.nR; }
      if (a.err) a.err[d.out] = 0.0;
    }
    return;
  }
  const double *EL = a.En + (size_t)d.en_off * n;
  const double *ER = EL + (size_t)(N + 1) * n;
  const zc *X = a.Xa + blk(a, d, N + 1);
  const zc *dX = a.carry + (size_t)pt * n * nc;   // last correction of a_{N+1}
  double acc = 0.0, accp = 0.0;
  for (int e = tid; e < d.nR * d.nL; e += NT) {
    const int i = e % d.nR, j = e / d.nR;
    const double f = sqrt(sqrt(d.E - ER[i]) / sqrt(d.E - EL[j]));
    const zc x = X[i + (size_t)j * n];
    const zc xp = csub(x, dX[i + (size_t)j * n]);
    const zc tv = mkc<double>(f * x.re, f * x.im);
    acc += cnorm2(tv);
    accp += f * f * cnorm2(xp);
    if (a.t) a.t[(size_t)d.out * n * n + i + (size_t)j * n] = tv;
  }
  for (int off = 16; off > 0; off >>= 1) {
    acc += __shfl_down_sync(0xffffffffu, acc, off);
    accp += __shfl_down_sync(0xffffffffu, accp, off);
  }
  __shared__ double red[2][NT / 32];
  if ((tid & 31) == 0) { red[0][tid >> 5] = acc; red[1][tid >> 5] = accp; }
  __syncthreads();
  if (tid == 0) {
    double T = 0.0, Tp = 0.0;
    for (int w = 0; w < NT / 32; ++w) { T += red[0][w]; Tp += red[1][w]; }
    a.T[d.out] = T;
    if (a.nopen) { a.nopen[2 * d.out] = d.nL; a.nopen[2 * d.out + 1] = d.nR; }
    const double c = a.corr[pt], cp = a.corr_prev[pt];
    const double rho = cp > 0.0 ? fmin(1.0, c / cp) : 1.0;
    if (a.err) a.err[d.out] = rho * fabs(T - Tp) / fmax(T, 1e-300);
  }
}

// ---------------------------------------------------------------------------
size_t refine_smem_bytes(int n) {
  const size_t kv = 4 * (size_t)n * sizeof(zc);
  const size_t fwd = (skinny_smem_elems<float>() + Tile<float>::NB * Tile<float>::NB) * sizeof(cc) + kv;
  const size_t bwd = skinny_smem_elems<float>() * sizeof(cc) + kv;
  const size_t res = skinny_smem_elems<double>() * sizeof(zc) + kv;
  return std::max(fwd, std::max(bwd, res)) + 64;
}

cudaError_t launch_refine(const RefineArgs &a, int npts, int min_iters, int max_iters, double tol,
                          cudaStream_t s, int *passes) {
  const size_t smem = refine_smem_bytes(a.n);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_refine_bwd_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
      (e = cudaFuncSetAttribute(k_refine_bwd_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
      (e = cudaFuncSetAttribute(k_refine_fwd_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
      (e = cudaFuncSetAttribute(k_refine_fwd_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
      (e = cudaFuncSetAttribute(k_refine_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return e;
  const dim3 rgrid((a.n + SKINNY_BM - 1) / SKINNY_BM, npts);
  const bool batched = a.Bw && a.Yw && a.O32 && a.n <= 1024;
  if (batched &&
      (e = cudaFuncSetAttribute(k_refine_bwd_mm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::cg_smem_bytes())))
    return e;
  const int mm_tiles = ((a.n + tc::CG_M / 2 - 1) / (tc::CG_M / 2)) * ((2 * a.nc * npts + tc::CG_N - 1) / tc::CG_N);
  auto backward = [&](int with_src) {
    for (int p = a.N; p >= 0; --p) {
      k_refine_bwd_a<<<rgrid, NT, smem, s>>>(a, p, with_src);
      if (batched) {
        k_refine_bwd_mm<<<mm_tiles, tc::CG_THREADS, tc::cg_smem_bytes(), s>>>(a, p, npts);
        k_refine_bwd_c<<<rgrid, NT, 0, s>>>(a, p, with_src);
      } else {
        k_refine_bwd_b<<<rgrid, NT, smem, s>>>(a, p, with_src);
      }
    }
  };
  auto forward = [&]() {
    for (int p = 0; p <= a.N; ++p) {
      if (p > 0) k_refine_fwd_a<<<rgrid, NT, smem, s>>>(a, p);
      k_refine_fwd_b<<<npts, NT, smem, s>>>(a, p);
    }
  };
  const size_t vec = (size_t)npts * a.n * a.nc * sizeof(zc);
  const size_t slot = (size_t)a.n * a.nc * sizeof(zc);
  if ((e = cudaMemsetAsync(a.Xa, 0, slot * a.x_slots, s)) || (e = cudaMemsetAsync(a.Xb, 0, slot * a.x_slots, s)) ||
      (e = cudaMemsetAsync(a.Gr, 0, slot * a.st_slots, s)) ||
      (e = cudaMemsetAsync(a.corr, 0, npts * sizeof(double), s)) ||
      (e = cudaMemsetAsync(a.corr_prev, 0, npts * sizeof(double), s)))
    return e;
  k_refine_init<<<npts, NT, 0, s>>>(a);
  // x0: backward pass over the first sweep's Z_p, u_p
  if ((e = cudaMemsetAsync(a.carry, 0, vec, s))) return e;
  backward(0);
  // stopping test: the correction of pass i shrinks the error by about
  // c_i / c_{i-1} (c = relative size of the correction of a_{N+1}), so the
  // error left after pass i is estimated as c_i^2 / c_{i-1}
  std::vector<double> corr(npts), prev(npts, 0.0);
  int it = 0;
  for (; it < max_iters; ++it) {
    k_refine_residual<<<dim3(a.N + 1, npts), NT, smem, s>>>(a);
    if ((e = cudaMemsetAsync(a.carry, 0, vec, s))) return e;
    forward();
    if (it + 1 >= max_iters) { ++it; break; }
    if ((e = cudaMemcpyAsync(corr.data(), a.corr, npts * sizeof(double), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
      return e;
    if (it + 1 >= min_iters) {
      double worst = 0.0;
      for (int i = 0; i < npts; ++i) {
        const double est = prev[i] > 0.0 ? corr[i] * corr[i] / prev[i] : corr[i];
        worst = std::max(worst, est);
      }
      if (worst < tol) { ++it; break; }
    }
    prev = corr;
    // interior corrections: backward from db_{N+1} = 0
    if ((e = cudaMemsetAsync(a.carry, 0, vec, s))) return e;
    backward(1);
  }
  if (passes) *passes = it;
  k_refine_finish<<<npts, NT, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace pw
