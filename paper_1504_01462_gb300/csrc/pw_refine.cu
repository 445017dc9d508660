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
#include <string.h>

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
  cta_lu_replay<float>(LU, n, piv, rhs, n, nc, gsm, a.piv_order);
  for (int e = threadIdx.x; e < n * nc; e += NT) {
    const int i = e % n;
    const cc u = rhs[e];
    Ust[e] = u;
    carry[e] = ccast<double>(cmul(eR[i], u));
  }
  __syncthreads();
  if (p == N) {
    // add the correction of a_{N+1}; record the size of the correction of t
    // (the flux-weighted open block, the part T is made of) relative to t,
    // with |t| taken as at least 1e-3: T below 1e-6 is judged absolutely
    zc *X = a.Xa + blk(a, d, N + 1);
    const double *EL = a.En + (size_t)d.en_off * n;
    const double *ER = EL + (size_t)(N + 1) * n;
    double dn = 0.0, xn = 0.0;
    for (int e = threadIdx.x; e < n * nc; e += NT) {
      const zc dx = carry[e];
      const zc x = cadd(X[e], dx);
      X[e] = x;
      const int i = e % n, j = e / n;
      if (i < d.nR && j < d.nL) {
        const double f2 = sqrt(d.E - ER[i]) / sqrt(d.E - EL[j]);
        dn += f2 * cnorm2(dx);
        xn += f2 * cnorm2(x);
      }
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
      a.corr[pt] = sqrt(sd / fmax(sx, 1e-6));
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 residual of every interface equation (one CTA per (interface, point)):
//   y1 = O (a_q + e_q b_q),  y2 = O K_q (a_q - e_q b_q),
//   f_p = -(e_p a_p - (y1 + K_p^{-1} y2)/2),  g_p = -(b_p - (y1 - K_p^{-1} y2)/2).
__global__ void __launch_bounds__(NT) k_refine_residual(RefineArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  // grid (points, interfaces): the CTAs that run together share one
  // interface's overlap in L2
  const int pt = blockIdx.x, p = blockIdx.y;
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
// The residual's products O y by exact slices on the tensor cores, when every
// point shares its overlaps (an error-free splitting in the manner of Ozaki et
// al., Numer. Algorithms 59, 2012).  In real form the product is A' B' with
//   A' = [[Re O, -Im O], [Im O, Re O]] (2n x 2n),  B' = [Re y; Im y] (2n x ncol),
// ncol = 2 nc npts (the columns a_q + e b_q and K_q (a_q - e b_q) of every
// point).  Row r of A' is scaled by 2^-ea_r and column j of B' by 2^-eb_j
// (powers of two that bring every entry below 1 in magnitude) and cut into
// RS_SLICES slices of RS_BITS bits: A' = 2^ea sum_s A_s, where A_s holds
// integers of at most 2^7 in magnitude times 2^-7(s+1) (likewise B' and B_t).
// Every slice is exact in BF16, every product of two slice entries is an
// integer of at most 2^14 times 2^-7(s+t+2), and a sum of K = 2n <= 1024 of
// them stays an integer of at most 2^24 units: the tensor core's FP32
// accumulation of A_s B_t is exact.  The pairs with s + t < RS_SLICES are
// summed in double-float in registers (the ones with s + t >= RS_SLICES lie
// below 2^-56 of the result); the operands are the double-float overlap and y
// rounded to double-float, so the products carry 48 bits like the CUDA-core
// double-float residual, at tensor-core speed.
namespace {
constexpr int RS_THREADS = 256;

// one block's maximum of a non-negative float
__device__ float block_maxf(float v, float *red) {
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = 0.f;
  for (int w = 0; w < RS_THREADS / 32; ++w) m = fmaxf(m, red[w]);
  __syncthreads();
  return m;
}

// 2^-e for the scaling exponent e of a block whose largest magnitude is m
__device__ __forceinline__ int scale_exponent(float m) {
  int e = 0;
  if (m > 0.f) frexpf(m, &e);   // m < 2^e
  return e;
}

// The slices of the double-float x = hi + lo scaled by 2^-e (|x| < 2^e), as
// BF16 bit patterns into out[s * stride].  Slice s is trunc(R 2^7(s+1)) 2^-7(s+1)
// of the remainder R, taken from R's high part: every step is exact in FP32
// (the truncation keeps the leading bits of hi, hi - c drops them, TwoSum
// renormalises), so the slices sum to x up to the last remainder.
__device__ __forceinline__ void cut_slices_df(float hi, float lo, int e, uint16_t *out, size_t stride) {
  float h = ldexpf(hi, -e), l = ldexpf(lo, -e);
#pragma unroll
  for (int s = 0; s < RS_SLICES; ++s) {
    const float up = __int_as_float((127 + RS_BITS * (s + 1)) << 23);    // 2^7(s+1)
    const float down = __int_as_float((127 - RS_BITS * (s + 1)) << 23);  // 2^-7(s+1)
    const float c = truncf(h * up) * down;
    out[(size_t)s * stride] = (uint16_t)(__float_as_uint(c) >> 16);   // c has at most 8 significant bits
    float sh, se;
    two_sum(h - c, l, sh, se);
    h = sh;
    l = se;
  }
}

// the slice pair (s, t) of step P, the pairs ordered by decreasing s + t
__device__ __forceinline__ int rs_pair(int P, int &s, int &t) {
  int d = RS_SLICES - 1;
  while (P > d) {
    P -= d + 1;
    --d;
  }
  s = P;
  t = d - P;
  return d;
}
}  // namespace

// A' of interface p: block i cuts rows i and i + n (one exponent: both hold
// the values Re O_ik, Im O_ik up to sign).
__global__ void __launch_bounds__(RS_THREADS) k_res_oslice(RefineArgs a, int p) {
  __shared__ float red[RS_THREADS / 32];
  const int n = a.n, i = blockIdx.x, K = 2 * n;
  const size_t ooff = ((size_t)a.pts[0].o_off + p) * (size_t)n * n + i;
  const cc *Oh = a.O32 + ooff, *Ol = a.O32lo + ooff;
  float m = 0.f;
  for (int k = threadIdx.x; k < n; k += RS_THREADS) {
    const cc h = Oh[(size_t)k * n];
    m = fmaxf(m, fmaxf(fabsf(h.re), fabsf(h.im)));
  }
  const int e = scale_exponent(block_maxf(m, red));
  if (threadIdx.x == 0) {
    a.Oexp[i] = e;
    a.Oexp[i + n] = e;
  }
  const size_t stride = (size_t)K * K;
  uint16_t *r1 = a.Osl + (size_t)i * K, *r2 = a.Osl + (size_t)(i + n) * K;
  for (int k = threadIdx.x; k < n; k += RS_THREADS) {
    const cc h = Oh[(size_t)k * n], l = Ol[(size_t)k * n];
    // row i = [Re O, -Im O], row i + n = [Im O, Re O]; the slices of -x are those of x negated
    cut_slices_df(h.re, l.re, e, r1 + k, stride);
    cut_slices_df(h.im, l.im, e, r2 + k, stride);
#pragma unroll
    for (int s = 0; s < RS_SLICES; ++s) {
      r2[(size_t)s * stride + n + k] = r1[(size_t)s * stride + k];
      r1[(size_t)s * stride + n + k] = r2[(size_t)s * stride + k] ^ 0x8000u;
    }
  }
}

// B' of interface p: block (pt, h) cuts the nc columns j = pt 2nc + h nc + ch,
// ch < nc (h = 0: a_q + e b_q of channel ch; h = 1: K_q (a_q - e b_q)); zero
// for points that are skipped, failed or shorter than p.  The wavenumbers and
// phases of slice q = p + 1 (FP64 square roots and exponentials) are formed
// once per block for its nc columns.
__global__ void __launch_bounds__(RS_THREADS) k_res_yslice(RefineArgs a, int p) {
  __shared__ float red[RS_THREADS / 32];
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = a.n, nc = a.nc, K = 2 * n, ncol = gridDim.x * 2 * nc;
  const int pt = blockIdx.x, h = blockIdx.y, jb = pt * 2 * nc + h * nc;
  const PointDesc d = a.pts[pt];
  const size_t stride = (size_t)ncol * K;
  if (d.skip || a.status[pt] || p > d.N) {
    for (int ch = 0; ch < nc; ++ch) {
      uint16_t *out = a.Ysl + (size_t)(jb + ch) * K;
      for (int k = threadIdx.x; k < K; k += RS_THREADS)
#pragma unroll
        for (int s = 0; s < RS_SLICES; ++s) out[(size_t)s * stride + k] = 0;
      if (threadIdx.x == 0) a.Yexp[jb + ch] = 0;
    }
    return;
  }
  KV v = carve_kv(smraw, 0, n);
  const int q = p + 1;
  {
    const double *Eq = a.En + ((size_t)d.en_off + q) * n;
    const double dzq = a.dz[d.dz_off + q];
    for (int i = threadIdx.x; i < n; i += RS_THREADS) {
      const zc kr = kz_branch(d.E, Eq[i]);
      v.kR[i] = kr;
      v.eR[i] = phase_fwd(kr, dzq);
    }
    __syncthreads();
  }
  const bool has_bq = q <= d.N;
  for (int ch = 0; ch < nc; ++ch) {
    const int j = jb + ch;
    uint16_t *out = a.Ysl + (size_t)j * K;
    const zc *aq = a.Xa + blk(a, d, q) + (size_t)ch * n;
    const zc *bq = a.Xb + blk(a, d, q) + (size_t)ch * n;
    auto yv = [&](int l) -> dfc {
      const zc A = aq[l];
      const zc eb = has_bq ? cmul(v.eR[l], bq[l]) : czero<double>();
      return dfc_of(h == 0 ? cadd(A, eb) : cmul(v.kR[l], csub(A, eb)));
    };
    float m = 0.f;
    for (int l = threadIdx.x; l < n; l += RS_THREADS) {
      const dfc y = yv(l);
      m = fmaxf(m, fmaxf(fabsf(y.re.hi), fabsf(y.im.hi)));
    }
    const int e = scale_exponent(block_maxf(m, red));
    if (threadIdx.x == 0) a.Yexp[j] = e;
    for (int l = threadIdx.x; l < n; l += RS_THREADS) {
      const dfc y = yv(l);
      cut_slices_df(y.re.hi, y.re.lo, e, out + l, stride);
      cut_slices_df(y.im.hi, y.im.lo, e, out + n + l, stride);
    }
  }
}

// Yacc = A' B' summed over the slice pairs.  One CTA per 128 x 128 tile of
// A' B'; K in stages of 64 (four BF16 MMAs of M = N = 128, K = 16) through a
// ring of RS_RING shared-memory stages filled by cp.async: RS_AHEAD stages of
// operand loads are in flight, and a stage's slot is refilled once the MMAs
// of the stage two back have completed, so that up to three stages of MMAs
// queue on the tensor core instead of one.
// Each pair accumulates in one of two TMEM buffers (128 columns each); the
// finished pair's buffer is read back and added into the double-float
// registers in eight column chunks spread over the next pair's stages, so the
// read-back overlaps the next pair's products.  Warp w holds TMEM lanes
// 32 (w % 4) .. + 31 (rows) and columns 64 (w / 4) .. + 63.
constexpr int RS_TILE = 128, RS_KS = 64, RS_RING = 6, RS_AHEAD = RS_RING - 2;
constexpr int RS_OPER = RS_TILE * RS_KS * 2;   // bytes of one operand per stage
constexpr int RS_STAGE = 2 * RS_OPER;
constexpr int RS_DF_BELOW = 4;                 // pairs with s + t < 4 add in double-float, the rest in FP32
size_t res_mm_smem_bytes() { return (size_t)RS_RING * RS_STAGE + 128; }

__global__ void __launch_bounds__(256, 1) k_res_mm(RefineArgs a, int ncol, int npts) {
  extern __shared__ __align__(128) unsigned char smtc[];
  const int n = a.n, M = 2 * n, K = 2 * n;
  const int tiles_m = (M + RS_TILE - 1) / RS_TILE;
  const int r0 = (blockIdx.x % tiles_m) * RS_TILE, j0 = (blockIdx.x / tiles_m) * RS_TILE;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smtc + RS_RING * RS_STAGE);   // [RS_RING]
  uint32_t *slot = reinterpret_cast<uint32_t *>(mbar + RS_RING);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ns = (K + RS_KS - 1) / RS_KS, G = RS_PAIRS * ns;
  if (warp == 0) tc::tmem_alloc(slot, 2 * RS_TILE);
  if (tid == 0)
    for (int b = 0; b < RS_RING; ++b) tc::mbar_init(&mbar[b], 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;

  // operand loads of stage g: 128 rows x 8 chunks of 16 bytes per operand;
  // task u (4 per warp) covers rows 8 (u / 2) .. + 7 and chunks 4 (u % 2) .. + 3,
  // lane -> row 8 (u / 2) + lane % 8, chunk 4 (u % 2) + lane / 8 (each 8-lane
  // phase writes 8 distinct bank groups; each row's 64 bytes are contiguous)
  auto load_stage = [&](int g) {
    if (g < G) {
      int s, t;
      const int P = g / ns, k0 = (g - P * ns) * RS_KS;
      rs_pair(P, s, t);
      unsigned char *A = smtc + (g % RS_RING) * RS_STAGE, *B = A + RS_OPER;
      const uint16_t *As = a.Osl + (size_t)s * M * K, *Bs = a.Ysl + (size_t)t * ncol * K;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int u = warp * 4 + i, row = 8 * (u >> 1) + (lane & 7), c = 4 * (u & 1) + (lane >> 3);
        const int kk = k0 + 8 * c;
        const uint32_t off = (uint32_t)(c >> 1) * (RS_TILE * 32) + (uint32_t)(row >> 3) * 256u +
                             (uint32_t)(c & 1) * 128u + (uint32_t)(row & 7) * 16u;
        const bool va = r0 + row < M && kk < K, vb = j0 + row < ncol && kk < K;
        tc::cp_async16(A + off, va ? As + (size_t)(r0 + row) * K + kk : As, va);
        tc::cp_async16(B + off, vb ? Bs + (size_t)(j0 + row) * K + kk : Bs, vb);
      }
    }
    tc::cp_async_commit();   // one group per stage, empty past the end
  };

  float ah[8][8], al[8][8];   // double-float sums of this thread's 64 results
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int i = 0; i < 8; ++i) ah[q][i] = al[q][i] = 0.f;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * (warp >> 2));
  // add chunk q of pair P's buffer into the sums
  auto read_chunk = [&](int P, int q, float (&hq)[8], float (&lq)[8]) {
    int s, t;
    const int d = rs_pair(P, s, t);
    float v[8];
    tc::tmem_ld8(lane_base + (uint32_t)((P & 1) * RS_TILE + 8 * q), v);
    // the slices carry their scale 2^-7(s+1), so the accumulator already holds
    // the pair's product (a multiple of 2^-7(s+t+2), exact in FP32)
    if (d >= RS_DF_BELOW) {
#pragma unroll
      for (int i = 0; i < 8; ++i) hq[i] += v[i];
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float sh, se;
        two_sum(hq[i], v[i], sh, se);
        hq[i] = sh;
        lq[i] += se;
      }
    }
  };

  for (int g = 0; g < RS_AHEAD; ++g) load_stage(g);
  bool ok = true;
  int last = -1;   // the last stage whose MMAs were issued
  for (int g = 0; g < G; ++g) {
    const int P = g / ns, st = g - P * ns;
    tc::cp_async_wait<RS_AHEAD - 1>();   // this thread's copies of stage g have landed
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    ok = __syncthreads_and(ok) != 0;
    if (!ok) break;
    if (tid == 0) {
      tc::fence_after_sync();
      const unsigned char *A = smtc + (g % RS_RING) * RS_STAGE, *B = A + RS_OPER;
      const uint32_t d = tmem + (uint32_t)((P & 1) * RS_TILE);
      constexpr uint32_t idesc = tc::idesc_bf16(RS_TILE, RS_TILE);
#pragma unroll
      for (int m = 0; m < RS_KS / 16; ++m)
        tc::mma_bf16(d, tc::smem_desc(A + m * RS_TILE * 32, 128, 256), tc::smem_desc(B + m * RS_TILE * 32, 128, 256),
                     idesc, (st > 0 || m > 0) ? 1u : 0u);
      tc::mma_commit(&mbar[g % RS_RING]);
    }
    last = g;
    // stage g - 2's slot is free once its MMAs are done: refill it with stage
    // g + RS_AHEAD (the slots of stages g - 1 .. g + RS_AHEAD - 1 stay in use)
    if (g >= 2) ok = tc::mbar_wait(&mbar[(g - 2) % RS_RING], ((g - 2) / RS_RING) & 1) && ok;
    tc::fence_after_sync();
    if (ok) load_stage(g + RS_AHEAD);
    else tc::cp_async_commit();
    // pair P - 1's last stage is g - st - 1, complete once st >= 1 (stage g - 2
    // waited for above); at st == 0 it is stage g - 1, waited for here
    if (P > 0 && st == 0 && ok) {
      ok = tc::mbar_wait(&mbar[(g - 1) % RS_RING], ((g - 1) / RS_RING) & 1) && ok;
      tc::fence_after_sync();
    }
    // read back pair P - 1's chunks q with q ns / 8 == st
    if (P > 0 && __all_sync(0xffffffffu, ok)) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if ((q * ns) / 8 == st) read_chunk(P - 1, q, ah[q], al[q]);
    }
  }
  if (ok) {
    ok = tc::mbar_wait(&mbar[(G - 1) % RS_RING], ((G - 1) / RS_RING) & 1);
    tc::fence_after_sync();
    if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
      for (int q = 0; q < 8; ++q) read_chunk(RS_PAIRS - 1, q, ah[q], al[q]);
    }
  }
  tc::cp_async_wait<0>();
  ok = __syncthreads_and(ok) != 0;
  if (ok) {
    const int row = r0 + 32 * (warp & 3) + lane;
    if (row < M) {
      const int er = a.Oexp[row];
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int j = j0 + 64 * (warp >> 2) + 8 * q + i;
          if (j < ncol) a.Yacc[(size_t)j * M + row] = ldexp((double)ah[q][i] + (double)al[q][i], er + a.Yexp[j]);
        }
    }
  } else {
    // a wait ran out: wait (bounded again) for the products still in flight, report
    if (last >= 0) tc::mbar_wait(&mbar[last % RS_RING], (last / RS_RING) & 1, 1u << 16);
    if (tid == 0)
      for (int pt = 0; pt < npts; ++pt) a.status[pt] = 2;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * RS_TILE);
}

// The residual of interface p from Yacc (block pt): with y1 = O (a_q + e b_q)
// and y2 = O K_q (a_q - e b_q),
//   f_p = (y1 + K_p^-1 y2)/2 - e_p a_p,  g_p = (y1 - K_p^-1 y2)/2 - b_p.
__global__ void __launch_bounds__(NT) k_res_finish(RefineArgs a, int p, int ncol) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const PointDesc d = a.pts[pt];
  if (d.skip || a.status[pt] || p > d.N) return;
  const int n = a.n, nc = a.nc, M = 2 * n;
  KV v = carve_kv(smraw, 0, n);
  load_kv(a, d, p, v);
  const zc *ap = a.Xa + blk(a, d, p);
  const zc *bp = a.Xb + blk(a, d, p);
  zc *F = a.Fr + iblk(a, d, p);
  zc *G = a.Gr + iblk(a, d, p);
  const double *Y1 = a.Yacc + (size_t)pt * 2 * nc * M;
  for (int e = threadIdx.x; e < n * nc; e += NT) {
    const int i = e % n, c = e / n;
    const double *c1 = Y1 + (size_t)c * M, *c2 = Y1 + (size_t)(nc + c) * M;
    const zc y1 = mkc<double>(c1[i], c1[i + n]);
    const zc y2 = cmul(v.kinvL[i], mkc<double>(c2[i], c2[i + n]));
    const zc fwd = mkc<double>(0.5 * (y1.re + y2.re), 0.5 * (y1.im + y2.im));
    const zc bwd = mkc<double>(0.5 * (y1.re - y2.re), 0.5 * (y1.im - y2.im));
    F[e] = csub(fwd, cmul(v.eL[i], ap[e]));
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
    if (a.err) a.err[d.out] = rho * fabs(T - Tp) / fmax(T, 1e-6);   // absolute below T = 1e-6
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
  // the residual by exact slices: every point shares its overlaps, K = 2n <= 1024 keeps
  // the slice products exact in FP32, and 2n is a multiple of 8 (whole 16-byte chunks)
  const bool sliced = a.Osl && a.Ysl && a.Oexp && a.Yexp && a.Yacc && a.O32 && a.O32lo && a.n <= 512 &&
                      (a.n % 4) == 0;
  const size_t kv_bytes = 4 * (size_t)a.n * sizeof(zc);
  const int rs_tiles = ((2 * a.n + RS_TILE - 1) / RS_TILE) * ((2 * a.nc * npts + RS_TILE - 1) / RS_TILE);
  if (sliced && ((e = cudaFuncSetAttribute(k_res_mm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)res_mm_smem_bytes())) ||
                 (e = cudaFuncSetAttribute(k_res_yslice, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kv_bytes)) ||
                 (e = cudaFuncSetAttribute(k_res_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kv_bytes))))
    return e;
  auto backward = [&](int with_src) {
    for (int p = a.N; p >= 0; --p) {
      PW_TIMED(KK_REF_BWD_A, s, k_refine_bwd_a<<<rgrid, NT, smem, s>>>(a, p, with_src));
      if (batched) {
        PW_TIMED(KK_REF_BWD_MM, s, k_refine_bwd_mm<<<mm_tiles, tc::CG_THREADS, tc::cg_smem_bytes(), s>>>(a, p, npts));
        PW_TIMED(KK_REF_BWD_C, s, k_refine_bwd_c<<<rgrid, NT, 0, s>>>(a, p, with_src));
      } else {
        PW_TIMED(KK_REF_BWD_B, s, k_refine_bwd_b<<<rgrid, NT, smem, s>>>(a, p, with_src));
      }
    }
  };
  auto forward = [&]() {
    for (int p = 0; p <= a.N; ++p) {
      if (p > 0) PW_TIMED(KK_REF_FWD_A, s, k_refine_fwd_a<<<rgrid, NT, smem, s>>>(a, p));
      PW_TIMED(KK_REF_FWD_B, s, k_refine_fwd_b<<<npts, NT, smem, s>>>(a, p));
    }
  };
  const size_t vec = (size_t)npts * a.n * a.nc * sizeof(zc);
  const size_t slot = (size_t)a.n * a.nc * sizeof(zc);
  if ((e = cudaMemsetAsync(a.Xa, 0, slot * a.x_slots, s)) || (e = cudaMemsetAsync(a.Xb, 0, slot * a.x_slots, s)) ||
      (e = cudaMemsetAsync(a.Gr, 0, slot * a.st_slots, s)) ||
      (e = cudaMemsetAsync(a.corr, 0, npts * sizeof(double), s)) ||
      (e = cudaMemsetAsync(a.corr_prev, 0, npts * sizeof(double), s)))
    return e;
  PW_TIMED(KK_REF_INIT, s, k_refine_init<<<npts, NT, 0, s>>>(a));
  // x0: backward pass over the first sweep's Z_p, u_p
  if ((e = cudaMemsetAsync(a.carry, 0, vec, s))) return e;
  backward(0);
  // stopping test: the correction of pass i shrinks the error by about
  // c_i / c_{i-1} (c = relative size of the correction of a_{N+1}), so the
  // error left after pass i is estimated as c_i^2 / c_{i-1}
  std::vector<double> corr(npts), prev(npts, 0.0);
  int it = 0;
  for (; it < max_iters; ++it) {
    if (sliced) {
      const int ncol = 2 * a.nc * npts;
      for (int p = 0; p <= a.N; ++p) {
        PW_TIMED(KK_RES_OSLICE, s, k_res_oslice<<<a.n, RS_THREADS, 0, s>>>(a, p));
        PW_TIMED(KK_RES_YSLICE, s, k_res_yslice<<<dim3(npts, 2), RS_THREADS, kv_bytes, s>>>(a, p));
        PW_TIMED(KK_RES_MM, s, k_res_mm<<<rs_tiles, 256, res_mm_smem_bytes(), s>>>(a, ncol, npts));
        PW_TIMED(KK_RES_FINISH, s, k_res_finish<<<npts, NT, kv_bytes, s>>>(a, p, ncol));
      }
    } else {
      PW_TIMED(KK_REF_RESIDUAL, s, k_refine_residual<<<dim3(npts, a.N + 1), NT, smem, s>>>(a));
    }
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
  PW_TIMED(KK_REF_FINISH, s, k_refine_finish<<<npts, NT, 0, s>>>(a));
  return cudaGetLastError();
}

}  // namespace pw

// ---------------------------------------------------------------------------
// Self-test of the exact-slice product (k_res_mm) on random slices.
extern "C" pw_status pw_selftest_slice_product(int n, int ncol, long long *mismatches, double *rel_err) {
  using namespace pw;
  if (!mismatches || !rel_err || n < 4 || n > 512 || n % 4 || ncol < 1 || ncol > 4096) return PW_EINVAL;
  const int M = 2 * n, K = 2 * n;
  const size_t asz = (size_t)RS_SLICES * M * K, bsz = (size_t)RS_SLICES * ncol * K;
  std::vector<int> IA(asz), IB(bsz);   // slice integers, |I| <= 128
  std::vector<uint16_t> HA(asz), HB(bsz);
  unsigned st = 2463534242u;
  auto rnd = [&]() {   // xorshift32
    st ^= st << 13;
    st ^= st >> 17;
    st ^= st << 5;
    return st;
  };
  auto bits = [](int I, int s) {   // BF16 pattern of I 2^-7(s+1)
    const float f = ldexpf((float)I, -RS_BITS * (s + 1));
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
  };
  pw_status res = PW_OK;
  uint16_t *dA = nullptr, *dB = nullptr;
  int *dexp = nullptr, *dstat = nullptr;
  double *dY = nullptr;
  std::vector<double> Y((size_t)M * ncol);
  if (cudaMalloc(&dA, asz * 2) || cudaMalloc(&dB, bsz * 2) || cudaMalloc(&dexp, (M + ncol) * sizeof(int)) ||
      cudaMalloc(&dstat, sizeof(int)) || cudaMalloc(&dY, Y.size() * sizeof(double))) {
    cudaGetLastError();
    res = PW_ENOMEM;
  }
  RefineArgs a;
  memset(&a, 0, sizeof(a));
  a.n = n;
  a.Osl = dA;
  a.Ysl = dB;
  a.Oexp = dexp;
  a.Yexp = dexp + M;
  a.Yacc = dY;
  a.status = dstat;
  const int tiles = ((M + RS_TILE - 1) / RS_TILE) * ((ncol + RS_TILE - 1) / RS_TILE);
  for (int pattern = 0; pattern < 2 && res == PW_OK; ++pattern) {
    // pattern 0: only the leading slices, with full-scale rows 0 (all +128) and
    // columns 0 (+128), 1 (-128) so that sums reach 2^24 units; pattern 1: every slice
    for (size_t e = 0; e < asz; ++e) {
      const int s = (int)(e / ((size_t)M * K)), r = (int)((e / K) % M);
      int I = (int)(rnd() % 257u) - 128;
      if (pattern == 0 && s > 0) I = 0;
      if (s == 0 && r == 0) I = 128;
      IA[e] = I;
      HA[e] = bits(I, s);
    }
    for (size_t e = 0; e < bsz; ++e) {
      const int t = (int)(e / ((size_t)ncol * K)), j = (int)((e / K) % ncol);
      int I = (int)(rnd() % 257u) - 128;
      if (pattern == 0 && t > 0) I = 0;
      if (t == 0 && j < 2) I = j == 0 ? 128 : -128;
      IB[e] = I;
      HB[e] = bits(I, t);
    }
    if (cudaMemcpy(dA, HA.data(), asz * 2, cudaMemcpyHostToDevice) ||
        cudaMemcpy(dB, HB.data(), bsz * 2, cudaMemcpyHostToDevice) || cudaMemset(dexp, 0, (M + ncol) * sizeof(int)) ||
        cudaMemset(dstat, 0, sizeof(int)) ||
        cudaFuncSetAttribute(k_res_mm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)res_mm_smem_bytes())) {
      res = PW_ECUDA;
      break;
    }
    k_res_mm<<<tiles, 256, res_mm_smem_bytes()>>>(a, ncol, 1);
    int hstat = 0;
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&hstat, dstat, sizeof(int), cudaMemcpyDeviceToHost) ||
        cudaMemcpy(Y.data(), dY, Y.size() * sizeof(double), cudaMemcpyDeviceToHost)) {
      res = PW_ECUDA;
      break;
    }
    if (hstat) {
      res = PW_ETIMEOUT;
      break;
    }
    if (pattern == 0) {
      // the exact product of the leading slices, an integer times 2^-14, compared bit for bit
      long long bad = 0;
      for (int r = 0; r < M; ++r)
        for (int j = 0; j < ncol; ++j) {
          long long I = 0;
          for (int k = 0; k < K; ++k) I += (long long)IA[(size_t)r * K + k] * IB[(size_t)j * K + k];
          if (Y[(size_t)j * M + r] != ldexp((double)I, -2 * RS_BITS)) ++bad;
        }
      *mismatches = bad;
    } else {
      // every pair with s + t < RS_SLICES, on rows 0, 64, 128, ...: the integer sums
      // X_d of each diagonal d = s + t are exact, their scaled sum is formed smallest first
      double num = 0.0, den = 0.0;
      for (int r = 0; r < M; r += 64)
        for (int j = 0; j < ncol; ++j) {
          long long X[RS_SLICES] = {0};
          for (int s = 0; s < RS_SLICES; ++s)
            for (int t = 0; s + t < RS_SLICES; ++t) {
              const int *pa = &IA[((size_t)s * M + r) * K], *pb = &IB[((size_t)t * ncol + j) * K];
              long long I = 0;
              for (int k = 0; k < K; ++k) I += (long long)pa[k] * pb[k];
              X[s + t] += I;
            }
          double ref = 0.0;
          for (int d = RS_SLICES - 1; d >= 0; --d) ref += ldexp((double)X[d], -RS_BITS * (d + 2));
          num = fmax(num, fabs(Y[(size_t)j * M + r] - ref));
          den = fmax(den, fabs(ref));
        }
      *rel_err = num / fmax(den, 1e-300);
    }
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dexp);
  cudaFree(dstat);
  cudaFree(dY);
  return res;
}

