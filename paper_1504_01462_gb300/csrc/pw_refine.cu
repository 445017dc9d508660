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

namespace pw {

namespace {

struct KV {   // per-interface vectors in shared memory: FP64, and FP32 copies for the FP32 passes
  zc *kinvL, *kR, *eL, *eR;
  cc *fkinvL, *fkR, *feL, *feR;
};

__device__ KV carve_kv(unsigned char *raw, size_t off, int n) {
  KV v;
  zc *c = reinterpret_cast<zc *>(raw + off);
  v.kinvL = c;
  v.kR = c + n;
  v.eL = c + 2 * n;
  v.eR = c + 3 * n;
  cc *f = reinterpret_cast<cc *>(c + 4 * n);
  v.fkinvL = f;
  v.fkR = f + n;
  v.feL = f + 2 * n;
  v.feR = f + 3 * n;
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
    const zc ki = cinv(kl), el = phase_fwd(kl, dz[p]), er = phase_fwd(kr, dz[p + 1]);
    v.kinvL[i] = ki;
    v.kR[i] = kr;
    v.eL[i] = el;
    v.eR[i] = er;
    v.fkinvL[i] = ccast<float>(ki);
    v.fkR[i] = ccast<float>(kr);
    v.feL[i] = ccast<float>(el);
    v.feR[i] = ccast<float>(er);
  }
  __syncthreads();
}

// P_lj (sel +1) or Q_lj (sel -1) in FP64 from O and the k vectors
__device__ __forceinline__ zc pq64(const zc *O, int n, int l, int j, const KV &v, double sel) {
  const zc o = O[l + (size_t)j * n];
  const zc r = cmul(v.kR[j], v.kinvL[l]);
  return cmul(o, mkc<double>(0.5 * (1.0 + sel * r.re), 0.5 * sel * r.im));
}

// The same in FP32 (the backward and forward passes apply the FP32
// preconditioner; only the residual needs FP64)
__device__ __forceinline__ cc pq32(const zc *O, const cc *O32, int n, int l, int j, const KV &v, float sel) {
  const cc o = O32 ? O32[l + (size_t)j * n] : ccast<float>(O[l + (size_t)j * n]);
  const cc r = cmul(v.fkR[j], v.fkinvL[l]);
  return cmul(o, mkc<float>(0.5f * (1.0f + sel * r.re), 0.5f * sel * r.im));
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
// Backward pass at interface p (launched for p = max N down to 0; a point
// starts at its own N):
//   da_q = Z_p (e_q db_q) + u_p,   db_p = Q_p da_q + P_p e_q db_q (+ g_p),
// accumulated into Xa[q], Xb[p]; db_p is carried to the next (left) interface.
__global__ void __launch_bounds__(NT) k_refine_backward(RefineArgs a, int p, int with_src) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const PointDesc d = a.pts[pt];
  if (d.skip || a.status[pt] || p > d.N) return;
  const int n = a.n, nc = a.nc, N = d.N, q = p + 1;
  cc *gsm = reinterpret_cast<cc *>(smraw);
  KV v = carve_kv(smraw, skinny_smem_elems<float>() * sizeof(cc), n);
  load_kv(a, d, p, v);
  const zc *O = overlap(a, d, p);
  const cc *O32 = a.O32 ? a.O32 + ((size_t)d.o_off + p) * (size_t)n * n : nullptr;
  const cc *Z = a.Zst + ((size_t)d.st_off + p) * n * n;
  const cc *U = a.Ust + ((size_t)d.st_off + p) * n * nc;
  zc *carry = a.carry + (size_t)pt * n * nc;       // db_q in, db_p out
  cc *tmp = a.tmp + (size_t)pt * 2 * n * nc;       // [da_q ; e_q db_q] as a 2n x nc block
  // e_q db_q (db_{N+1} = 0)
  for (int e = threadIdx.x; e < n * nc; e += NT) {
    const int i = e % n, c = e / n;
    const zc b = (q <= N) ? carry[e] : czero<double>();
    tmp[n + i + (size_t)c * 2 * n] = ccast<float>(cmul(v.eR[i], b));
  }
  __syncthreads();
  zc *Xa = a.Xa + blk(a, d, q);
  zc *Xb = a.Xb + blk(a, d, p);
  // da_q
  cta_gemm_skinny<float>(
      n, nc, n, [=](int i, int l) { return Z[i + (size_t)l * n]; },
      [=](int l, int j) { return tmp[n + l + (size_t)j * 2 * n]; },
      [=](int i, int j, cc acc) {
        const cc da = cadd(acc, U[i + (size_t)j * n]);
        tmp[i + (size_t)j * 2 * n] = da;
        if (q <= N || !with_src) {   // a correction of a_{N+1} was added by the forward pass
          zc &x = Xa[i + (size_t)j * n];
          x = cadd(x, ccast<double>(da));
        }
      },
      gsm);
  // db_p = [Q | P] [da_q ; e_q db_q] (+ g_p)
  const KV vc = v;
  const zc *G = a.Gr + iblk(a, d, p);
  cta_gemm_skinny<float>(
      n, nc, 2 * n,
      [=](int i, int l) { return l < n ? pq32(O, O32, n, i, l, vc, -1.0f) : pq32(O, O32, n, i, l - n, vc, 1.0f); },
      [=](int l, int j) { return tmp[l + (size_t)j * 2 * n]; },
      [=](int i, int j, cc acc) {
        zc db = ccast<double>(acc);
        if (with_src) db = cadd(db, G[i + (size_t)j * n]);
        carry[i + (size_t)j * n] = db;
        zc &x = Xb[i + (size_t)j * n];
        x = cadd(x, db);
      },
      gsm);
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
      n, 2 * nc, n, [=](int i, int l) { return dfc_of(O[i + (size_t)l * n]); },
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
// Forward correction sweep at interface p (launched for p = 0..max N):
//   u_p = W_p^{-1}(c_p + R_p g_p - f_p),  R_p = e_p Z_{p-1} e_p,  c_{p+1} = e_q u_p,
// with W_p's LU factors kept by the first sweep (an O(n^2 nc) replay).  u_p
// replaces the stored one for the backward pass.  At p = N the carry holds the
// correction of a_{N+1} (= u_N); on the last iteration (no backward pass
// follows) it is added to Xa[N+1] here.
__global__ void __launch_bounds__(NT) k_refine_forward(RefineArgs a, int p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  const PointDesc d = a.pts[pt];
  if (d.skip || a.status[pt] || p > d.N) return;
  const int n = a.n, nc = a.nc, N = d.N;
  cc *gsm = reinterpret_cast<cc *>(smraw);
  const size_t kv_off = (skinny_smem_elems<float>() + Tile<float>::NB * Tile<float>::NB) * sizeof(cc);
  KV v = carve_kv(smraw, kv_off, n);
  load_kv(a, d, p, v);
  const cc *Zprev = p > 0 ? a.Zst + ((size_t)d.st_off + p - 1) * n * n : nullptr;
  const cc *LU = a.LUst + ((size_t)d.st_off + p) * n * n;
  const int *piv = a.PIVst + ((size_t)d.st_off + p) * n;
  cc *Ust = a.Ust + ((size_t)d.st_off + p) * n * nc;
  cc *rhs = a.M + (size_t)pt * n * (n + nc);   // n x nc scratch
  zc *carry = a.carry + (size_t)pt * n * nc;   // c_p in, c_{p+1} out
  const zc *F = a.Fr + iblk(a, d, p);
  const zc *G = a.Gr + iblk(a, d, p);
  const KV vc = v;
  if (p == 0) {
    for (int e = threadIdx.x; e < n * nc; e += NT) rhs[e] = ccast<float>(csub(carry[e], F[e]));
    __syncthreads();
  } else {
    // rhs = c_p + R_p g_p - f_p
    cta_gemm_skinny<float>(
        n, nc, n,
        [=](int i, int l) {
          return cmul(cmul(vc.feL[i], Zprev[i + (size_t)l * n]), vc.feL[l]);
        },
        [=](int l, int j) { return ccast<float>(G[l + (size_t)j * n]); },
        [=](int i, int j, cc acc) {
          const zc r = csub(cadd(carry[i + (size_t)j * n], ccast<double>(acc)), F[i + (size_t)j * n]);
          rhs[i + (size_t)j * n] = ccast<float>(r);
        },
        gsm);
  }
  cta_lu_replay<float>(LU, n, piv, rhs, n, nc, gsm);
  for (int e = threadIdx.x; e < n * nc; e += NT) {
    const int i = e % n;
    const cc u = rhs[e];
    Ust[e] = u;
    carry[e] = cmul(vc.eR[i], ccast<double>(u));
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
  const size_t kv = 4 * (size_t)n * (sizeof(zc) + sizeof(cc));
  const size_t fwd = (skinny_smem_elems<float>() + Tile<float>::NB * Tile<float>::NB) * sizeof(cc) + kv;
  const size_t bwd = skinny_smem_elems<float>() * sizeof(cc) + kv;
  const size_t res = skinny_smem_elems<double>() * sizeof(zc) + kv;
  return std::max(fwd, std::max(bwd, res)) + 64;
}

cudaError_t launch_refine(const RefineArgs &a, int npts, int min_iters, int max_iters, double tol,
                          cudaStream_t s, int *passes) {
  const size_t smem = refine_smem_bytes(a.n);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_refine_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
      (e = cudaFuncSetAttribute(k_refine_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
      (e = cudaFuncSetAttribute(k_refine_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return e;
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
  for (int p = a.N; p >= 0; --p) k_refine_backward<<<npts, NT, smem, s>>>(a, p, 0);
  // stopping test: the correction of pass i shrinks the error by about
  // c_i / c_{i-1} (c = relative size of the correction of a_{N+1}), so the
  // error left after pass i is estimated as c_i^2 / c_{i-1}
  std::vector<double> corr(npts), prev(npts, 0.0);
  int it = 0;
  for (; it < max_iters; ++it) {
    k_refine_residual<<<dim3(a.N + 1, npts), NT, smem, s>>>(a);
    if ((e = cudaMemsetAsync(a.carry, 0, vec, s))) return e;
    for (int p = 0; p <= a.N; ++p) k_refine_forward<<<npts, NT, smem, s>>>(a, p);
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
    for (int p = a.N; p >= 0; --p) k_refine_backward<<<npts, NT, smem, s>>>(a, p, 1);
  }
  if (passes) *passes = it;
  k_refine_finish<<<npts, NT, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace pw
