// Periodic electrodes on the GPU, FP64 (App. B: complex band structure by the
// generalised Bloch eigenproblem Eq. cmp with the tilted cell's phases; App. C:
// the transmission between two periodic electrodes), without nonlocal terms.
//
// Amplitudes are referenced at each slice's right edge, as in the star
// products: S(c_M, c_M') of one electrode period maps (a of the reference
// slice, b of the same slice one period on) to (a one period on, b of the
// reference slice), and a Bloch state X = [a; b] with factor lambda solves
//     [[S11, 0], [S21, -1]] X = lambda [[1, -S12], [0, -S22]] X     (Eq. cmp).
// Writing the pencil as (A, B), the Cayley map mu = (lambda - s)/(lambda + s)
// with |s| = 1 takes it to the standard eigenproblem of the bounded matrix
// C = (A + sB)^{-1} (A - sB): the unit circle |lambda| = 1 goes to the
// imaginary axis, decaying states (|lambda| < 1) to Re mu < 0, growing ones
// to Re mu > 0, so the complex Schur form of C, reordered, gives orthonormal
// bases of the decaying and growing invariant subspaces without forming the
// ill-conditioned transfer matrix.  Propagating states (|lambda| within 1e-7
// of 1) are grouped by lambda (within 1e-6); each group's eigenspace comes from
// the Schur form reordered with the group first, and is split by the z-flux
// form F = (psi^H psi' - psi'^H psi) / 2i at the reference plane into
// flux-orthogonal states of unit flux, right-going for positive flux.
#include <math.h>

#include "pw_cta.cuh"
#include "pw_eig_ns.cuh"
#include "pw_internal.h"

namespace pw {

namespace {

constexpr int PT = NT;   // threads per problem

size_t band_smem_bytes() {
  return (gemm_smem_elems<double>() + (size_t)Tile<double>::NB * Tile<double>::NB) * sizeof(zc) +
         32 * sizeof(double) + 64 * sizeof(int) + (PT + 16) * sizeof(double) + 64;
}

struct BandSmem {
  zc *gemm;
  double *sval;
  int *sidx, *flag;
  double *red, *rs;
};
__device__ BandSmem band_carve(unsigned char *raw) {
  BandSmem s;
  zc *c = reinterpret_cast<zc *>(raw);
  s.gemm = c;
  c += gemm_smem_elems<double>() + Tile<double>::NB * Tile<double>::NB;
  s.sval = reinterpret_cast<double *>(c);
  s.sidx = reinterpret_cast<int *>(s.sval + 32);
  s.flag = s.sidx + 32;
  s.red = reinterpret_cast<double *>(s.flag + 32);
  s.rs = s.red + PT + 8;
  return s;
}

// Cyclic Jacobi eigen-decomposition of the Hermitian g x g matrix F (row-major,
// g <= 8), one thread: F <- diag(w), V (row-major) the eigenvectors as columns.
__device__ void jacobi_herm(zc *F, zc *V, int g) {
  for (int i = 0; i < g; ++i)
    for (int j = 0; j < g; ++j) V[i * g + j] = mkc<double>(i == j ? 1.0 : 0.0, 0.0);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < g; ++p)
      for (int q = p + 1; q < g; ++q) off += cnorm2(F[p * g + q]);
    if (off < 1e-30) break;
    for (int p = 0; p < g; ++p)
      for (int q = p + 1; q < g; ++q) {
        const zc c = F[p * g + q];
        const double ac = hypot(c.re, c.im);
        if (ac < 1e-300) continue;
        const double app = F[p * g + p].re, aqq = F[q * g + q].re;
        // rotate by R = [[cs, -sn conj(e)], [sn e, cs]] with e = c/|c| so that (R^H F R)_pq = 0
        const double th = 0.5 * atan2(2.0 * ac, aqq - app);
        const double cs = cos(th), sn = sin(th);
        const zc e = mkc<double>(c.re / ac, c.im / ac);
        for (int k = 0; k < g; ++k) {   // columns p, q of F and V
          const zc fp = F[k * g + p], fq = F[k * g + q];
          F[k * g + p] = csub(cscale(cs, fp), cscale(sn, cmul(cconj(e), fq)));
          F[k * g + q] = cadd(cscale(sn, cmul(e, fp)), cscale(cs, fq));
          const zc vp = V[k * g + p], vq = V[k * g + q];
          V[k * g + p] = csub(cscale(cs, vp), cscale(sn, cmul(cconj(e), vq)));
          V[k * g + q] = cadd(cscale(sn, cmul(e, vp)), cscale(cs, vq));
        }
        for (int k = 0; k < g; ++k) {   // rows p, q of F
          const zc fp = F[p * g + k], fq = F[q * g + k];
          F[p * g + k] = csub(cscale(cs, fp), cscale(sn, cmul(e, fq)));
          F[q * g + k] = cadd(cscale(sn, cmul(cconj(e), fp)), cscale(cs, fq));
        }
      }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Self-test of the team eigen-kernels: Schur form of one N x N matrix, then
// (sel) the entries with Re < 0 moved first.  One CTA; out: T, Z, count.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PT) k_schur_test(zc *A, zc *Z, zc *v, int N, int sel, int *keys, int *out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  BandSmem s = band_carve(smraw);
  ns::Team t{(int)threadIdx.x, PT, s.red};
  for (size_t e = threadIdx.x; e < (size_t)N * N; e += PT) Z[e] = mkc<double>((e % N) == (e / N) ? 1.0 : 0.0, 0.0);
  t.sync();
  ns::hessenberg(t, A, Z, N, v);
  const bool ok = ns::schur(t, A, Z, N, s.rs);
  int cnt = 0;
  if (ok && sel) {
    if (threadIdx.x == 0)
      for (int i = 0; i < N; ++i) keys[i] = A[i + (size_t)i * N].re < 0.0 ? 0 : 1;
    t.sync();
    cnt = ns::schur_select(t, A, Z, N, keys, s.rs);
  }
  if (threadIdx.x == 0) {
    out[0] = ok ? 1 : 0;
    out[1] = cnt;
  }
}

// ---------------------------------------------------------------------------
// Complex bands of one electrode cell per problem (one CTA each).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PT) k_cbands(BandArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  BandSmem s = band_carve(smraw);
  const int b = blockIdx.x, n = a.n, N2 = 2 * n;
  const size_t NN = (size_t)N2 * N2, nn = (size_t)n * n;
  ns::Team t{(int)threadIdx.x, PT, s.red};
  zc *W = a.work + (size_t)b * band_work_elems(n);
  zc *Aug = W, *T = Aug + 2 * NN, *Z = T + NN, *T0 = Z + NN, *Z0 = T0 + NN, *T2 = Z0 + NN, *Z2 = T2 + NN;
  zc *v = Z2 + NN;
  double *lam = reinterpret_cast<double *>(v + N2);   // 2 N2: lambda (re, im)
  int *keys = a.keys + (size_t)b * 4 * N2;             // class, selection keys, group members
  int *key2 = keys + N2, *grp = keys + 2 * N2, *gl = keys + 3 * N2;
  const zc *S11 = a.S + (size_t)b * 4 * nn, *S12 = S11 + nn, *S21 = S12 + nn, *S22 = S21 + nn;
  const zc sg = mkc<double>(cos(0.7), sin(0.7));   // |s| = 1, away from the real axis
  int *status = a.status + b;
  if (threadIdx.x == 0) { *s.flag = 0; *status = 0; }
  // [A + sB | A - sB],  A = [[S11, 0], [S21, -1]],  B = [[1, -S12], [0, -S22]]
  for (size_t e = threadIdx.x; e < 2 * NN; e += PT) {
    const int r = (int)(e % N2), c = (int)(e / N2);
    const bool minus = c >= N2;
    const int cc_ = minus ? c - N2 : c;
    const zc sgn = minus ? mkc<double>(-sg.re, -sg.im) : sg;
    const int br = r / n, bc = cc_ / n, i = r % n, j = cc_ % n;
    const double id = i == j ? 1.0 : 0.0;
    zc Av, Bv;
    if (br == 0 && bc == 0) { Av = S11[i + (size_t)j * n]; Bv = mkc<double>(id, 0.0); }
    else if (br == 0) { Av = czero<double>(); Bv = cscale(-1.0, S12[i + (size_t)j * n]); }
    else if (bc == 0) { Av = S21[i + (size_t)j * n]; Bv = czero<double>(); }
    else { Av = mkc<double>(-id, 0.0); Bv = cscale(-1.0, S22[i + (size_t)j * n]); }
    Aug[e] = cadd(Av, cmul(sgn, Bv));
  }
  __syncthreads();
  cta_lu_solve<double>(Aug, N2, N2, 2 * N2, a.ipiv + (size_t)b * N2, s.gemm, s.sval, s.sidx, s.flag);
  if (*s.flag & 1) {
    if (threadIdx.x == 0) *status = 1;
    return;
  }
  for (size_t e = threadIdx.x; e < NN; e += PT) {
    T[e] = Aug[NN + e];
    Z[e] = mkc<double>((e % N2) == (e / N2) ? 1.0 : 0.0, 0.0);
  }
  t.sync();
  ns::hessenberg(t, T, Z, N2, v);
  if (!ns::schur(t, T, Z, N2, s.rs)) {
    if (threadIdx.x == 0) *status = 2;
    return;
  }
  // classes: 0 decaying (|lambda| < 1), 1 propagating, 2 growing
  if (threadIdx.x == 0) {
    for (int i = 0; i < N2; ++i) {
      const zc mu = T[i + (size_t)i * N2];
      const zc den = mkc<double>(1.0 - mu.re, -mu.im);
      double m = INFINITY;
      zc l = mkc<double>(INFINITY, 0.0);
      if (cabs1(den) > 1e-300) {
        l = cmul(sg, cdiv(mkc<double>(1.0 + mu.re, mu.im), den));
        m = hypot(l.re, l.im);
      }
      keys[i] = m < 1.0 - 1e-7 ? 0 : (m > 1.0 + 1e-7 ? 2 : 1);
      lam[2 * i] = l.re;
      lam[2 * i + 1] = l.im;
    }
  }
  t.sync();
  for (size_t e = threadIdx.x; e < NN; e += PT) { T0[e] = T[e]; Z0[e] = Z[e]; }
  t.sync();
  const size_t st = (size_t)b * 4 * nn;
  zc *aR = a.states + st, *bR = aR + nn, *aL = bR + nn, *bL = aL + nn;
  int *prop = a.prop + (size_t)b * N2;
  for (int e = threadIdx.x; e < N2; e += PT) prop[e] = 0;
  // decaying subspace: class 0 first
  if (threadIdx.x == 0)
    for (int i = 0; i < N2; ++i) key2[i] = keys[i] == 0 ? 0 : 1;
  t.sync();
  const int ndec = ns::schur_select(t, T, Z, N2, key2, s.rs);
  for (size_t e = threadIdx.x; e < (size_t)n * min(ndec, n); e += PT) {
    const int i = (int)(e % n), c = (int)(e / n);
    aR[i + (size_t)c * n] = Z[i + (size_t)c * N2];
    bR[i + (size_t)c * n] = Z[n + i + (size_t)c * N2];
  }
  // growing subspace: class 2 first (from the unordered form)
  t.sync();
  for (size_t e = threadIdx.x; e < NN; e += PT) { T[e] = T0[e]; Z[e] = Z0[e]; }
  if (threadIdx.x == 0)
    for (int i = 0; i < N2; ++i) key2[i] = keys[i] == 2 ? 0 : 1;
  t.sync();
  const int ngrow = ns::schur_select(t, T, Z, N2, key2, s.rs);
  for (size_t e = threadIdx.x; e < (size_t)n * min(ngrow, n); e += PT) {
    const int i = (int)(e % n), c = (int)(e / n);
    aL[i + (size_t)c * n] = Z[i + (size_t)c * N2];
    bL[i + (size_t)c * n] = Z[n + i + (size_t)c * N2];
  }
  t.sync();
  // propagating groups
  if (threadIdx.x == 0) {
    for (int i = 0; i < N2; ++i) grp[i] = -1;
    int ng = 0;
    for (int i = 0; i < N2; ++i) {
      if (keys[i] != 1 || grp[i] >= 0) continue;
      for (int j = i; j < N2; ++j)
        if (keys[j] == 1 && grp[j] < 0 && hypot(lam[2 * j] - lam[2 * i], lam[2 * j + 1] - lam[2 * i + 1]) < 1e-6)
          grp[j] = ng;
      ++ng;
    }
    gl[0] = ng;
  }
  t.sync();
  const int ngroups = gl[0];
  int nR = min(ndec, n), nL = min(ngrow, n);
  const double *Eref = a.Eref + (a.ref_shared ? 0 : (size_t)b * n);
  const zc *U = a.Uref + (a.ref_shared ? 0 : (size_t)b * nn);
  const double E = a.E[b];
  for (int gi = 0; gi < ngroups; ++gi) {
    for (size_t e = threadIdx.x; e < NN; e += PT) { T2[e] = T0[e]; Z2[e] = Z0[e]; }
    if (threadIdx.x == 0)
      for (int i = 0; i < N2; ++i) key2[i] = grp[i] == gi ? 0 : 1;
    t.sync();
    const int g = ns::schur_select(t, T2, Z2, N2, key2, s.rs);
    if (threadIdx.x == 0) {
      // flux form of the group's orthonormal basis X = Z2[:, 0:g] at the reference plane
      zc F[64], V[64];
      const int gg = min(g, 8);
      for (int p = 0; p < gg; ++p)
        for (int q = 0; q < gg; ++q) {
          // psi = U (a + b), dpsi = i U K (a - b); F_pq = (psi_p^H dpsi_q - dpsi_p^H psi_q) / 2i
          zc acc = czero<double>();
          for (int r = 0; r < n; ++r) {
            zc pp = czero<double>(), dp = czero<double>(), pq = czero<double>(), dq = czero<double>();
            for (int l = 0; l < n; ++l) {
              const zc u = U[r + (size_t)l * n];
              const zc k = kz_branch(E, Eref[l]);
              const zc ap = Z2[l + (size_t)p * N2], bp = Z2[n + l + (size_t)p * N2];
              const zc aq = Z2[l + (size_t)q * N2], bq = Z2[n + l + (size_t)q * N2];
              cfma(pp, u, cadd(ap, bp));
              cfma(pq, u, cadd(aq, bq));
              const zc ik = mkc<double>(-k.im, k.re);
              cfma(dp, u, cmul(ik, csub(ap, bp)));
              cfma(dq, u, cmul(ik, csub(aq, bq)));
            }
            acc = cadd(acc, csub(cmul(cconj(pp), dq), cmul(cconj(dp), pq)));
          }
          // divide by 2i
          F[p * gg + q] = mkc<double>(0.5 * acc.im, -0.5 * acc.re);
        }
      for (int p = 0; p < gg; ++p)
        for (int q = p; q < gg; ++q) {
          const zc h = cscale(0.5, cadd(F[p * gg + q], cconj(F[q * gg + p])));
          F[p * gg + q] = h;
          F[q * gg + p] = cconj(h);
        }
      jacobi_herm(F, V, gg);
      for (int c = 0; c < gg; ++c) {
        const double w = F[c * gg + c].re;
        if (fabs(w) < 1e-12) { *status = 4; continue; }
        const double sc = 1.0 / sqrt(fabs(w));
        const bool right = w > 0.0;
        const int col = right ? nR++ : nL++;
        if (col >= n) { *status = 3; continue; }
        zc *da = right ? aR : aL, *db = right ? bR : bL;
        for (int r = 0; r < n; ++r) {
          zc xa = czero<double>(), xb = czero<double>();
          for (int q = 0; q < gg; ++q) {
            cfma(xa, Z2[r + (size_t)q * N2], V[q * gg + c]);
            cfma(xb, Z2[n + r + (size_t)q * N2], V[q * gg + c]);
          }
          da[r + (size_t)col * n] = cscale(sc, xa);
          db[r + (size_t)col * n] = cscale(sc, xb);
        }
        prop[(right ? 0 : n) + col] = 1;
      }
      if (g > 8) *status = 3;
      gl[1] = nR;
      gl[2] = nL;
    }
    t.sync();
    nR = gl[1];
    nL = gl[2];
  }
  if (threadIdx.x == 0 && *status == 0 && (nR != n || nL != n)) *status = 3;
}

__host__ __device__ size_t band_work_elems(int n) {
  const size_t N2 = 2 * (size_t)n, NN = N2 * N2;
  return 2 * NN + 6 * NN + N2 + N2;   // Aug, T, Z, T0, Z0, T2, Z2, v, lambda
}

cudaError_t launch_cbands(const BandArgs &a, cudaStream_t s) {
  const size_t sm = band_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_cbands, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_cbands<<<a.nprob, PT, sm, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The transmission between the periodic electrodes per point (one CTA each):
// with S = S(c_M, r_1) of [left reference slice, device, right reference
// slice], the unknowns beta (left-going states of the left electrode) and
// gamma (right-going states of the right electrode) solve
//   [[-S11 aL, cR - S12 dR], [bL - S21 aL, -S22 dR]] [beta; gamma]
//       = [S11 aR_alpha; S21 aR_alpha - bR_alpha]
// for the incident propagating right-going states alpha of the left
// electrode, and T = sum |gamma|^2 over the right electrode's propagating
// right-going states (all states have unit flux).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PT) k_periodic_solve(PeriodicArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  BandSmem s = band_carve(smraw);
  const int pt = blockIdx.x, n = a.n, N2 = 2 * n;
  const size_t nn = (size_t)n * n;
  const zc *S11 = a.Sdev + (size_t)pt * 4 * nn, *S12 = S11 + nn, *S21 = S12 + nn, *S22 = S21 + nn;
  const zc *L = a.statesL + (size_t)pt * 4 * nn, *R = a.statesR + (size_t)pt * 4 * nn;
  const zc *aR = L, *bR = L + nn, *aL = L + 2 * nn, *bL = L + 3 * nn;
  const zc *cR = R, *dR = R + nn;
  const int *propL = a.propL + (size_t)pt * N2, *propR = a.propR + (size_t)pt * N2;
  __shared__ int alpha[64];
  __shared__ int na;
  if (threadIdx.x == 0) {
    *s.flag = 0;
    int c = 0;
    for (int j = 0; j < n && c < 64; ++j)
      if (propL[j]) alpha[c++] = j;
    na = c;
    if (a.bad[pt]) na = -1;
  }
  __syncthreads();
  if (na < 0) {
    if (threadIdx.x == 0) a.T[a.out[pt]] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  if (na == 0) {
    if (threadIdx.x == 0) a.T[a.out[pt]] = 0.0;
    return;
  }
  zc *M = a.work + (size_t)pt * N2 * (N2 + 64);   // [M | rhs], 2n x (2n + na)
  const int ncols = N2 + na;
  // -S11 aL, -S21 aL into columns 0..n-1; -S12 dR, -S22 dR into n..2n-1
  // [[S11, S12], [S21, S22]] times the block diagonal [[aL, 0], [0, dR]]
  cta_gemm<double>(
      N2, N2, N2,
      [=](int i, int l) {
        const zc *blk = i < n ? (l < n ? S11 : S12) : (l < n ? S21 : S22);
        return blk[(i % n) + (size_t)(l % n) * n];
      },
      [=](int l, int j) {
        if (l < n && j < n) return aL[l + (size_t)j * n];
        if (l >= n && j >= n) return dR[l - n + (size_t)(j - n) * n];
        return czero<double>();
      },
      [=](int i, int j, zc acc) {
        zc v = cscale(-1.0, acc);
        if (j < n && i >= n) v = cadd(v, bL[i - n + (size_t)j * n]);
        if (j >= n && i < n) v = cadd(v, cR[i + (size_t)(j - n) * n]);
        M[i + (size_t)j * N2] = v;
      },
      s.gemm);
  cta_gemm<double>(
      N2, na, n, [=](int i, int l) { return i < n ? S11[i + (size_t)l * n] : S21[i - n + (size_t)l * n]; },
      [=](int l, int j) { return aR[l + (size_t)alpha[j] * n]; },
      [=](int i, int j, zc acc) {
        M[i + (size_t)(N2 + j) * N2] = i < n ? acc : csub(acc, bR[i - n + (size_t)alpha[j] * n]);
      },
      s.gemm);
  cta_lu_solve<double>(M, N2, N2, ncols, a.ipiv + (size_t)pt * N2, s.gemm, s.sval, s.sidx, s.flag);
  if (*s.flag & 1) {
    if (threadIdx.x == 0) a.T[a.out[pt]] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  double acc = 0.0;
  for (int e = threadIdx.x; e < n * na; e += PT) {
    const int i = e % n, j = e / n;
    if (propR[i]) acc += cnorm2(M[n + i + (size_t)(N2 + j) * N2]);
  }
  acc = ns::Team{(int)threadIdx.x, PT, s.red}.sum(acc);
  if (threadIdx.x == 0) a.T[a.out[pt]] = acc;
}

size_t periodic_work_elems(int n) { return 2 * (size_t)n * (2 * (size_t)n + 64); }

cudaError_t launch_periodic_solve(const PeriodicArgs &a, int npts, cudaStream_t s) {
  const size_t sm = band_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_periodic_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_periodic_solve<<<npts, PT, sm, s>>>(a);
  return cudaGetLastError();
}

// modes of a moved cell: U'(G, j) = e^{-i G.a3} U(G, j) (count matrices)
__global__ void k_tilt_modes(const zc *U, zc *Ut, const double *G, double ax, double ay, int n, int count) {
  const size_t tot = (size_t)count * n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(e % n);
    double sn, cs;
    sincos(G[2 * g] * ax + G[2 * g + 1] * ay, &sn, &cs);
    Ut[e] = cmul(U[e], mkc<double>(cs, -sn));
  }
}

cudaError_t launch_tilt_modes(const zc *U, zc *Ut, const double *G, double ax, double ay, int n, int count,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_tilt_modes<<<256, 256, 0, s>>>(U, Ut, G, ax, ay, n, count);
  return cudaGetLastError();
}

cudaError_t schur_selftest(zc *A, zc *Z, zc *v, int N, int sel, int *keys, int *out) {
  const size_t sm = band_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_schur_test, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_schur_test<<<1, PT, sm>>>(A, Z, v, N, sel, keys, out);
  return cudaGetLastError();
}

}  // namespace pw

// Self-test of the team eigen-kernels on one N x N matrix (host in / out).
extern "C" pw_status pw_selftest_schur(int N, const pw_c128 *A_host, pw_c128 *T_host, pw_c128 *Z_host, int select,
                                       int *count) {
  using namespace pw;
  if (N < 1 || N > 1024 || !A_host || !T_host || !Z_host || !count) return PW_EINVAL;
  const size_t NN = (size_t)N * N;
  zc *A = nullptr, *Z = nullptr, *v = nullptr;
  int *keys = nullptr, *out = nullptr;
  if (cudaMalloc(&A, NN * sizeof(zc)) || cudaMalloc(&Z, NN * sizeof(zc)) || cudaMalloc(&v, N * sizeof(zc)) ||
      cudaMalloc(&keys, N * sizeof(int)) || cudaMalloc(&out, 2 * sizeof(int))) {
    cudaGetLastError();
    cudaFree(A); cudaFree(Z); cudaFree(v); cudaFree(keys); cudaFree(out);
    return PW_ENOMEM;
  }
  int h[2] = {0, 0};
  cudaError_t e = cudaMemcpy(A, A_host, NN * sizeof(zc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = schur_selftest(A, Z, v, N, select, keys, out);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(T_host, A, NN * sizeof(zc), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(Z_host, Z, NN * sizeof(zc), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h, out, 2 * sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(A); cudaFree(Z); cudaFree(v); cudaFree(keys); cudaFree(out);
  if (e != cudaSuccess) return PW_ECUDA;
  *count = h[1];
  return h[0] ? PW_OK : PW_ENOTCONV;
}
