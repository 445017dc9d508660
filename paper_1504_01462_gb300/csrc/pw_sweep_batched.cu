// Batched launch sequence of the sweep (the production path of
// pw_transmission).  One interface step of App. A Eqs. transfer / scatter and
// Eq. recurrence (the fused update in pw_sweep.cu) is split into phases, each a
// launch over (output tiles) x (points), so every phase fills the GPU:
//   vectors   k^p, k^{p+1}, E+ per point            (p = 0 also seeds [P|-Q|I])
//   wy        [W | Y] = [P | -Q] + [-R Q | R P]     (GEMM tiles x points)
//   panel     LU panel with row pivoting + U12       (one CTA per point)
//   trail     trailing update of the panel           (GEMM tiles x points)
//   bs_diag   diagonal block of the back substitution
//   bs_upd    back-substitution update               (GEMM tiles x points)
//   finish    R <- E+ Z_Y E+, Tacc <- E+ Z_T, refinement storage, t and T
// In the FP64 form the arithmetic of each element is the same as in the
// one-CTA-per-point kernel (same tile loops and accumulation order).  The
// tensor-core FP32 form takes the LU's 32-column panels and the back
// substitution's 32-row blocks in pairs, so that its wide updates run with
// K = 64 (see the panel loop and the back substitution in sweep_step).
#include <math.h>
#include <stdio.h>

#include <type_traits>

#include "pw_cta.cuh"
#include "pw_internal.h"
#include "pw_tc.cuh"

namespace pw {

namespace {

constexpr int VT = 256;   // threads of the per-point vector phases (vectors, finish)

// Shared memory of kb_panel ahead of the staged panel: L11, the arg-max
// scratch and the zero-pivot flag (rounded to 16 bytes).
template <typename T, int BT>
__host__ __device__ constexpr size_t panel_head_bytes() {
  return ((size_t)Tile<T, BT>::NB * Tile<T, BT>::NB * sizeof(cx<T>) + 40 * sizeof(T) + 96 * sizeof(int) + 15) &
         ~size_t(15);
}

int g_smem_optin = 0;   // opt-in shared memory per block of the device (set by prepare)
// kb_panel's static shared memory (the row-swap fold of the pair's L swap)
// comes out of the same per-block limit as its staged panel
constexpr size_t PANEL_STATIC_RESERVE = 1024;
constexpr int FINISH_BLOCKS = 8;   // blocks per point of kb_finish

template <typename T>
struct KVb {
  const cx<T> *kinvL, *kR, *ep;
};

template <typename T>
__device__ __forceinline__ KVb<T> kv_of(const SweepArgs &a, int pt) {
  const cx<T> *base = reinterpret_cast<const cx<T> *>(a.KV) + (size_t)pt * 3 * a.n;
  return KVb<T>{base, base + a.n, base + 2 * a.n};
}

// P_lj (sel +1) or Q_lj (sel -1); `tr` reads the overlap transposed.  The FP32
// kernels read the FP32 copy O32 of the overlaps when there is one.
template <typename T>
__device__ __forceinline__ cx<T> pqb(const zc *O, const cc *O32, int n, int l, int j, const KVb<T> &v, T sel,
                                     bool tr = false) {
  const size_t e = tr ? j + (size_t)l * n : l + (size_t)j * n;
  const cx<T> o = (std::is_same<T, float>::value && O32) ? ccast<T>(O32[e]) : ccast<T>(O[e]);
  const cx<T> r = cmul(v.kR[j], v.kinvL[l]);
  return cmul(o, mkc<T>(T(0.5) * (T(1) + sel * r.re), T(0.5) * sel * r.im));
}

// Points whose problem ended at an earlier interface (a.p > N of the point)
// take no part in the remaining steps.
// P_lj (sel +1) or Q_lj (sel -1) from the transposed FP32 overlaps Ot[j + l n]
__device__ __forceinline__ cc pqt(const cc *Ot, int n, int l, int j, const KVb<float> &v, float sel) {
  const cc o = Ot[j + (size_t)l * n];
  const cc r = cmul(v.kR[j], v.kinvL[l]);
  return cmul(o, mkc<float>(0.5f * (1.f + sel * r.re), 0.5f * sel * r.im));
}

__device__ __forceinline__ bool inactive(const SweepArgs &a, int pt) {
  const PointDesc &d = a.pts[pt];
  return d.skip || a.status[pt] || a.p > d.N;
}

// Slice q and interface p of the problem being swept.  The mirrored problem
// (slices in reverse order, overlaps transposed) is the transposed problem
// (H_p -> H_p^T = conj(H_p), eigenvectors conj(U_p), overlaps conj(O_p))
// seen from the right electrode: its interface p joins original slices
// N+1-p and N-p, whose overlap conj(U_{N+1-p})^H conj(U_{N-p}) = O_{N-p}^T.
__device__ __forceinline__ int slice_of(const SweepArgs &a, const PointDesc &d, int q) {
  return a.mirror ? d.N + 1 - q : q;
}
__device__ __forceinline__ const double *energies_of(const SweepArgs &a, const PointDesc &d, int q) {
  return a.En + ((size_t)d.en_off + slice_of(a, d, q)) * a.n;
}
__device__ __forceinline__ const zc *overlap_of(const SweepArgs &a, const PointDesc &d, int p) {
  return a.O + ((size_t)d.o_off + (a.mirror ? d.N - p : p)) * a.n * a.n;
}
__device__ __forceinline__ const cc *overlap32_of(const SweepArgs &a, const PointDesc &d, int p) {
  return a.O32 ? a.O32 + ((size_t)d.o_off + (a.mirror ? d.N - p : p)) * a.n * a.n : nullptr;
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(VT) kb_vectors(SweepArgs a, int p) {
  const int pt = blockIdx.x;
  if (inactive(a, pt)) return;
  const PointDesc d = a.pts[pt];
  const int n = a.n, nc = a.nc, ncols = 2 * n + nc;
  const double *Ep = energies_of(a, d, p);
  const double *Eq = energies_of(a, d, p + 1);
  cx<T> *kv = reinterpret_cast<cx<T> *>(a.KV) + (size_t)pt * 3 * n;
  const double dz = a.dz[d.dz_off + slice_of(a, d, p + 1)];
  for (int i = threadIdx.x; i < n; i += VT) {
    const zc kl = kz_branch(d.E, Ep[i]);
    const zc kr = kz_branch(d.E, Eq[i]);
    kv[i] = ccast<T>(cinv(kl));
    kv[n + i] = ccast<T>(kr);
    kv[2 * n + i] = ccast<T>(phase_fwd(kr, dz));
  }
  if (p != 0) return;
  __syncthreads();
  // S(0,0) = I: R = 0, Tacc = the open left columns of I  ->  W = P, Y = -Q
  const zc *O = overlap_of(a, d, 0);
  const cc *O32 = overlap32_of(a, d, 0);
  const bool tr = a.mirror != 0;
  const KVb<T> v = kv_of<T>(a, pt);
  cx<T> *M = reinterpret_cast<cx<T> *>(a.M) + (size_t)pt * n * ncols;
  for (size_t e = threadIdx.x; e < (size_t)n * ncols; e += VT) {
    const int i = e % n, j = e / n;
    cx<T> val;
    if (j < n) val = pqb<T>(O, O32, n, i, j, v, T(1), tr);
    else if (j < 2 * n) { val = pqb<T>(O, O32, n, i, j - n, v, T(-1), tr); val.re = -val.re; val.im = -val.im; }
    else { const int c = j - 2 * n; val = mkc<T>((i == c && c < d.nL) ? T(1) : T(0), T(0)); }
    M[e] = val;
  }
}

template <typename T, int BT>
__global__ void __launch_bounds__(BT) kb_wy(SweepArgs a, int p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const PointDesc d = a.pts[pt];
  const int n = a.n, ncols = 2 * n + a.nc;
  const zc *O = overlap_of(a, d, p);
  const cc *O32 = overlap32_of(a, d, p);
  const bool tr = a.mirror != 0;
  const cx<T> *R = reinterpret_cast<const cx<T> *>(a.R) + (size_t)pt * n * n;
  cx<T> *M = reinterpret_cast<cx<T> *>(a.M) + (size_t)pt * n * ncols;
  // the point's 1/k^p and k^{p+1} staged in shared memory for the operand loads
  cx<T> *gsm = reinterpret_cast<cx<T> *>(smraw);
  cx<T> *skinv = gsm + gemm_smem_elems<T, BT>();
  cx<T> *skr = skinv + n;
  const KVb<T> g = kv_of<T>(a, pt);
  for (int i = threadIdx.x; i < n; i += BT) {
    skinv[i] = g.kinvL[i];
    skr[i] = g.kR[i];
  }
  __syncthreads();
  const KVb<T> v{skinv, skr, nullptr};
  cta_gemm_t<T, Tile<T, BT>::BM, Tile<T, BT>::BN, Tile<T, BT>::BK, 4, BT>(
      n, 2 * n, n, [=](int i, int l) { return R[i + (size_t)l * n]; },
      [=](int l, int j) {
        return j < n ? pqb<T>(O, O32, n, l, j, v, T(-1), tr) : pqb<T>(O, O32, n, l, j - n, v, T(1), tr);
      },
      [=](int i, int j, cx<T> acc) {
        if (j < n) M[i + (size_t)j * n] = csub(pqb<T>(O, O32, n, i, j, v, T(1), tr), acc);
        else M[i + (size_t)j * n] = csub(acc, pqb<T>(O, O32, n, i, j - n, v, T(-1), tr));
      },
      gsm, blockIdx.x, gridDim.x);
}

// The GEMM phases of the FP32 sweep on the fifth-generation tensor cores
// (tc::cgemm_tile: TF32 hi/lo split, FP32 accumulation in tensor memory).
// Grid (64-row x 128-column output tiles, points), CG_THREADS threads.
size_t wy_tc_smem_bytes(int n) { return tc::cg_smem_bytes() + 2 * (size_t)n * sizeof(cc); }

// [W | Y] = [P | -Q] + [-R Q | R P]
__global__ void __launch_bounds__(tc::CG_THREADS) kb_wy_tc(SweepArgs a, int p) {
  extern __shared__ __align__(128) unsigned char smtc[];
  unsigned char *smraw = smtc;
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const PointDesc d = a.pts[pt];
  const int n = a.n, ncols = 2 * n + a.nc;
  const int tiles_m = (n + tc::CG_M / 2 - 1) / (tc::CG_M / 2);
  const int r0 = (blockIdx.x % tiles_m) * (tc::CG_M / 2), c0 = (blockIdx.x / tiles_m) * tc::CG_N;
  const zc *O = overlap_of(a, d, p);
  const bool tr = a.mirror != 0;
  const cc *R = reinterpret_cast<const cc *>(a.R) + (size_t)pt * n * n;
  cc *M = reinterpret_cast<cc *>(a.M) + (size_t)pt * n * ncols;
  cc *skinv = reinterpret_cast<cc *>(smraw + tc::cg_smem_bytes());
  cc *skr = skinv + n;
  const KVb<float> g = kv_of<float>(a, pt);
  for (int i = threadIdx.x; i < n; i += tc::CG_THREADS) {
    skinv[i] = g.kinvL[i];
    skr[i] = g.kR[i];
  }
  __syncthreads();
  const KVb<float> v{skinv, skr, nullptr};
  const cc *O32 = overlap32_of(a, d, p);
  // B(l, j) from the transposed FP32 copy (consecutive j contiguous for fixed l:
  // one column per thread, coalesced across the warp) when the k-set has one
  const cc *Ot = (a.O32t && !tr) ? a.O32t + ((size_t)d.o_off + p) * n * n : nullptr;
  const bool ok = tc::cgemm_tile<false, false>(
      n, 2 * n, n, r0, c0, [=](int i, int l) { return R[i + (size_t)l * n]; },
      [=](int l, int j) {
        if (Ot) return j < n ? pqt(Ot, n, l, j, v, -1.f) : pqt(Ot, n, l, j - n, v, 1.f);
        return j < n ? pqb<float>(O, O32, n, l, j, v, -1.f, tr) : pqb<float>(O, O32, n, l, j - n, v, 1.f, tr);
      },
      [=](int, int) { return czero<float>(); },
      [=](int i, int j, cc acc, cc) {
        if (j < n) M[i + (size_t)j * n] = csub(pqb<float>(O, O32, n, i, j, v, 1.f, tr), acc);
        else M[i + (size_t)j * n] = csub(acc, pqb<float>(O, O32, n, i, j - n, v, -1.f, tr));
      },
      smraw);
  if (!ok && threadIdx.x == 0) a.status[pt] = 2;
}

// [W | Y] for two points that share their overlaps (same k-set, same slices):
// with P = (O + K_L^{-1} O K_R)/2 and Q = (O - K_L^{-1} O K_R)/2 (K_L^{-1} =
// diag(kinvL), K_R = diag(kR)),
//   R Q = (X1 - X2 K_R)/2,  R P = (X1 + X2 K_R)/2,  X1 = R O,  X2 = (R K_L^{-1}) O,
// so the four products X1, X2 of both points share the B operand O (one tile
// staged per four A tiles).  W = P - R Q, Y = R P - Q are formed in the
// epilogue.  Grid (64-row x 128-column tiles of the n x n products, point
// pairs); one CTA per SM (the four accumulators fill tensor memory).
size_t wy2_tc_smem_bytes(int n) { return tc::c4_smem_bytes() + 4 * (size_t)n * sizeof(cc); }

__global__ void __launch_bounds__(tc::CG_THREADS, 1) kb_wy2_tc(SweepArgs a, int p, int npts) {
  extern __shared__ __align__(128) unsigned char smtc[];
  unsigned char *smraw = smtc;
  const int pt0 = 2 * blockIdx.y, pt1 = pt0 + 1;
  const bool act0 = !inactive(a, pt0), act1 = pt1 < npts && !inactive(a, pt1);
  if (!act0 && !act1) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  const int tiles_m = (n + tc::CG_M / 2 - 1) / (tc::CG_M / 2);
  const int r0 = (blockIdx.x % tiles_m) * (tc::CG_M / 2), c0 = (blockIdx.x / tiles_m) * tc::CG_N;
  const PointDesc d = a.pts[act0 ? pt0 : pt1];   // both points have this one's overlaps
  const bool tr = a.mirror != 0;
  const int pi = tr ? d.N - p : p;
  const zc *O = overlap_of(a, d, p);
  const cc *O32 = overlap32_of(a, d, p);
  const cc *O32t = a.O32t ? a.O32t + ((size_t)d.o_off + pi) * n * n : nullptr;
  // the (possibly transposed) overlap, element (l, j) of the product's O
  auto ov = [=](int l, int j) -> cc {
    if (tr) {
      if (O32) return tc::ldg_cc(O32 + j + (size_t)l * n);
      return ccast<float>(O[j + (size_t)l * n]);
    }
    if (O32t) return tc::ldg_cc(O32t + j + (size_t)l * n);
    if (O32) return tc::ldg_cc(O32 + l + (size_t)j * n);
    return ccast<float>(O[l + (size_t)j * n]);
  };
  // the same element read along a column (consecutive l contiguous)
  auto ovc = [=](int l, int j) -> cc {
    if (tr) {
      if (O32t) return O32t[l + (size_t)j * n];
      if (O32) return O32[j + (size_t)l * n];
      return ccast<float>(O[j + (size_t)l * n]);
    }
    if (O32) return O32[l + (size_t)j * n];
    return ccast<float>(O[l + (size_t)j * n]);
  };
  const cc *R0 = reinterpret_cast<const cc *>(a.R) + (size_t)pt0 * n * n;
  const cc *R1 = reinterpret_cast<const cc *>(a.R) + (size_t)(act1 ? pt1 : pt0) * n * n;
  cc *M0 = reinterpret_cast<cc *>(a.M) + (size_t)pt0 * n * ncols;
  cc *M1 = reinterpret_cast<cc *>(a.M) + (size_t)(act1 ? pt1 : pt0) * n * ncols;
  cc *sk = reinterpret_cast<cc *>(smraw + tc::c4_smem_bytes());   // kinvL0, kR0, kinvL1, kR1
  const KVb<float> g0 = kv_of<float>(a, pt0), g1 = kv_of<float>(a, act1 ? pt1 : pt0);
  for (int i = threadIdx.x; i < n; i += tc::CG_THREADS) {
    sk[i] = g0.kinvL[i];
    sk[n + i] = g0.kR[i];
    sk[2 * n + i] = g1.kinvL[i];
    sk[3 * n + i] = g1.kR[i];
  }
  __syncthreads();
  const unsigned amask = (act0 ? 3u : 0u) | (act1 ? 12u : 0u);
  const bool ok = tc::cgemm_tile_shared_b(
      n, n, n, r0, c0, amask,
      [=](int h, int i, int l) { return tc::ldg_cc((h ? R1 : R0) + i + (size_t)l * n); },
      [=](int h, int l) { return sk[h * 2 * n + l]; },   // kinvL of point h
      [=](int l, int j) { return ov(l, j); },
      [=](int i, int j, const cc (&x)[4]) {
        const cc o = ovc(i, j);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!((amask >> (2 * h)) & 1u)) continue;
          const cc *kinv = sk + h * 2 * n, *kr = kinv + n;
          const cc r = cmul(kr[j], kinv[i]);
          const cc P = cmul(o, mkc<float>(0.5f * (1.f + r.re), 0.5f * r.im));
          const cc Q = cmul(o, mkc<float>(0.5f * (1.f - r.re), -0.5f * r.im));
          const cc t = cmul(kr[j], x[2 * h + 1]);
          const cc rq = mkc<float>(0.5f * (x[2 * h].re - t.re), 0.5f * (x[2 * h].im - t.im));
          const cc rp = mkc<float>(0.5f * (x[2 * h].re + t.re), 0.5f * (x[2 * h].im + t.im));
          cc *M = h ? M1 : M0;
          M[i + (size_t)j * n] = csub(P, rq);
          M[i + (size_t)(n + j) * n] = csub(rp, Q);
        }
      },
      smraw);
  if (!ok && threadIdx.x == 0) {
    if (act0) a.status[pt0] = 2;
    if (act1) a.status[pt1] = 2;
  }
}

// Row scales of the FP16-split [W|Y] (kb_wy2_tc16): for every point and row i,
// rowexp[2i] = e with max_l |R_il| < 2^e (largest real or imaginary part) and
// rowexp[2i+1] the same for R_il / k_l^p.  One thread per row (consecutive
// rows are contiguous in R).
__global__ void __launch_bounds__(256) kb_rowexp(SweepArgs a) {
  const int pt = blockIdx.y, i = blockIdx.x * 256 + threadIdx.x;
  if (inactive(a, pt) || i >= a.n) return;
  const int n = a.n;
  const cc *R = reinterpret_cast<const cc *>(a.R) + (size_t)pt * n * n;
  const KVb<float> v = kv_of<float>(a, pt);
  float m0 = 0.f, m1 = 0.f;
  for (int l = 0; l < n; ++l) {
    const cc r = R[i + (size_t)l * n];
    const cc rs = cmul(r, v.kinvL[l]);
    m0 = fmaxf(m0, fmaxf(fabsf(r.re), fabsf(r.im)));
    m1 = fmaxf(m1, fmaxf(fabsf(rs.re), fabsf(rs.im)));
  }
  int e0 = 0, e1 = 0;
  if (m0 > 0.f) frexpf(m0, &e0);
  if (m1 > 0.f) frexpf(m1, &e1);
  // keep the scales inside FP32's normal range (the values themselves are)
  a.rowexp[(size_t)pt * 2 * n + 2 * i] = max(-100, min(100, e0));
  a.rowexp[(size_t)pt * 2 * n + 2 * i + 1] = max(-100, min(100, e1));
}

// [W|Y] of point pairs as kb_wy2_tc, the products in the FP16 split with the
// row scales of kb_rowexp (the overlap, the shared B, is bounded by 1).
size_t wy2_tc16_smem_bytes(int n) { return tc::c4_smem_bytes16() + 4 * (size_t)n * sizeof(cc); }

__global__ void __launch_bounds__(tc::CG_THREADS, 1) kb_wy2_tc16(SweepArgs a, int p, int npts) {
  extern __shared__ __align__(128) unsigned char smtc[];
  unsigned char *smraw = smtc;
  const int pt0 = 2 * blockIdx.y, pt1 = pt0 + 1;
  const bool act0 = !inactive(a, pt0), act1 = pt1 < npts && !inactive(a, pt1);
  if (!act0 && !act1) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  const int tiles_m = (n + tc::CG_M / 2 - 1) / (tc::CG_M / 2);
  const int r0 = (blockIdx.x % tiles_m) * (tc::CG_M / 2), c0 = (blockIdx.x / tiles_m) * tc::CG_N;
  const PointDesc d = a.pts[act0 ? pt0 : pt1];   // both points have this one's overlaps
  const bool tr = a.mirror != 0;
  const int pi = tr ? d.N - p : p;
  const zc *O = overlap_of(a, d, p);
  const cc *O32 = overlap32_of(a, d, p);
  const cc *O32t = a.O32t ? a.O32t + ((size_t)d.o_off + pi) * n * n : nullptr;
  auto ov = [=](int l, int j) -> cc {
    if (tr) {
      if (O32) return tc::ldg_cc(O32 + j + (size_t)l * n);
      return ccast<float>(O[j + (size_t)l * n]);
    }
    if (O32t) return tc::ldg_cc(O32t + j + (size_t)l * n);
    if (O32) return tc::ldg_cc(O32 + l + (size_t)j * n);
    return ccast<float>(O[l + (size_t)j * n]);
  };
  auto ovc = [=](int l, int j) -> cc {
    if (tr) {
      if (O32t) return O32t[l + (size_t)j * n];
      if (O32) return O32[j + (size_t)l * n];
      return ccast<float>(O[j + (size_t)l * n]);
    }
    if (O32) return O32[l + (size_t)j * n];
    return ccast<float>(O[l + (size_t)j * n]);
  };
  const int q1 = act1 ? pt1 : pt0;
  const cc *R0 = reinterpret_cast<const cc *>(a.R) + (size_t)pt0 * n * n;
  const cc *R1 = reinterpret_cast<const cc *>(a.R) + (size_t)q1 * n * n;
  const int *X0 = a.rowexp + (size_t)pt0 * 2 * n, *X1 = a.rowexp + (size_t)q1 * 2 * n;
  cc *M0 = reinterpret_cast<cc *>(a.M) + (size_t)pt0 * n * ncols;
  cc *M1 = reinterpret_cast<cc *>(a.M) + (size_t)q1 * n * ncols;
  cc *sk = reinterpret_cast<cc *>(smraw + tc::c4_smem_bytes16());   // kinvL0, kR0, kinvL1, kR1
  const KVb<float> g0 = kv_of<float>(a, pt0), g1 = kv_of<float>(a, q1);
  for (int i = threadIdx.x; i < n; i += tc::CG_THREADS) {
    sk[i] = g0.kinvL[i];
    sk[n + i] = g0.kR[i];
    sk[2 * n + i] = g1.kinvL[i];
    sk[3 * n + i] = g1.kR[i];
  }
  __syncthreads();
  const unsigned amask = (act0 ? 3u : 0u) | (act1 ? 12u : 0u);
  const bool ok = tc::cgemm_tile_shared_b_f16(
      n, n, n, r0, c0, amask,
      [=](int h, int i, int l) { return tc::ldg_cc((h ? R1 : R0) + i + (size_t)l * n); },
      [=](int h, int l) { return sk[h * 2 * n + l]; },   // kinvL of point h
      [=](int l, int j) { return ov(l, j); },
      [=](int q, int i) { return ((q >> 1) ? X1 : X0)[2 * i + (q & 1)]; },
      [=](int i, int j, const cc (&x)[4]) {
        const cc o = ovc(i, j);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!((amask >> (2 * h)) & 1u)) continue;
          const cc *kinv = sk + h * 2 * n, *kr = kinv + n;
          const cc r = cmul(kr[j], kinv[i]);
          const cc P = cmul(o, mkc<float>(0.5f * (1.f + r.re), 0.5f * r.im));
          const cc Q = cmul(o, mkc<float>(0.5f * (1.f - r.re), -0.5f * r.im));
          const cc t = cmul(kr[j], x[2 * h + 1]);
          const cc rq = mkc<float>(0.5f * (x[2 * h].re - t.re), 0.5f * (x[2 * h].im - t.im));
          const cc rp = mkc<float>(0.5f * (x[2 * h].re + t.re), 0.5f * (x[2 * h].im + t.im));
          cc *M = h ? M1 : M0;
          M[i + (size_t)j * n] = csub(P, rq);
          M[i + (size_t)(n + j) * n] = csub(rp, Q);
        }
      },
      smraw);
  if (!ok && threadIdx.x == 0) {
    if (act0) a.status[pt0] = 2;
    if (act1) a.status[pt1] = 2;
  }
}

// Tile width of the update kernels (read-modify-write of C): 64 complex
// columns keep the prefetched C values of a thread in 32 registers.
constexpr int RMW_TN = 64;

// trailing update of the kb columns from j0: M[c0:n, c0:ncols] -= L21 U12
// (c0 = j0 + kb; kb = 64 for a pair of panels), or of columns c0 .. c0+cmax-1 only
__global__ void __launch_bounds__(tc::CG_THREADS, 3) kb_trail_tc(SweepArgs a, int j0, int kb, int cmax) {
  extern __shared__ __align__(128) unsigned char smtc[];
  unsigned char *smraw = smtc;
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  const int nb = min(kb, n - j0), c0 = j0 + nb;
  const int m = n - c0, ncol = min(cmax, (a.lapack_piv ? n : ncols) - c0);   // lapack_piv: W's columns only
  const int tiles_m = (m + tc::CG_M / 2 - 1) / (tc::CG_M / 2);
  const int r0 = (blockIdx.x % tiles_m) * (tc::CG_M / 2), q0 = (blockIdx.x / tiles_m) * RMW_TN;
  if (q0 >= ncol) return;
  cc *M = reinterpret_cast<cc *>(a.M) + (size_t)pt * n * ncols;
  const bool ok = tc::cgemm_tile<true, true, RMW_TN>(
      m, ncol, nb, r0, q0, [=](int i, int l) { return M[c0 + i + (size_t)(j0 + l) * n]; },
      [=](int l, int j) { return M[j0 + l + (size_t)(c0 + j) * n]; },
      [=](int i, int j) { return M[c0 + i + (size_t)(c0 + j) * n]; },
      [=](int i, int j, cc acc, cc old) { M[c0 + i + (size_t)(c0 + j) * n] = csub(old, acc); }, smraw);
  if (!ok && threadIdx.x == 0) a.status[pt] = 2;
}

// back-substitution update above block j0 (kb rows): M[0:j0, n:ncols] -= U[0:j0, b] X_b
// (rows lo .. j0-1 only when lo > 0)
__global__ void __launch_bounds__(tc::CG_THREADS, 3) kb_bsupd_tc(SweepArgs a, int j0, int kb, int lo = 0) {
  extern __shared__ __align__(128) unsigned char smtc[];
  unsigned char *smraw = smtc;
  const int pt = blockIdx.y;
  if (inactive(a, pt) || j0 <= lo) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  const int nb = min(kb, n - j0);
  const int m = j0 - lo, ncol = ncols - n;
  const int tiles_m = (m + tc::CG_M / 2 - 1) / (tc::CG_M / 2);
  const int r0 = (blockIdx.x % tiles_m) * (tc::CG_M / 2), q0 = (blockIdx.x / tiles_m) * RMW_TN;
  if (q0 >= ncol) return;
  cc *M = reinterpret_cast<cc *>(a.M) + (size_t)pt * n * ncols + lo;   // row lo as row 0
  const cc *X = M - lo;
  const bool ok = tc::cgemm_tile<true, true, RMW_TN>(
      m, ncol, nb, r0, q0, [=](int i, int l) { return M[i + (size_t)(j0 + l) * n]; },
      [=](int l, int j) { return X[j0 + l + (size_t)(n + j) * n]; },
      [=](int i, int j) { return M[i + (size_t)(n + j) * n]; },
      [=](int i, int j, cc acc, cc old) { M[i + (size_t)(n + j) * n] = csub(old, acc); }, smraw);
  if (!ok && threadIdx.x == 0) a.status[pt] = 2;
}

// Diagonal 128-row block of the triangular solves of the tensor-core FP32
// form: X_b <- U_bb^{-1} X_b (back substitution, UPPER) or X_b <- L_bb^{-1} X_b
// (forward elimination, L unit lower), for BS_COLS right-hand-side columns per
// CTA.  The block's triangle and the columns are staged in shared memory, the
// triangle's loads batched eight per thread so that many are in flight; the
// reciprocals of U's diagonal are formed once per CTA, so the recurrence
// multiplies instead of dividing.  Each warp solves four columns at once (lane
// r holds rows r, r+32, r+64, r+96; the solved value of row s passes by
// shuffle from its lane), so every element of the triangle read serves four
// columns and the four recurrences interleave.  With 128-row blocks the
// updates beside each block (kb_bsupd_tc, kb_fsupd_tc) have K = 128 and there
// are four blocks instead of sixteen at N_G = 512.
constexpr int BS_FB = 128, BS_COLS = 64, BS_THREADS = 512;
static_assert(BS_COLS == 4 * (BS_THREADS / 32), "four columns per warp");
size_t bsdiag_big_smem() {
  return ((size_t)BS_FB * BS_FB + (size_t)BS_FB * BS_COLS + BS_FB) * sizeof(cc);
}

template <bool UPPER>
__global__ void __launch_bounds__(BS_THREADS, 1) kb_diag_big(SweepArgs a, int j0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const int n = a.n, ncols = 2 * n + a.nc, nrhs = ncols - n;
  const int fb = min(BS_FB, n - j0);
  const int cf = blockIdx.x * BS_COLS;
  if (cf >= nrhs) return;
  const int ncl = min(BS_COLS, nrhs - cf);
  cc *M = reinterpret_cast<cc *>(a.M) + (size_t)pt * n * ncols;
  cc *Ts = reinterpret_cast<cc *>(smraw);    // Ts[r + c fb]: U's upper or L's strict lower triangle
  cc *Xs = Ts + (size_t)BS_FB * BS_FB;      // Xs[r + q fb]: the block rows of column cf + q
  cc *dinv = Xs + (size_t)BS_FB * BS_COLS;  // 1 / U_ss
  constexpr int U8 = 8;
  const int tt = fb * fb;
  for (int e0 = threadIdx.x; e0 < tt; e0 += U8 * BS_THREADS) {
    cc v[U8];
#pragma unroll
    for (int u = 0; u < U8; ++u) {
      const int e = e0 + u * BS_THREADS, r = e % fb, c = e / fb;
      const bool in = e < tt && (UPPER ? r <= c : r > c);
      v[u] = in ? M[j0 + r + (size_t)(j0 + c) * n] : czero<float>();
    }
#pragma unroll
    for (int u = 0; u < U8; ++u)
      if (e0 + u * BS_THREADS < tt) Ts[e0 + u * BS_THREADS] = v[u];
  }
  const int tx = fb * ncl;
  for (int e0 = threadIdx.x; e0 < tx; e0 += U8 * BS_THREADS) {
    cc v[U8];
#pragma unroll
    for (int u = 0; u < U8; ++u) {
      const int e = e0 + u * BS_THREADS, r = e % fb, q = e / fb;
      v[u] = e < tx ? M[j0 + r + (size_t)(n + cf + q) * n] : czero<float>();
    }
#pragma unroll
    for (int u = 0; u < U8; ++u)
      if (e0 + u * BS_THREADS < tx) Xs[e0 + u * BS_THREADS] = v[u];
  }
  if (UPPER)
    for (int r = threadIdx.x; r < fb; r += BS_THREADS) dinv[r] = cinv(M[j0 + r + (size_t)(j0 + r) * n]);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q0 = 4 * warp;   // this warp's four columns
  if (q0 < ncl) {
    cc x[4][4];   // [column][row slot t: row lane + 32 t]
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int r = lane + 32 * t;
        x[c][t] = (q0 + c < ncl && r < fb) ? Xs[r + (q0 + c) * fb] : czero<float>();
      }
    const int nsb = (fb + 31) >> 5;
    for (int k = 0; k < nsb; ++k) {
      const int sb = UPPER ? nsb - 1 - k : k;     // row slot of s
      const int cnt = min(32, fb - 32 * sb);
      for (int m = 0; m < cnt; ++m) {
        const int sl = UPPER ? cnt - 1 - m : m;
        const int s = 32 * sb + sl;
        cc xs[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          cc v = x[c][0];
#pragma unroll
          for (int t = 1; t < 4; ++t)
            if (t == sb) v = x[c][t];
          if (UPPER && lane == sl) {
            v = cmul(v, dinv[s]);
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (t == sb) x[c][t] = v;
          }
          xs[c] = mkc<float>(__shfl_sync(0xffffffffu, v.re, sl), __shfl_sync(0xffffffffu, v.im, sl));
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int r = lane + 32 * t;
          const bool live = UPPER ? (t <= sb && r < s) : (t >= sb && r > s && r < fb);
          if (live) {
            const cc u = Ts[r + s * fb];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              x[c][t].re -= u.re * xs[c].re - u.im * xs[c].im;
              x[c][t].im -= u.re * xs[c].im + u.im * xs[c].re;
            }
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int r = lane + 32 * t;
        if (q0 + c < ncl && r < fb) Xs[r + (q0 + c) * fb] = x[c][t];
      }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < tx; e += BS_THREADS) {
    const int r = e % fb, q = e / fb;
    M[j0 + r + (size_t)(n + cf + q) * n] = Xs[e];
  }
}

// The right-hand sides of the tensor-core FP32 form after the LU of W
// (P W = L U): X <- P X (kb_rhs_perm), then X <- L^{-1} X by 128-row blocks
// (kb_diag_big<false> on the diagonal blocks, kb_fsupd_tc below them), then the
// back substitution as before.  P applies the pivots in order: row j swaps
// with piv[j] for j = 0 .. n-1.
constexpr int RP_COLS = 16;   // right-hand-side columns per CTA of kb_rhs_perm
size_t rhs_perm_smem(int n) { return (size_t)RP_COLS * n * sizeof(cc) + (size_t)n * sizeof(int); }

__global__ void __launch_bounds__(256) kb_rhs_perm(SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const int n = a.n, ncols = 2 * n + a.nc, nrhs = ncols - n;
  const int cf = blockIdx.x * RP_COLS;
  if (cf >= nrhs) return;
  const int ncl = min(RP_COLS, nrhs - cf);
  cc *S = reinterpret_cast<cc *>(smraw);                         // S[r + q n]
  int *perm = reinterpret_cast<int *>(S + (size_t)RP_COLS * n);   // row r of P X is row perm[r] of X
  cc *M = reinterpret_cast<cc *>(a.M) + (size_t)pt * n * ncols;
  const int *piv = a.piv + (size_t)pt * n;
  for (int e = threadIdx.x; e < n * ncl; e += 256) S[e] = M[e % n + (size_t)(n + cf + e / n) * n];
  if (threadIdx.x == 0) {
    for (int r = 0; r < n; ++r) perm[r] = r;
    for (int j = 0; j < n; ++j) {
      const int p = piv[j];
      if (p > j && p < n) {   // p < j or out of range cannot come from the factorisation
        const int t = perm[j];
        perm[j] = perm[p];
        perm[p] = t;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * ncl; e += 256) {
    const int r = e % n, q = e / n;
    M[r + (size_t)(n + cf + q) * n] = S[perm[r] + q * n];
  }
}

// Forward update below block [j0, j0+kb): M[j0+kb:n, n:ncols] -= L[j0+kb:n, b] X_b
__global__ void __launch_bounds__(tc::CG_THREADS) kb_fsupd_tc(SweepArgs a, int j0, int kb) {
  extern __shared__ __align__(128) unsigned char smtc[];
  unsigned char *smraw = smtc;
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  const int nb = min(kb, n - j0), c0 = j0 + nb;
  const int m = n - c0, ncol = ncols - n;
  if (m <= 0) return;
  const int tiles_m = (m + tc::CG_M / 2 - 1) / (tc::CG_M / 2);
  const int r0 = (blockIdx.x % tiles_m) * (tc::CG_M / 2), q0 = (blockIdx.x / tiles_m) * RMW_TN;
  if (q0 >= ncol) return;
  cc *M = reinterpret_cast<cc *>(a.M) + (size_t)pt * n * ncols;
  const bool ok = tc::cgemm_tile<true, true, RMW_TN>(
      m, ncol, nb, r0, q0, [=](int i, int l) { return M[c0 + i + (size_t)(j0 + l) * n]; },
      [=](int l, int j) { return M[j0 + l + (size_t)(n + j) * n]; },
      [=](int i, int j) { return M[c0 + i + (size_t)(n + j) * n]; },
      [=](int i, int j, cc acc, cc old) { M[c0 + i + (size_t)(n + j) * n] = csub(old, acc); }, smraw);
  if (!ok && threadIdx.x == 0) a.status[pt] = 2;
}

// left0 >= 0 (FP32, the second panel of a pair): after the factorisation the
// panel's row swaps also reach the first panel's L columns left0 .. j0-1
// (rows j0 and below), so that they match the rows the pair's K = 64
// trailing update reaches
template <typename T, int BT>
__global__ void __launch_bounds__(BT) kb_panel(SweepArgs a, int j0, int left0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.x;
  if (inactive(a, pt)) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  constexpr int NB = Tile<T, BT>::NB;
  cx<T> *Ls = reinterpret_cast<cx<T> *>(smraw);
  T *sval = reinterpret_cast<T *>(Ls + NB * NB);
  int *sidx = reinterpret_cast<int *>(sval + 40);
  int *flag = sidx + 40;
  cx<T> *P = reinterpret_cast<cx<T> *>(smraw + panel_head_bytes<T, BT>());
  if (threadIdx.x == 0) *flag = 0;
  __syncthreads();
  cx<T> *M = reinterpret_cast<cx<T> *>(a.M) + (size_t)pt * n * ncols;
  if constexpr (std::is_same<T, float>::value) {
    // the staged panel must fit the launch's dynamic shared memory
    unsigned dyn = 0;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const bool fits = panel_head_bytes<T, BT>() + (size_t)(n - j0) * NB * sizeof(cx<T>) <= dyn;
    if (a.panel_smem && !fits && threadIdx.x == 0 && pt == 0 && j0 == 0)
      printf("kb_panel: staged panel of %d rows does not fit %u bytes; global path taken\n", n - j0, dyn);
    // FP32: the right-hand columns are left to kb_panel_apply (many CTAs per point)
    if (a.panel_smem && fits)
      lu_panel_smem<T, BT>(M, n, n, ncols, j0, a.piv + (size_t)pt * n, P, Ls, sval, sidx, flag, false);
    else lu_panel<T, BT>(M, n, n, ncols, j0, a.piv + (size_t)pt * n, Ls, sval, sidx, flag, false);
    if (left0 >= 0)
      panel_right_apply<T, BT>(M, n, left0, j0, j0, min(NB, n - j0), n - j0, a.piv + (size_t)pt * n, Ls, flag,
                               false);
  } else {
    lu_panel<T, BT>(M, n, n, ncols, j0, a.piv + (size_t)pt * n, Ls, sval, sidx, flag);
  }
  if (threadIdx.x == 0 && (*flag & 4)) printf("kb_panel: pivot row out of range (point %d, panel %d)\n", pt, j0);
  if (threadIdx.x == 0 && *flag) a.status[pt] = 1;
}

// Right-hand columns of panel j0 after kb_panel (FP32): row swaps and
// U12 = L11^{-1} A12, BT columns per CTA; grid (column blocks, points).
template <typename T, int BT>
__global__ void __launch_bounds__(BT) kb_panel_apply(SweepArgs a, int j0) {
  constexpr int NB = Tile<T, BT>::NB;
  __shared__ cx<T> Ls[NB * NB];
  __shared__ int flag;
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  const int nb = min(NB, n - j0), c0 = j0 + nb;
  // lapack_piv: column blocks [0, j0) take the swaps only (the L columns of
  // earlier panels), then [c0, n) swaps and the L11 solve; the right-hand
  // sides are left to the elimination after the LU
  const int nleft = a.lapack_piv ? (j0 + BT - 1) / BT : 0;
  const bool left = (int)blockIdx.x < nleft;
  const int cb = left ? blockIdx.x * BT : c0 + ((int)blockIdx.x - nleft) * BT;
  const int ce = left ? min(j0, cb + BT) : min(a.lapack_piv ? n : ncols, cb + BT);
  if (cb >= ce) return;
  cx<T> *M = reinterpret_cast<cx<T> *>(a.M) + (size_t)pt * n * ncols;
  for (int e = threadIdx.x; e < nb * nb; e += BT) {
    const int r = e % nb, s2 = e / nb;
    Ls[r + s2 * NB] = M[j0 + r + (size_t)(j0 + s2) * n];
  }
  if (threadIdx.x == 0) flag = 0;
  __syncthreads();
  panel_right_apply<T, BT>(M, n, cb, ce, j0, nb, n - j0, a.piv + (size_t)pt * n, Ls, &flag, !left);
  if (threadIdx.x == 0 && (flag & 4)) {
    printf("kb_panel_apply: pivot row out of range (point %d, panel %d)\n", pt, j0);
    a.status[pt] = 1;
  }
}

// Right-hand columns of the second panel of a pair (j0, j1 = j0 + NB) after
// kb_panel(j1): the panel's row swaps, the first panel's update of the 32
// swapped rows (A23 - L21 U13, with L21 already in the second panel's row
// order), then U23 = L22^{-1} (A23 - L21 U13); the rows below keep the first
// panel's update for the pair's K = 64 trailing update.  Grid (column blocks
// of [j1 + nb, ncols), points).
template <int BT>
__global__ void __launch_bounds__(BT) kb_panel_apply_pair(SweepArgs a, int j0) {
  constexpr int NB = Tile<float, BT>::NB;
  __shared__ cc Ls[NB * NB], L1s[NB * NB];
  __shared__ int flag;
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  const int j1 = j0 + NB, nb = min(NB, n - j1), c1 = j1 + nb;
  const int cb = c1 + blockIdx.x * BT, ce = min(ncols, cb + BT);
  if (cb >= ce) return;
  cc *M = reinterpret_cast<cc *>(a.M) + (size_t)pt * n * ncols;
  for (int e = threadIdx.x; e < NB * NB; e += BT) {
    const int r = e % NB, s2 = e / NB;
    Ls[e] = (r < nb && s2 < nb) ? M[j1 + r + (size_t)(j1 + s2) * n] : czero<float>();
    L1s[e] = r < nb ? M[j1 + r + (size_t)(j0 + s2) * n] : czero<float>();
  }
  if (threadIdx.x == 0) flag = 0;
  __syncthreads();
  panel_right_apply<float, BT>(M, n, cb, ce, j1, nb, n - j1, a.piv + (size_t)pt * n, Ls, &flag, true, L1s, j0);
  if (threadIdx.x == 0 && (flag & 4)) {
    printf("kb_panel_apply_pair: pivot row out of range (point %d, panel %d)\n", pt, j1);
    a.status[pt] = 1;
  }
}

template <typename T, int BT>
__global__ void __launch_bounds__(BT) kb_trail(SweepArgs a, int j0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  cx<T> *M = reinterpret_cast<cx<T> *>(a.M) + (size_t)pt * n * ncols;
  lu_trailing<T, BT>(M, n, n, ncols, j0, reinterpret_cast<cx<T> *>(smraw), blockIdx.x, gridDim.x);
}

template <typename T, int BT>
__global__ void __launch_bounds__(BT) kb_bsdiag(SweepArgs a, int j0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  cx<T> *M = reinterpret_cast<cx<T> *>(a.M) + (size_t)pt * n * ncols;
  const int per = (ncols - n + gridDim.x - 1) / gridDim.x;
  const int c0 = n + blockIdx.x * per, c1 = min(ncols, c0 + per);
  if constexpr (std::is_same<T, float>::value) {
    if (c0 < c1) lu_bs_diag_staged<BT>(M, n, n, j0, c0, c1, reinterpret_cast<cc *>(smraw));
  } else {
    lu_bs_diag<T, BT>(M, n, n, j0, c0, c1, reinterpret_cast<cx<T> *>(smraw));
  }
}

template <typename T, int BT>
__global__ void __launch_bounds__(BT) kb_bsupd(SweepArgs a, int j0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pt = blockIdx.y;
  if (inactive(a, pt)) return;
  const int n = a.n, ncols = 2 * n + a.nc;
  cx<T> *M = reinterpret_cast<cx<T> *>(a.M) + (size_t)pt * n * ncols;
  lu_bs_update<T, BT>(M, n, n, ncols, j0, reinterpret_cast<cx<T> *>(smraw), blockIdx.x, gridDim.x);
}

template <typename T>
__global__ void __launch_bounds__(VT) kb_finish(SweepArgs a, int p) {
  // grid (FINISH_BLOCKS, points): the n x n stores and the R update are spread
  // over all blocks of a point; block 0 also stores u_p and the pivots, scales
  // Tacc and, after the last interface, forms t and T
  const int pt = blockIdx.y, tid = threadIdx.x, blk = blockIdx.x, nblk = gridDim.x;
  const PointDesc d = a.pts[pt];
  const int n = a.n, N = d.N, nc = a.nc, ncols = 2 * n + nc;
  if (p > N) return;
  if (inactive(a, pt)) {
    if (p == N && tid == 0 && blk == 0) {
      a.T[d.out] = __longlong_as_double(0x7ff8000000000000ll);
      if (a.nopen) { a.nopen[2 * d.out] = d.nL; a.nopen[2 * d.out + 1] = d.nR; }
      if (a.err) a.err[d.out] = 0.0;
    }
    return;
  }
  cx<T> *R = reinterpret_cast<cx<T> *>(a.R) + (size_t)pt * n * n;
  cx<T> *M = reinterpret_cast<cx<T> *>(a.M) + (size_t)pt * n * ncols;
  const int *piv = a.piv + (size_t)pt * n;
  const KVb<T> v = kv_of<T>(a, pt);
  const size_t nn = (size_t)n * n;
  const size_t e0 = nn * blk / nblk, e1 = nn * (blk + 1) / nblk;
  // R <- E+ Z_Y E+, with the stores of Z_Y and of W's LU factors for the
  // refinement in the same pass (Z_Y's element read once)
  cx<T> *Zs = a.Zst ? reinterpret_cast<cx<T> *>(a.Zst) + ((size_t)d.st_off + p) * nn : nullptr;
  cx<T> *Ls = a.LUst ? reinterpret_cast<cx<T> *>(a.LUst) + ((size_t)d.st_off + p) * nn : nullptr;
  for (size_t e = e0 + tid; e < e1; e += VT) {
    const int i = e % n, j = e / n;
    const cx<T> z = M[nn + e];   // Z_Y(i, j) = M(i, n + j)
    if (Zs) Zs[e] = z;
    if (Ls) Ls[e] = M[e];
    R[e] = cmul(cmul(v.ep[i], z), v.ep[j]);
  }
  if (blk != 0) return;
  if (a.Zst) {
    cx<T> *Us = reinterpret_cast<cx<T> *>(a.Ust) + ((size_t)d.st_off + p) * n * nc;
    for (size_t e = tid; e < (size_t)n * nc; e += VT) Us[e] = M[2 * nn + e];
  }
  if (a.LUst) {
    int *Ps = a.PIVst + ((size_t)d.st_off + p) * n;
    for (int e = tid; e < n; e += VT) Ps[e] = piv[e];
  }
  // Tacc <- E+ Z_T (after its store above: the same thread owns each element)
  for (size_t e = tid; e < (size_t)n * nc; e += VT) {
    const int i = e % n, c = e / n;
    cx<T> &x = M[i + (size_t)(2 * n + c) * n];
    x = cmul(v.ep[i], x);
  }
  if (a.pivratio) {
    // the spread of U's diagonal (a lower bound on U's condition number)
    float hi = 0.f, lo = INFINITY;
    for (int i = tid; i < n; i += VT) {
      const cx<T> u = M[i + (size_t)i * n];
      const float m = hypotf(float(u.re), float(u.im));
      hi = fmaxf(hi, m);
      lo = fminf(lo, m);
    }
    for (int off = 16; off > 0; off >>= 1) {
      hi = fmaxf(hi, __shfl_down_sync(0xffffffffu, hi, off));
      lo = fminf(lo, __shfl_down_sync(0xffffffffu, lo, off));
    }
    __shared__ float ext[2][VT / 32];
    if ((tid & 31) == 0) { ext[0][tid >> 5] = hi; ext[1][tid >> 5] = lo; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < VT / 32; ++w) { hi = fmaxf(hi, ext[0][w]); lo = fminf(lo, ext[1][w]); }
      const float r = lo > 0.f ? hi / lo : INFINITY;
      a.pivratio[pt] = fmaxf(a.pivratio[pt], r);
    }
  }
  if (p < N) return;
  __syncthreads();
  // t_ij = sqrt(k_i^R / k_j^L) S11_ij on open channels, T = sum |t_ij|^2
  const double *EL = energies_of(a, d, 0);
  const double *ER = energies_of(a, d, N + 1);
  double acc = 0.0;
  for (int e = tid; e < d.nR * d.nL; e += VT) {
    const int i = e % d.nR, j = e / d.nR;
    const double f = sqrt(sqrt(d.E - ER[i]) / sqrt(d.E - EL[j]));
    const cx<T> x = M[i + (size_t)(2 * n + j) * n];
    const zc tv = mkc<double>(f * double(x.re), f * double(x.im));
    acc += tv.re * tv.re + tv.im * tv.im;
    if (a.t) a.t[(size_t)d.out * n * n + i + (size_t)j * n] = tv;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  __shared__ double red[VT / 32];
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double tsum = 0.0;
    for (int w = 0; w < VT / 32; ++w) tsum += red[w];
    a.T[d.out] = tsum;
    if (a.nopen) { a.nopen[2 * d.out] = d.nL; a.nopen[2 * d.out + 1] = d.nR; }
    if (a.err) a.err[d.out] = 0.0;
  }
}

template <typename T, int BT>
static cudaError_t sweep_step(const SweepArgs &a0, int npts, int p, cudaStream_t s, cudaEvent_t wy0,
                              cudaEvent_t wy1, bool tensor_core, bool f16 = false, bool big = false) {
  SweepArgs a = a0;
  a.p = p;
  const int n = a.n, ncols = 2 * n + a.nc;
  constexpr int BM = Tile<T, BT>::BM, BN = Tile<T, BT>::BN, NB = Tile<T, BT>::NB;
  const size_t gsm = gemm_smem_elems<T, BT>() * sizeof(cx<T>);
  const size_t psm_big = panel_head_bytes<T, BT>() + (size_t)n * NB * sizeof(cx<T>);
  a.panel_smem = std::is_same<T, float>::value && psm_big + PANEL_STATIC_RESERVE <= (size_t)g_smem_optin;
  const size_t psm = a.panel_smem ? psm_big : panel_head_bytes<T, BT>();
  const size_t dsm = (size_t)2 * NB * NB * sizeof(cx<T>);
  auto tiles = [](int m, int nn, int bm, int bn) { return ((m + bm - 1) / bm) * ((nn + bn - 1) / bn); };
  PW_TIMED(KK_VECTORS, s, kb_vectors<T><<<npts, VT, 0, s>>>(a, p));
  if (p > 0) {
    const size_t wsm = gsm + 2 * (size_t)n * sizeof(cx<T>);
    if (wy0) cudaEventRecord(wy0, s);
    if (std::is_same<T, float>::value && tensor_core && a.wy_pairs && f16 && a.rowexp) {
      PW_TIMED(KK_ROWEXP, s, kb_rowexp<<<dim3((n + 255) / 256, npts), 256, 0, s>>>(a));
      PW_TIMED(KK_WY, s,
               kb_wy2_tc16<<<dim3(tiles(n, n, tc::CG_M / 2, tc::CG_N), (npts + 1) / 2), tc::CG_THREADS,
                             wy2_tc16_smem_bytes(n), s>>>(a, p, npts));
    } else if (std::is_same<T, float>::value && tensor_core && a.wy_pairs)
      PW_TIMED(KK_WY, s,
               kb_wy2_tc<<<dim3(tiles(n, n, tc::CG_M / 2, tc::CG_N), (npts + 1) / 2), tc::CG_THREADS,
                           wy2_tc_smem_bytes(n), s>>>(a, p, npts));
    else if (std::is_same<T, float>::value && tensor_core)
      PW_TIMED(KK_WY, s,
               kb_wy_tc<<<dim3(tiles(n, 2 * n, tc::CG_M / 2, tc::CG_N), npts), tc::CG_THREADS,
                          wy_tc_smem_bytes(n), s>>>(a, p));
    else
      PW_TIMED(KK_WY, s, kb_wy<T, BT><<<dim3(tiles(n, 2 * n, BM, BN), npts), BT, wsm, s>>>(a, p));
    if (wy1) cudaEventRecord(wy1, s);
  }
  // separable nonlocal terms (FP64 form): the source columns of Tacc take
  // Y fa_q + fb_p before the solve
  if constexpr (std::is_same<T, double>::value) {
    if (a.nl_m > 0) {
      const cudaError_t e = launch_nl_sources(a, npts, p, s);
      if (e != cudaSuccess) return e;
    }
  }
  // tensor-core FP32 form with 128-row blocks (variant bit 3): LAPACK-ordered
  // pivots, the LU of W alone, then the right-hand sides eliminated in 128-row
  // blocks (see kb_rhs_perm); otherwise each panel's swaps and L11 solve reach
  // the right-hand sides too and the trailing updates carry them along
  const bool lapack = std::is_same<T, float>::value && tensor_core && big;
  a.lapack_piv = lapack ? 1 : 0;
  const int ucols = lapack ? n : ncols;   // columns the LU updates
  // tensor-core FP32 form without LAPACK pivots: panels in pairs (j0, j1 =
  // j0 + 32).  The first panel's update reaches only the second panel's
  // columns (a 32-column update) and, at the second panel's apply, its 32
  // rows; the rest of the matrix takes both panels at once (K = 64), so the
  // trailing matrix is read and written once per pair instead of per panel
  const bool paired = std::is_same<T, float>::value && tensor_core && !lapack;
  const int TAIL = 1 << 30;
  for (int j0 = 0; j0 < n;) {
    PW_TIMED(KK_PANEL, s, kb_panel<T, BT><<<npts, BT, psm, s>>>(a, j0, -1));
    const int c0 = j0 + min(NB, n - j0);
    if constexpr (std::is_same<T, float>::value) {
      const int blocks = (lapack ? (j0 + BT - 1) / BT : 0) + (ucols - c0 + BT - 1) / BT;
      if (blocks > 0) PW_TIMED(KK_PANEL_APPLY, s, kb_panel_apply<T, BT><<<dim3(blocks, npts), BT, 0, s>>>(a, j0));
    }
    if (paired && c0 < n) {
      const int j1 = c0, c1 = j1 + min(NB, n - j1);
      const dim3 gn(tiles(n - j1, c1 - j1, tc::CG_M / 2, RMW_TN), npts);
      PW_TIMED(KK_TRAIL, s, kb_trail_tc<<<gn, tc::CG_THREADS, tc::cg_smem_bytes<RMW_TN>(), s>>>(a, j0, NB, c1 - j1));
      PW_TIMED(KK_PANEL, s, kb_panel<T, BT><<<npts, BT, psm, s>>>(a, j1, j0));
      const int blocks = (ncols - c1 + BT - 1) / BT;
      if (blocks > 0)
        PW_TIMED(KK_PANEL_APPLY, s, kb_panel_apply_pair<BT><<<dim3(blocks, npts), BT, 0, s>>>(a, j0));
      if (c1 < n) {
        const dim3 gw(tiles(n - c1, ncols - c1, tc::CG_M / 2, RMW_TN), npts);
        PW_TIMED(KK_TRAIL, s, kb_trail_tc<<<gw, tc::CG_THREADS, tc::cg_smem_bytes<RMW_TN>(), s>>>(a, j0, 2 * NB, TAIL));
      }
      j0 = c1;
      continue;
    }
    if (c0 < n) {
      if (std::is_same<T, float>::value && tensor_core)
        PW_TIMED(KK_TRAIL, s,
                 kb_trail_tc<<<dim3(tiles(n - c0, ucols - c0, tc::CG_M / 2, RMW_TN), npts), tc::CG_THREADS,
                               tc::cg_smem_bytes<RMW_TN>(), s>>>(a, j0, NB, TAIL));
      else
        PW_TIMED(KK_TRAIL, s, kb_trail<T, BT><<<dim3(tiles(n - c0, ncols - c0, BM, BN), npts), BT, gsm, s>>>(a, j0));
    }
    j0 = c0;
  }
  if (lapack) {
    const int cgroups = (ncols - n + BS_COLS - 1) / BS_COLS;
    PW_TIMED(KK_RHS_PERM, s,
             kb_rhs_perm<<<dim3((ncols - n + RP_COLS - 1) / RP_COLS, npts), 256, rhs_perm_smem(n), s>>>(a));
    for (int j0 = 0; j0 < n; j0 += BS_FB) {
      PW_TIMED(KK_FSDIAG, s, kb_diag_big<false><<<dim3(cgroups, npts), BS_THREADS, bsdiag_big_smem(), s>>>(a, j0));
      const int c1 = j0 + std::min(BS_FB, n - j0);
      if (c1 < n)
        PW_TIMED(KK_FSUPD, s,
                 kb_fsupd_tc<<<dim3(tiles(n - c1, ncols - n, tc::CG_M / 2, RMW_TN), npts), tc::CG_THREADS,
                               tc::cg_smem_bytes<RMW_TN>(), s>>>(a, j0, BS_FB));
    }
  }
  const int rhs_blocks = max(1, (ncols - n + BT - 1) / BT);
  // FP32: the diagonal solves stage their right-hand-side columns in shared memory
  const size_t bsm = std::is_same<T, float>::value
                         ? lu_bs_diag_staged_smem((ncols - n + rhs_blocks - 1) / rhs_blocks)
                         : dsm;
  if (lapack) {
    // 128-row blocks: four diagonal solves and three K = 128 updates at N_G = 512
    const int cgroups = (ncols - n + BS_COLS - 1) / BS_COLS;
    for (int j0 = ((n - 1) / BS_FB) * BS_FB; j0 >= 0; j0 -= BS_FB) {
      PW_TIMED(KK_BSDIAG, s, kb_diag_big<true><<<dim3(cgroups, npts), BS_THREADS, bsdiag_big_smem(), s>>>(a, j0));
      if (j0 > 0)
        PW_TIMED(KK_BSUPD, s,
                 kb_bsupd_tc<<<dim3(tiles(j0, ncols - n, tc::CG_M / 2, RMW_TN), npts), tc::CG_THREADS,
                               tc::cg_smem_bytes<RMW_TN>(), s>>>(a, j0, BS_FB));
    }
  } else if (std::is_same<T, float>::value && tensor_core) {
    // blocks in pairs from the bottom: block b, the 32 rows of block b-1
    // updated from it, block b-1, then one update of the rows above both with
    // K = 32 + (rows of b) instead of two with K = 32 over all of them
    for (int jb = ((n - 1) / NB) * NB; jb >= 0; jb -= 2 * NB) {
      PW_TIMED(KK_BSDIAG, s, kb_bsdiag<T, BT><<<dim3(rhs_blocks, npts), BT, bsm, s>>>(a, jb));
      if (jb == 0) break;
      const int j0 = jb - NB;
      // block b-1's rows take block b's contribution (32 rows, K = rows of b)
      PW_TIMED(KK_BSUPD, s,
               kb_bsupd_tc<<<dim3(tiles(NB, ncols - n, tc::CG_M / 2, RMW_TN), npts), tc::CG_THREADS,
                             tc::cg_smem_bytes<RMW_TN>(), s>>>(a, jb, NB, j0));
      PW_TIMED(KK_BSDIAG, s, kb_bsdiag<T, BT><<<dim3(rhs_blocks, npts), BT, bsm, s>>>(a, j0));
      if (j0 > 0)
        PW_TIMED(KK_BSUPD, s,
                 kb_bsupd_tc<<<dim3(tiles(j0, ncols - n, tc::CG_M / 2, RMW_TN), npts), tc::CG_THREADS,
                               tc::cg_smem_bytes<RMW_TN>(), s>>>(a, j0, 2 * NB));
    }
  } else {
    for (int j0 = ((n - 1) / NB) * NB; j0 >= 0; j0 -= NB) {
      PW_TIMED(KK_BSDIAG, s, kb_bsdiag<T, BT><<<dim3(rhs_blocks, npts), BT, bsm, s>>>(a, j0));
      if (j0 > 0) {
        if (std::is_same<T, float>::value && tensor_core)
          PW_TIMED(KK_BSUPD, s,
                   kb_bsupd_tc<<<dim3(tiles(j0, ncols - n, tc::CG_M / 2, RMW_TN), npts), tc::CG_THREADS,
                                 tc::cg_smem_bytes<RMW_TN>(), s>>>(a, j0, NB));
        else
          PW_TIMED(KK_BSUPD, s, kb_bsupd<T, BT><<<dim3(tiles(j0, ncols - n, BM, BN), npts), BT, gsm, s>>>(a, j0));
      }
    }
  }
  PW_TIMED(KK_FINISH, s, kb_finish<T><<<dim3(FINISH_BLOCKS, npts), VT, 0, s>>>(a, p));
  return cudaGetLastError();
}

// Dynamic shared-memory limits of the variant's kernels (outside any stream
// capture: attributes are set once per process and size).
template <typename T, int BT>
static cudaError_t sweep_prepare(int n) {
  const size_t gsm = gemm_smem_elems<T, BT>() * sizeof(cx<T>);
  const size_t wsm = gsm + 2 * (size_t)n * sizeof(cx<T>);
  if (!g_smem_optin) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  const size_t psm_big = panel_head_bytes<T, BT>() + (size_t)n * Tile<T, BT>::NB * sizeof(cx<T>);
  if (std::is_same<T, float>::value && psm_big + PANEL_STATIC_RESERVE <= (size_t)g_smem_optin) {
    const cudaError_t ep =
        cudaFuncSetAttribute(kb_panel<T, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm_big);
    if (ep != cudaSuccess) return ep;
  }
  if (std::is_same<T, float>::value) {
    // the staged diagonal solves: at most BT columns a CTA
    cudaError_t eb = cudaFuncSetAttribute(kb_bsdiag<T, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)lu_bs_diag_staged_smem(BT));
    if (eb != cudaSuccess) return eb;
  }
  cudaError_t e = cudaFuncSetAttribute(kb_wy<T, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_trail<T, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_bsupd<T, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
  return e;
}

cudaError_t prepare_sweep_batched(int n, int precision, int variant) {
  if (precision == PW_FP64)
    return (variant & 1) ? sweep_prepare<double, 512>(n) : sweep_prepare<double, 256>(n);
  cudaError_t e = (variant & 1) ? sweep_prepare<float, 512>(n) : sweep_prepare<float, 256>(n);
  if (e == cudaSuccess && (variant & 2))
    e = cudaFuncSetAttribute(kb_wy_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wy_tc_smem_bytes(n));
  if (e == cudaSuccess && (variant & 2))
    e = cudaFuncSetAttribute(kb_wy2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wy2_tc_smem_bytes(n));
  if (e == cudaSuccess && (variant & 2))
    e = cudaFuncSetAttribute(kb_trail_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::cg_smem_bytes<RMW_TN>());
  if (e == cudaSuccess && (variant & 2))
    e = cudaFuncSetAttribute(kb_bsupd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::cg_smem_bytes<RMW_TN>());
  if (e == cudaSuccess && (variant & 2))
    e = cudaFuncSetAttribute(kb_diag_big<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsdiag_big_smem());
  if (e == cudaSuccess && (variant & 2))
    e = cudaFuncSetAttribute(kb_diag_big<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsdiag_big_smem());
  if (e == cudaSuccess && (variant & 2))
    e = cudaFuncSetAttribute(kb_fsupd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::cg_smem_bytes<RMW_TN>());
  if (e == cudaSuccess && (variant & 2))
    e = cudaFuncSetAttribute(kb_rhs_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhs_perm_smem(n));
  if (e == cudaSuccess && (variant & 6) == 6)
    e = cudaFuncSetAttribute(kb_wy2_tc16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wy2_tc16_smem_bytes(n));
  return e;
}

cudaError_t launch_sweep_batched(const SweepArgs &a, int npts, int p, int precision, cudaStream_t s,
                                 cudaEvent_t wy0, cudaEvent_t wy1, int variant) {
  const bool tcore = (variant & 2) != 0;
  if (precision == PW_FP64)
    return (variant & 1) ? sweep_step<double, 512>(a, npts, p, s, wy0, wy1, false)
                         : sweep_step<double, 256>(a, npts, p, s, wy0, wy1, false);
  const bool f16 = (variant & 4) != 0;   // FP16 split for the paired [W|Y]
  const bool big = (variant & 8) != 0;   // LAPACK-ordered pivots, 128-row triangular blocks
  return (variant & 1) ? sweep_step<float, 512>(a, npts, p, s, wy0, wy1, tcore, f16, big)
                       : sweep_step<float, 256>(a, npts, p, s, wy0, wy1, tcore, f16, big);
}

int sweep_variants(int precision) { return precision == PW_FP64 ? 2 : 128; }

std::vector<int> sweep_variant_candidates(int precision) {
  if (precision == PW_FP64) return {0, 1};
  return {2, 3, 6, 10, 14};
}

int sweep_batched_launches(int n, int precision, int variant) {
  const int NB = Tile<float, 256>::NB;
  const int panels = (n + NB - 1) / NB;
  const bool fp32 = precision != PW_FP64, tensor = fp32 && (variant & 2) && (variant & 8);
  // vectors, [W|Y], finish; per panel: factorisation, trailing update (not
  // after the last), the FP32 form's right-hand apply (panels in pairs: the
  // 32-column update of the second panel and the pair's K = 64 update, none
  // after the last pair, give the same count); the back substitution:
  // a diagonal solve per block and an update above every block but the first
  // (32-row blocks, or 128-row blocks in the tensor-core form)
  const int bblocks = tensor ? (n + BS_FB - 1) / BS_FB : panels;
  // the tensor-core form without LAPACK pivots pairs the 32-row blocks: a
  // 32-row update inside every pair and one update above every pair but the
  // lowest-placed
  const int bsupd = (fp32 && (variant & 2) && !tensor) ? panels / 2 + (panels + 1) / 2 - 1 : bblocks - 1;
  // the tensor-core form adds the right-hand sides' elimination: a
  // permutation, a diagonal solve per 128-row block and an update below every
  // block but the last
  return 3 + 2 * panels - 1 + (fp32 ? panels : 0) + bblocks + bsupd + (tensor ? 2 * bblocks : 0);
}

}  // namespace pw
