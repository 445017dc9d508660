// CTA-wide dense complex linear algebra on column-major matrices in global
// memory: a tiled GEMM with functor operands/epilogue, and a right-looking
// blocked LU with partial pivoting that eliminates on an augmented matrix
// [A | B] and back-substitutes, i.e. solves A X = B in place.
//
// One CTA owns one problem (one (E, k_par) point); every function here must be
// called by all threads of the CTA and ends with a __syncthreads().
#pragma once
#include <type_traits>
#include "pw_cx.cuh"

namespace pw {

constexpr int NT = 256;   // threads per CTA for every per-point kernel

// GEMM tile (BM x BN x BK, 4 x 4 complex micro-tiles) and LU panel width NB
// for a CTA of NTH threads.
template <typename T, int NTH = NT>
struct Tile {
  static constexpr int BM = NTH >= 512 ? 128 : 64, BN = 64, BK = 16, NB = 32;
};

template <typename T, int NTH = NT>
__host__ __device__ constexpr size_t gemm_smem_elems() {
  return size_t(Tile<T, NTH>::BK) * (Tile<T, NTH>::BM + 1) +
         size_t(Tile<T, NTH>::BK) * (Tile<T, NTH>::BN + 1);
}

// Accumulators of the native types need no renormalisation between k-tiles
// (the double-float accumulator of pw_df.cuh overloads this).
template <typename T>
__device__ __forceinline__ void cacc_renorm(cx<T> &) {}

// C(i,j) = fe(i, j, sum_l fa(i,l) fb(l,j)) for 0 <= i < m, 0 <= j < n, 0 <= l < k.
// fa/fb return cx<T>; fa is read with i fastest (A column-major), fb with l
// fastest (B column-major), so plain column-major operands load coalesced.
// Tile BM x BN x BK; each of the NTH threads owns a (BM/TY) x TN micro-tile with
// TX = BN/TN threads along N and TY = NTH/TX along M.  The CTA computes output
// tiles t_first, t_first + t_step, ... (all of them by default); several CTAs
// can share one product by striding over its tiles.  smem must hold
// BK*(BM+1) + BK*(BN+1) elements.
template <typename T, int BM, int BN, int BK, int TN, int NTH, class FA, class FB, class FE>
__device__ void cta_gemm_t(int m, int n, int k, FA fa, FB fb, FE fe, cx<T> *smem, int t_first = 0,
                           int t_step = 1) {
  constexpr int NT = NTH;
  constexpr int TX = BN / TN, TY = NT / TX, TM = BM / TY;
  static_assert(TX * TN == BN && TY * TM == BM && TX * TY == NT, "tile shape");
  constexpr int LDA = BM + 1, LDB = BN + 1;
  constexpr int LA = (BM * BK + NT - 1) / NT, LB = (BK * BN + NT - 1) / NT;
  cx<T> *As = smem;
  cx<T> *Bs = smem + BK * LDA;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const int tilesM = (m + BM - 1) / BM, tilesN = (n + BN - 1) / BN;
  for (int t = t_first; t < tilesM * tilesN; t += t_step) {
    const int i0 = (t % tilesM) * BM, j0 = (t / tilesM) * BN;
    cx<T> acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
      for (int c = 0; c < TN; ++c) acc[r][c] = czero<T>();
    // register stage of the next k-tile: global loads overlap the current tile's math
    cx<T> ra[LA], rb[LB];
    auto fetch = [&](int l0) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int e = tid + q * NT, ii = e % BM, ll = e / BM;
        const int i = i0 + ii, l = l0 + ll;
        ra[q] = (e < BM * BK && i < m && l < k) ? fa(i, l) : czero<T>();
      }
#pragma unroll
      for (int q = 0; q < LB; ++q) {
        const int e = tid + q * NT, ll = e % BK, jj = e / BK;
        const int l = l0 + ll, j = j0 + jj;
        rb[q] = (e < BK * BN && l < k && j < n) ? fb(l, j) : czero<T>();
      }
    };
    fetch(0);
    for (int l0 = 0; l0 < k; l0 += BK) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int e = tid + q * NT;
        if (e < BM * BK) As[(e / BM) * LDA + e % BM] = ra[q];
      }
#pragma unroll
      for (int q = 0; q < LB; ++q) {
        const int e = tid + q * NT;
        if (e < BK * BN) Bs[(e % BK) * LDB + e / BK] = rb[q];
      }
      __syncthreads();
      if (l0 + BK < k) fetch(l0 + BK);
      // the next tile's loads stay here, ahead of the math that hides their
      // latency (a compiler fence: no memory access moves across it)
      asm volatile("" ::: "memory");
#pragma unroll 4
      for (int ll = 0; ll < BK; ++ll) {
        cx<T> a[TM], b[TN];
#pragma unroll
        for (int r = 0; r < TM; ++r) a[r] = As[ll * LDA + ty + TY * r];
#pragma unroll
        for (int c = 0; c < TN; ++c) b[c] = Bs[ll * LDB + tx + TX * c];
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
          for (int c = 0; c < TN; ++c) cfma(acc[r][c], a[r], b[c]);
      }
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) cacc_renorm(acc[r][c]);
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        const int i = i0 + ty + TY * r, j = j0 + tx + TX * c;
        if (i < m && j < n) fe(i, j, acc[r][c]);
      }
  }
  __syncthreads();
}

template <typename T, int NTH = NT, class FA, class FB, class FE>
__device__ void cta_gemm(int m, int n, int k, FA fa, FB fb, FE fe, cx<T> *smem) {
  cta_gemm_t<T, Tile<T, NTH>::BM, Tile<T, NTH>::BN, Tile<T, NTH>::BK, 4, NTH>(m, n, k, fa, fb, fe, smem);
}

// Tall-skinny product (n <= 16 columns per tile): 128 x 16 tiles.
constexpr int SKINNY_BM = 128, SKINNY_BN = 16, SKINNY_BK = 16;
template <typename T>
__host__ __device__ constexpr size_t skinny_smem_elems() {
  return size_t(SKINNY_BK) * (SKINNY_BM + 1) + size_t(SKINNY_BK) * (SKINNY_BN + 1);
}
template <typename T, int NTH = NT, class FA, class FB, class FE>
__device__ void cta_gemm_skinny(int m, int n, int k, FA fa, FB fb, FE fe, cx<T> *smem) {
  constexpr int TNS = NTH / 256;   // 1 column per thread at 256 threads, 2 at 512
  cta_gemm_t<T, SKINNY_BM, SKINNY_BN, SKINNY_BK, (TNS < 1 ? 1 : TNS), NTH>(m, n, k, fa, fb, fe, smem);
}

// Plain column-major operand accessors.
template <typename T>
struct ColMajor {
  const cx<T> *p;
  int ld;
  __device__ cx<T> operator()(int i, int j) const { return p[i + (size_t)j * ld]; }
};

// Block-wide arg-max of a per-thread (value, index) pair; returns the winning
// index to every thread.  Ties go to the smaller index.
template <typename T, int NTH = NT>
__device__ int block_argmax(T v, int idx, T *sval, int *sidx) {
  constexpr int NT = NTH;
  for (int off = 16; off > 0; off >>= 1) {
    T ov = __shfl_down_sync(0xffffffffu, v, off);
    int oi = __shfl_down_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sval[warp] = v; sidx[warp] = idx; }
  __syncthreads();
  if (warp == 0) {
    v = lane < NT / 32 ? sval[lane] : T(-1);
    idx = lane < NT / 32 ? sidx[lane] : 0x7fffffff;
    for (int off = 16; off > 0; off >>= 1) {
      T ov = __shfl_down_sync(0xffffffffu, v, off);
      int oi = __shfl_down_sync(0xffffffffu, idx, off);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    if (lane == 0) sidx[0] = idx;
  }
  __syncthreads();
  const int r = sidx[0];
  __syncthreads();
  return r;
}

// block_argmax with one barrier: every warp reduces the per-warp partials
// itself.  sval/sidx may be written again only after a later barrier of the
// whole block (the caller's next step has one).
template <typename T, int NTH = NT>
__device__ int block_argmax1(T v, int idx, T *sval, int *sidx) {
  for (int off = 16; off > 0; off >>= 1) {
    T ov = __shfl_down_sync(0xffffffffu, v, off);
    int oi = __shfl_down_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sval[warp] = v; sidx[warp] = idx; }
  __syncthreads();
  v = lane < NTH / 32 ? sval[lane] : T(-1);
  idx = lane < NTH / 32 ? sidx[lane] : 0x7fffffff;
  for (int off = 16; off > 0; off >>= 1) {
    T ov = __shfl_xor_sync(0xffffffffu, v, off);
    int oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  return idx;
}

template <typename T>
__device__ __forceinline__ T tiny_pivot();
template <>
__device__ __forceinline__ double tiny_pivot<double>() { return 1e-300; }
template <>
__device__ __forceinline__ float tiny_pivot<float>() { return 1e-30f; }

// Columns [c_begin, c_end) of panel j0 (rows j0 ..; the panel spans columns
// j0 .. j0+nb-1): the panel's row swaps, then (solve) U12 = L11^{-1} A12 with each column's nb
// entries in registers (Ls: the factored nb x nb diagonal block, leading
// dimension NB).  The swap sequence r <-> p_r (p_r >= r, in order r = 0 ..
// nb-1) is first folded into a gather: row r < nb ends up holding original row
// src[r], and each displaced row q >= nb (some p_r) an original row from
// [0, nb) -- a row below the panel only ever receives the value that sat in
// row r at step r, which is an original panel row.  So a column's new rows are
// read before any row is written and the reads are independent (the
// sequential swaps make every step wait for the previous one's memory round
// trip).  `flag` gets bit 4 if the pivots break p_r >= r or the fold finds a
// displaced source outside the panel (neither can come from the
// factorisation).
// FP64 keeps the sequential swaps and an in-place solve: a register column of
// NB FP64 complex values would not fit beside the rest of the kernel.
// L1s (FP32 only, optional): the second panel of a pair.  The columns have
// not yet taken the first panel's update, so the swapped rows take
// x -= L1s U1 before the solve, with L1s the first panel's L rows j0 .. j0+nb-1
// (NB x NB in shared memory, already in this panel's row order) and U1 the
// column's NB rows from row ju (the first panel's U12).
template <typename T, int NTH = NT>
__device__ void panel_right_apply(cx<T> *M, int ld, int c_begin, int c_end, int j0, int nb, int R,
                                  const int *piv, const cx<T> *Ls, int *flag, bool solve = true,
                                  const cx<T> *L1s = nullptr, int ju = 0) {
  constexpr int NB = Tile<T, NTH>::NB;
  const int tid = threadIdx.x;
  if constexpr (sizeof(T) != 4) {
    for (int c = c_begin + tid; c < c_end; c += NTH) {
      cx<T> *col = M + (size_t)c * ld + j0;
      for (int r = 0; r < nb; ++r) {
        const int p = piv[j0 + r] - j0;
        if (p < r || p >= R) continue;   // cannot happen (flagged by the factorisation)
        if (p != r) { const cx<T> a = col[r]; col[r] = col[p]; col[p] = a; }
      }
      for (int r = 1; r < nb && solve; ++r) {
        cx<T> x = col[r];
        for (int s2 = 0; s2 < r; ++s2) {
          const cx<T> l = Ls[r + s2 * NB], y = col[s2];
          x.re -= l.re * y.re - l.im * y.im;
          x.im -= l.re * y.im + l.im * y.re;
        }
        col[r] = x;
      }
    }
    __syncthreads();
  } else {
    __shared__ int s_src[NB], s_dpos[NB], s_dsrc[NB], s_piv[NB], s_nd;
    // the pivots are read in parallel: the fold below is one thread's serial loop
    for (int r = tid; r < nb; r += NTH) s_piv[r] = piv[j0 + r] - j0;
    __syncthreads();
    if (tid == 0) {
      int nd = 0;
      for (int r = 0; r < nb; ++r) s_src[r] = r;
      for (int r = 0; r < nb; ++r) {
        const int p = s_piv[r];
        if (p < r || p >= R) {
          atomicOr(flag, 4);
          continue;
        }
        if (p == r) continue;
        if (p < nb) {
          const int t = s_src[r];
          s_src[r] = s_src[p];
          s_src[p] = t;
          continue;
        }
        int k = 0;
        while (k < nd && s_dpos[k] != p) ++k;
        if (k == nd) {
          s_dpos[nd] = p;
          s_dsrc[nd] = p;
          ++nd;
        }
        const int t = s_src[r];
        s_src[r] = s_dsrc[k];
        s_dsrc[k] = t;
      }
      for (int k = 0; k < nd; ++k)
        if (s_dsrc[k] >= nb) {
          atomicOr(flag, 4);
          nd = 0;
          break;
        }
      s_nd = nd;
    }
    __syncthreads();
    const int nd = s_nd;
    for (int c = c_begin + tid; c < c_end; c += NTH) {
      cx<T> *col = M + (size_t)c * ld + j0;
      cx<T> x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) x[r] = r < nb ? col[s_src[r]] : czero<T>();
      // displaced rows: sources in [0, nb) (still original), targets >= nb
      for (int k0 = 0; k0 < nd; k0 += 8) {
        cx<T> y[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) y[k] = k0 + k < nd ? col[s_dsrc[k0 + k]] : czero<T>();
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k0 + k < nd) col[s_dpos[k0 + k]] = y[k];
      }
      if (L1s) {
        const cx<T> *u1 = M + (size_t)c * ld + ju;
        for (int k = 0; k < NB; ++k) {
          const cx<T> uk = u1[k];
#pragma unroll
          for (int r = 0; r < NB; ++r) {
            const cx<T> l = L1s[r + k * NB];
            x[r].re -= l.re * uk.re - l.im * uk.im;
            x[r].im -= l.re * uk.im + l.im * uk.re;
          }
        }
      }
      if (solve) {
#pragma unroll
        for (int r = 1; r < NB; ++r) {
#pragma unroll
          for (int s2 = 0; s2 < r; ++s2) {
            const cx<T> l = Ls[r + s2 * NB];
            x[r].re -= l.re * x[s2].re - l.im * x[s2].im;
            x[r].im -= l.re * x[s2].im + l.im * x[s2].re;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < nb) col[r] = x[r];
    }
    __syncthreads();
  }
}

// Pieces of a right-looking blocked LU with partial pivoting that eliminates on
// an augmented n x ncols column-major matrix M = [A | B] (leading dimension ld)
// and back-substitutes, i.e. solves A X = B in place (X over B).  Every piece
// is called by all NTH threads of one CTA and ends with a __syncthreads().
//
// lu_panel: unblocked factorisation of columns j0..j0+nb-1 (rows j0..n-1) with
// row pivoting (piv[j] = chosen row), then (right = true) the panel's row
// swaps and U12 = L11^{-1} A12 on every column right of the panel.  `flag` gets bit 1 on
// a zero pivot.  Ls: NB x NB staging in shared memory.
template <typename T, int NTH = NT>
__device__ void lu_panel(cx<T> *M, int ld, int n, int ncols, int j0, int *piv, cx<T> *Ls, T *sval,
                         int *sidx, int *flag, bool right = true) {
  constexpr int NT = NTH;
  constexpr int NB = Tile<T, NTH>::NB;
  const int tid = threadIdx.x;
  const int nb = min(NB, n - j0);
  for (int j = j0; j < j0 + nb; ++j) {
    T best = T(-1);
    int bi = j;
    for (int i = j + tid; i < n; i += NT) {
      const T v = cabs1(M[i + (size_t)j * ld]);
      if (v > best) { best = v; bi = i; }
    }
    const int p = block_argmax<T, NTH>(best, bi, sval, sidx);
    if (tid == 0) piv[j] = p;
    if (p != j) {
      for (int c = j0 + tid; c < j0 + nb; c += NT) {
        const cx<T> a = M[j + (size_t)c * ld];
        M[j + (size_t)c * ld] = M[p + (size_t)c * ld];
        M[p + (size_t)c * ld] = a;
      }
    }
    __syncthreads();
    cx<T> d = M[j + (size_t)j * ld];
    if (d.re == T(0) && d.im == T(0)) {
      if (tid == 0) atomicOr(flag, 1);
      d = mkc<T>(tiny_pivot<T>(), T(0));
    }
    const cx<T> inv = cinv(d);
    for (int i = j + 1 + tid; i < n; i += NT) M[i + (size_t)j * ld] = cmul(M[i + (size_t)j * ld], inv);
    __syncthreads();
    const int rows = n - j - 1, cols = j0 + nb - j - 1;
    for (int e = tid; e < rows * cols; e += NT) {
      const int i = j + 1 + e % rows, c = j + 1 + e / rows;
      cx<T> v = M[i + (size_t)c * ld];
      const cx<T> l = M[i + (size_t)j * ld], u = M[j + (size_t)c * ld];
      v.re -= l.re * u.re - l.im * u.im;
      v.im -= l.re * u.im + l.im * u.re;
      M[i + (size_t)c * ld] = v;
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += NT) {
    const int r = e % nb, s2 = e / nb;
    Ls[r + s2 * NB] = M[j0 + r + (size_t)(j0 + s2) * ld];
  }
  __syncthreads();
  if (right) panel_right_apply<T, NTH>(M, ld, j0 + nb, ncols, j0, nb, n - j0, piv, Ls, flag);
}

// lu_panel with the panel staged in shared memory: P holds rows j0..n-1 of
// the panel's columns (leading dimension n - j0), so every column step of the
// unblocked factorisation (pivot search, row swap, scaling, rank-1 update)
// reads and writes shared memory only.  The right-hand columns then get the
// panel's row swaps and U12 = L11^{-1} A12 (panel_right_apply; with right =
// false that is left to a separate launch over column blocks).  Same pivots,
// same operations and the same result layout as lu_panel (FP32 only: an FP64
// panel of 512 rows does not fit).
template <typename T, int NTH = NT>
__device__ void lu_panel_smem(cx<T> *M, int ld, int n, int ncols, int j0, int *piv, cx<T> *P, cx<T> *Ls,
                              T *sval, int *sidx, int *flag, bool right = true) {
  constexpr int NB = Tile<T, NTH>::NB;
  const int tid = threadIdx.x;
  const int nb = min(NB, n - j0), R = n - j0;
  for (int e = tid; e < R * nb; e += NTH) {
    const int r = e % R, c = e / R;
    P[e] = M[(j0 + r) + (size_t)(j0 + c) * ld];
  }
  __syncthreads();
  // Each thread owns the rows r = tid (mod NTH) for the whole panel: it scales
  // and updates them, and the update of column jj+1 yields its candidates for
  // the next pivot, so a column step needs two barriers (pivot choice, row
  // swap).  Pivot ties go to the smaller row, as in lu_panel.
  T best = T(-1);
  int bi = 0;
  for (int r = tid; r < R; r += NTH) {
    const T v = cabs1(P[r]);
    if (v > best) { best = v; bi = r; }
  }
  for (int jj = 0; jj < nb; ++jj) {
    int p = block_argmax1<T, NTH>(best, bi, sval, sidx);
    if (p < jj || p >= R) {   // cannot happen; recorded rather than followed
      if (tid == 0) atomicOr(flag, 4);
      p = jj;
    }
    if (tid == 0) piv[j0 + jj] = j0 + p;
    if (p != jj) {
      for (int c = tid; c < nb; c += NTH) {
        const cx<T> a = P[jj + c * R];
        P[jj + c * R] = P[p + c * R];
        P[p + c * R] = a;
      }
    }
    __syncthreads();
    cx<T> d = P[jj + jj * R];
    if (d.re == T(0) && d.im == T(0)) {
      if (tid == 0) atomicOr(flag, 1);
      d = mkc<T>(tiny_pivot<T>(), T(0));
    }
    const cx<T> inv = cinv(d);
    best = T(-1);
    bi = jj + 1;
    // rows below the pivot: l = a / d, then a_rc -= l u_c for the panel's
    // remaining columns (u = the pivot row)
    for (int r = (jj + 1) + ((tid - (jj + 1)) % NTH + NTH) % NTH; r < R; r += NTH) {
      const cx<T> l = cmul(P[r + jj * R], inv);
      P[r + jj * R] = l;
      for (int c = jj + 1; c < nb; ++c) {
        cx<T> v = P[r + c * R];
        const cx<T> u = P[jj + c * R];
        v.re -= l.re * u.re - l.im * u.im;
        v.im -= l.re * u.im + l.im * u.re;
        P[r + c * R] = v;
        if (c == jj + 1) {
          const T av = cabs1(v);
          if (av > best) { best = av; bi = r; }
        }
      }
    }
    // the next step's pivot barrier orders these updates before its row swap
  }
  __syncthreads();
  for (int e = tid; e < R * nb; e += NTH) {
    const int r = e % R, c = e / R;
    M[(j0 + r) + (size_t)(j0 + c) * ld] = P[e];
  }
  for (int e = tid; e < nb * nb; e += NTH) {
    const int r = e % nb, s2 = e / nb;
    Ls[r + s2 * NB] = P[r + s2 * R];
  }
  __syncthreads();
  if (right) panel_right_apply<T, NTH>(M, ld, j0 + nb, ncols, j0, nb, R, piv, Ls, flag);
}

// Trailing update of panel j0: M[c0:n, c0:ncols] -= L21 U12 (c0 = j0 + nb);
// output tiles t_first, t_first + t_step, ...
template <typename T, int NTH = NT>
__device__ void lu_trailing(cx<T> *M, int ld, int n, int ncols, int j0, cx<T> *gsm, int t_first = 0,
                            int t_step = 1) {
  constexpr int NB = Tile<T, NTH>::NB;
  const int nb = min(NB, n - j0), c0 = j0 + nb;
  if (c0 >= n || c0 >= ncols) return;
  cta_gemm_t<T, Tile<T, NTH>::BM, Tile<T, NTH>::BN, Tile<T, NTH>::BK, 4, NTH>(
      n - c0, ncols - c0, nb, [=](int i, int l) { return M[c0 + i + (size_t)(j0 + l) * ld]; },
      [=](int l, int j) { return M[j0 + l + (size_t)(c0 + j) * ld]; },
      [=](int i, int j, cx<T> acc) {
        cx<T> &v = M[c0 + i + (size_t)(c0 + j) * ld];
        v = csub(v, acc);
      },
      gsm, t_first, t_step);
}

// Diagonal block j0 of the back substitution: X_b = U_bb^{-1} B_b for the
// right-hand-side columns [c_first, c_last) (a subset of [n, ncols)).
// Ls: 2*NB*NB elements (the FP32 variant keeps the inverted block after it).
template <typename T, int NTH = NT>
__device__ void lu_bs_diag(cx<T> *M, int ld, int n, int j0, int c_first, int c_last, cx<T> *Ls) {
  constexpr int NT = NTH;
  constexpr int NB = Tile<T, NTH>::NB;
  const int tid = threadIdx.x, nb = min(NB, n - j0);
  for (int e = tid; e < nb * nb; e += NT) {
    const int r = e % nb, s2 = e / nb;
    Ls[r + s2 * NB] = M[j0 + r + (size_t)(j0 + s2) * ld];
  }
  __syncthreads();
  if constexpr (std::is_same<T, float>::value) {
    // FP32: X = U11^{-1} B with U11^{-1} formed once per block in shared memory
    // (column j by back substitution on e_j: one warp per column, lane r holding
    // row r, solved values passed by shuffles), then every RHS column is an
    // independent triangular matrix-vector product
    static_assert(NB == 32, "one lane per row of a diagonal block");
    cx<T> *Ui = Ls + NB * NB;   // NB x NB, upper triangular
    const int warp = tid >> 5, lane = tid & 31;
    for (int j = warp; j < nb; j += NT / 32) {
      cx<T> x = mkc<T>(lane == j ? T(1) : T(0), T(0));
      for (int s2 = j; s2 >= 0; --s2) {
        if (lane == s2) x = cdiv(x, Ls[s2 + s2 * NB]);
        const cx<T> xs = mkc<T>(__shfl_sync(0xffffffffu, x.re, s2), __shfl_sync(0xffffffffu, x.im, s2));
        if (lane < s2) {
          const cx<T> u = Ls[lane + s2 * NB];
          x.re -= u.re * xs.re - u.im * xs.im;
          x.im -= u.re * xs.im + u.im * xs.re;
        }
      }
      if (lane < nb) Ui[lane + j * NB] = lane <= j ? x : czero<T>();
    }
    __syncthreads();
    for (int c = c_first + tid; c < c_last; c += NT) {
      cx<T> *col = M + (size_t)c * ld + j0;
      cx<T> x[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) x[r] = czero<T>();
#pragma unroll
      for (int s2 = 0; s2 < NB; ++s2) {
        if (s2 < nb) {
          const cx<T> b = col[s2];
#pragma unroll
          for (int r = 0; r <= s2; ++r) cfma(x[r], Ui[r + s2 * NB], b);
        }
      }
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < nb) col[r] = x[r];
    }
  } else {
    for (int c = c_first + tid; c < c_last; c += NT) {
      cx<T> *col = M + (size_t)c * ld + j0;
      for (int r = nb - 1; r >= 0; --r) {
        cx<T> x = col[r];
        for (int s2 = r + 1; s2 < nb; ++s2) {
          const cx<T> u = Ls[r + s2 * NB], y = col[s2];
          x.re -= u.re * y.re - u.im * y.im;
          x.im -= u.re * y.im + u.im * y.re;
        }
        col[r] = cdiv(x, Ls[r + r * NB]);
      }
    }
  }
  __syncthreads();
}

// lu_bs_diag for the FP32 sweep with its right-hand-side columns staged in
// shared memory: the columns [c_first, c_last) of rows j0 .. j0+nb-1 are read
// and written back row-contiguous (coalesced), each thread solves one column
// from the padded staging copy, and the inverse of the diagonal block is
// formed with the diagonal's reciprocals taken once.  smem: 2 NB^2 + NB +
// (c_last - c_first) (NB + 1) complex.
template <int NTH>
__device__ void lu_bs_diag_staged(cc *M, int ld, int n, int j0, int c_first, int c_last, cc *smem) {
  constexpr int NT = NTH, NB = Tile<float, NTH>::NB, LDB = NB + 1;
  static_assert(NB == 32, "one lane per row of a diagonal block");
  cc *Ls = smem, *Ui = Ls + NB * NB, *dinv = Ui + NB * NB, *Bs = dinv + NB;
  const int tid = threadIdx.x, nb = min(NB, n - j0), ncol = c_last - c_first;
  for (int e = tid; e < nb * nb; e += NT) {
    const int r = e % nb, s2 = e / nb;
    Ls[r + s2 * NB] = M[j0 + r + (size_t)(j0 + s2) * ld];
  }
  if (tid < nb) dinv[tid] = cinv(M[j0 + tid + (size_t)(j0 + tid) * ld]);
  for (int e = tid; e < nb * ncol; e += NT) {
    const int r = e % nb, c = e / nb;
    Bs[r + c * LDB] = M[j0 + r + (size_t)(c_first + c) * ld];
  }
  __syncthreads();
  // U11^{-1}, column j by back substitution on e_j (one warp per column, lane
  // r holding row r, solved values passed by shuffles)
  const int warp = tid >> 5, lane = tid & 31;
  for (int j = warp; j < nb; j += NT / 32) {
    cc x = mkc<float>(lane == j ? 1.f : 0.f, 0.f);
    for (int s2 = j; s2 >= 0; --s2) {
      if (lane == s2) x = cmul(x, dinv[s2]);
      const cc xs = mkc<float>(__shfl_sync(0xffffffffu, x.re, s2), __shfl_sync(0xffffffffu, x.im, s2));
      if (lane < s2) {
        const cc u = Ls[lane + s2 * NB];
        x.re -= u.re * xs.re - u.im * xs.im;
        x.im -= u.re * xs.im + u.im * xs.re;
      }
    }
    if (lane < nb) Ui[lane + j * NB] = lane <= j ? x : czero<float>();
  }
  __syncthreads();
  for (int c = tid; c < ncol; c += NT) {
    cc *col = Bs + c * LDB;
    cc x[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) x[r] = czero<float>();
#pragma unroll
    for (int s2 = 0; s2 < NB; ++s2) {
      if (s2 < nb) {
        const cc b = col[s2];
#pragma unroll
        for (int r = 0; r <= s2; ++r) cfma(x[r], Ui[r + s2 * NB], b);
      }
    }
#pragma unroll
    for (int r = 0; r < NB; ++r)
      if (r < nb) col[r] = x[r];
  }
  __syncthreads();
  for (int e = tid; e < nb * ncol; e += NT) {
    const int r = e % nb, c = e / nb;
    M[j0 + r + (size_t)(c_first + c) * ld] = Bs[r + c * LDB];
  }
}

inline size_t lu_bs_diag_staged_smem(int ncol) {
  return ((size_t)2 * 32 * 32 + 32 + (size_t)ncol * 33) * sizeof(cc);
}


// Back-substitution update above block j0: M[0:j0, n:ncols] -= U[0:j0, b] X_b.
template <typename T, int NTH = NT>
__device__ void lu_bs_update(cx<T> *M, int ld, int n, int ncols, int j0, cx<T> *gsm, int t_first = 0,
                             int t_step = 1) {
  constexpr int NB = Tile<T, NTH>::NB;
  const int nb = min(NB, n - j0);
  if (j0 <= 0) return;
  cta_gemm_t<T, Tile<T, NTH>::BM, Tile<T, NTH>::BN, Tile<T, NTH>::BK, 4, NTH>(
      j0, ncols - n, nb, [=](int i, int l) { return M[i + (size_t)(j0 + l) * ld]; },
      [=](int l, int j) { return M[j0 + l + (size_t)(n + j) * ld]; },
      [=](int i, int j, cx<T> acc) {
        cx<T> &v = M[i + (size_t)(n + j) * ld];
        v = csub(v, acc);
      },
      gsm, t_first, t_step);
}

// Solves A X = B in place for the n x n matrix A held in columns [0, n) of the
// n x ncols column-major M (leading dimension ld) and the right-hand sides in
// columns [n, ncols): the pieces above run one after the other in one CTA.
// smem: gemm_smem_elems<T, NTH>() + NB*NB complex, plus sval/sidx scratch.
template <typename T, int NTH = NT>
__device__ void cta_lu_solve(cx<T> *M, int ld, int n, int ncols, int *piv, cx<T> *smem,
                             T *sval, int *sidx, int *flag) {
  constexpr int NB = Tile<T, NTH>::NB;
  cx<T> *Ls = smem + gemm_smem_elems<T, NTH>();
  for (int j0 = 0; j0 < n; j0 += NB) {
    lu_panel<T, NTH>(M, ld, n, ncols, j0, piv, Ls, sval, sidx, flag);
    lu_trailing<T, NTH>(M, ld, n, ncols, j0, smem);
  }
  const int jlast = ((n - 1) / NB) * NB;
  for (int j0 = jlast; j0 >= 0; j0 -= NB) {
    lu_bs_diag<T, NTH>(M, ld, n, j0, n, ncols, Ls);
    lu_bs_update<T, NTH>(M, ld, n, ncols, j0, smem);
  }
  __syncthreads();
}

// Applies a factorisation made by cta_lu_solve (LU held in the n x n
// column-major block `LU`, row swaps `piv`) to new right-hand sides B (n x nrhs,
// leading dimension ldb): replays the same panel-by-panel elimination, then
// back-substitutes, so B <- A^{-1} B.  smem: skinny_smem_elems + NB*NB.
// Per block of NB = 32 rows, the block's row swaps are folded into a gather
// (as in panel_right_apply) and each right-hand side is solved by one warp,
// lane r holding row r (the diagonal block from shared memory, the solved
// values passed by shuffles), so no step waits on a global-memory round trip.
// order says how the factors were stored:
//   0  each panel's swaps reached only the columns right of it;
//   1  (lapack) P A = L U: every panel's swaps reached the L columns left of
//      it (the tensor-core FP32 sweep with 128-row blocks): B <- P B first,
//      then the blocks without swaps;
//   2  panels in pairs (the tensor-core FP32 sweep's default): the second
//      panel of a pair also swapped the first panel's L rows below it, so the
//      replay applies the second block's swaps before the first block's
//      update of the rows below, and none at the second block.
// Needs n <= 1024.
template <typename T, int NTH = NT>
__device__ void cta_lu_replay(const cx<T> *LU, int n, const int *piv, cx<T> *B, int ldb, int nrhs,
                              cx<T> *smem, int order = 0) {
  const bool lapack = order == 1;
  constexpr int NB = Tile<T, NTH>::NB;
  static_assert(NB == 32, "one lane per row of a diagonal block");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  cx<T> *Ls = smem + skinny_smem_elems<T>();
  __shared__ int s_src[NB], s_dpos[NB], s_dsrc[NB], s_piv[NB], s_nd;
  auto shfl = [](cx<T> v, int src) {
    return mkc<T>(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
  };
  if (lapack) {
    __shared__ int s_perm[1024];
    __shared__ cx<T> s_col[1024];
    if (tid == 0) {
      for (int r = 0; r < n; ++r) s_perm[r] = r;
      for (int j = 0; j < n; ++j) {
        const int p = piv[j];
        if (p > j && p < n) {
          const int t = s_perm[j];
          s_perm[j] = s_perm[p];
          s_perm[p] = t;
        }
      }
    }
    for (int c = 0; c < nrhs; ++c) {
      __syncthreads();
      for (int r = tid; r < n; r += NTH) s_col[r] = B[r + (size_t)c * ldb];
      __syncthreads();
      for (int r = tid; r < n; r += NTH) B[r + (size_t)c * ldb] = s_col[s_perm[r]];
    }
    __syncthreads();
  }
  // the swaps of rows jb .. jb+nbb-1 (piv relative to jb, R rows from jb) as
  // a gather: s_src, and s_nd displaced rows s_dpos <- s_dsrc (tid 0)
  auto fold = [&](int nbb, int R) {
    int nd = 0;
    for (int r = 0; r < nbb; ++r) s_src[r] = r;
    for (int r = 0; r < nbb; ++r) {
      const int p = s_piv[r];
      if (p <= r || p >= R) continue;   // p < r or out of range cannot come from the factorisation
      if (p < nbb) {
        const int t = s_src[r];
        s_src[r] = s_src[p];
        s_src[p] = t;
        continue;
      }
      int k = 0;
      while (k < nd && s_dpos[k] != p) ++k;
      if (k == nd) {
        s_dpos[nd] = p;
        s_dsrc[nd] = p;
        ++nd;
      }
      const int t = s_src[r];
      s_src[r] = s_dsrc[k];
      s_dsrc[k] = t;
    }
    for (int k = 0; k < nd; ++k)
      if (s_dsrc[k] >= nbb) nd = 0;   // cannot happen (the fold keeps displaced sources in the block)
    s_nd = nd;
  };
  bool ahead = false;   // order 2: this block's swaps were applied with the block before
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int nb = min(NB, n - j0), R = n - j0;
    for (int e = tid; e < nb * nb; e += NTH) {
      const int r = e % nb, c = e / nb;
      Ls[r + c * NB] = LU[j0 + r + (size_t)(j0 + c) * n];
    }
    // lapack: B is already in pivot order, so the block's swaps are identities
    if (tid < nb) s_piv[tid] = (lapack || ahead) ? tid : piv[j0 + tid] - j0;
    __syncthreads();
    if (tid == 0) fold(nb, R);
    __syncthreads();
    const int nd = s_nd;
    for (int c = warp; c < nrhs; c += NTH / 32) {
      cx<T> *col = B + (size_t)c * ldb + j0;
      cx<T> x = lane < nb ? col[s_src[lane]] : czero<T>();
      const cx<T> y = lane < nd ? col[s_dsrc[lane]] : czero<T>();
      __syncwarp();
      if (lane < nd) col[s_dpos[lane]] = y;
      // x <- L11^{-1} x (unit lower triangular)
      for (int s2 = 0; s2 + 1 < nb; ++s2) {
        const cx<T> xs = shfl(x, s2);
        if (lane > s2 && lane < nb) {
          const cx<T> l = Ls[lane + s2 * NB];
          x.re -= l.re * xs.re - l.im * xs.im;
          x.im -= l.re * xs.im + l.im * xs.re;
        }
      }
      if (lane < nb) col[lane] = x;
    }
    __syncthreads();
    // order 2, first block of a pair: the rows below take the second block's
    // swaps now, matching the first block's L rows (which took them too)
    ahead = order == 2 && !ahead && (j0 / NB) % 2 == 0 && j0 + NB < n;
    if (ahead) {
      const int j1 = j0 + NB, nb1 = min(NB, n - j1);
      if (tid < nb1) s_piv[tid] = piv[j1 + tid] - j1;
      __syncthreads();
      if (tid == 0) fold(nb1, n - j1);
      __syncthreads();
      const int nd1 = s_nd;
      for (int c = warp; c < nrhs; c += NTH / 32) {
        cx<T> *col = B + (size_t)c * ldb + j1;
        const cx<T> x = lane < nb1 ? col[s_src[lane]] : czero<T>();
        const cx<T> y = lane < nd1 ? col[s_dsrc[lane]] : czero<T>();
        __syncwarp();
        if (lane < nd1) col[s_dpos[lane]] = y;
        if (lane < nb1) col[lane] = x;
      }
      __syncthreads();
    }
    if (j0 + nb < n) {
      const int c0 = j0 + nb;
      cta_gemm_skinny<T, NTH>(
          n - c0, nrhs, nb, [=](int i, int l) { return LU[c0 + i + (size_t)(j0 + l) * n]; },
          [=](int l, int j) { return B[j0 + l + (size_t)j * ldb]; },
          [=](int i, int j, cx<T> acc) {
            cx<T> &v = B[c0 + i + (size_t)j * ldb];
            v = csub(v, acc);
          },
          smem);
    }
  }
  const int jlast = ((n - 1) / NB) * NB;
  for (int j0 = jlast; j0 >= 0; j0 -= NB) {
    const int nb = min(NB, n - j0);
    for (int e = tid; e < nb * nb; e += NTH) {
      const int r = e % nb, c = e / nb;
      Ls[r + c * NB] = LU[j0 + r + (size_t)(j0 + c) * n];
    }
    __syncthreads();
    for (int c = warp; c < nrhs; c += NTH / 32) {
      cx<T> *col = B + (size_t)c * ldb + j0;
      cx<T> x = lane < nb ? col[lane] : czero<T>();
      // x <- U11^{-1} x
      for (int s2 = nb - 1; s2 >= 0; --s2) {
        if (lane == s2) x = cdiv(x, Ls[s2 + s2 * NB]);
        const cx<T> xs = shfl(x, s2);
        if (lane < s2) {
          const cx<T> u = Ls[lane + s2 * NB];
          x.re -= u.re * xs.re - u.im * xs.im;
          x.im -= u.re * xs.im + u.im * xs.re;
        }
      }
      if (lane < nb) col[lane] = x;
    }
    __syncthreads();
    if (j0 > 0) {
      cta_gemm_skinny<T, NTH>(
          j0, nrhs, nb, [=](int i, int l) { return LU[i + (size_t)(j0 + l) * n]; },
          [=](int l, int j) { return B[j0 + l + (size_t)j * ldb]; },
          [=](int i, int j, cx<T> acc) {
            cx<T> &v = B[i + (size_t)j * ldb];
            v = csub(v, acc);
          },
          smem);
    }
  }
  __syncthreads();
}

}  // namespace pw
