// Fifth-generation tensor-core building blocks (sm_100a / sm_103a): tcgen05
// MMA with operands in shared memory and the accumulator in tensor memory
// (TMEM), completion through an mbarrier, results read back with tcgen05.ld.
//
// Operand layout: "K-major, no swizzle".  A tile of R rows by K elements is a
// grid of core matrices of 8 rows x 16 bytes (8 rows x 4 FP32/TF32 values),
// each stored as 128 contiguous bytes (row r of the core matrix at 16 r).
// The shared-memory matrix descriptor gives the byte distance between core
// matrices that are adjacent along K (leading byte offset, LBO) and along the
// rows (stride byte offset, SBO).  Here LBO = 128 (the two K-chunks of one MMA
// step are adjacent) and SBO = 256, so one MMA step (K = 8 for TF32) of an
// R-row operand occupies R * 32 contiguous bytes.
//
// Every wait is bounded: a wait that runs out records an error and returns.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "pw_cx.cuh"

namespace pw {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05 format, no swizzle).
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = smem_u32(p);
  uint64_t d = (uint64_t)((a & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;   // descriptor version of the tcgen05 family
  return d;          // base offset 0, relative LBO mode, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4)                      // D format: FP32
         | (2u << 7)                    // A format: TF32
         | (2u << 10)                   // B format: TF32
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

// Instruction descriptor of kind::f16 with BF16 A and B, D FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                      // D format: FP32
         | (1u << 7)                    // A format: BF16
         | (1u << 10)                   // B format: BF16
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

// Instruction descriptor of kind::f16 with FP16 A and B, D FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4)                      // D format: FP32
         | ((uint32_t)(N >> 3) << 17)   // N / 8 (A and B format 0: FP16)
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

// TMEM allocation by one full warp; the address is written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] B[smem], issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// D[tmem] (+)= A[smem] B[smem] with BF16 operands (K = 16 per instruction).
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Asynchronous 16-byte global -> shared copy (cp.async, L2 only); with
// valid == false nothing is read and the 16 bytes are zero-filled.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// every group of this thread but the newest N has landed
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// D[tmem] (+)= A[smem] B[smem], kind::f16 (16-bit A and B, K = 16 per instruction).
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on the mbarrier once every MMA issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// One arrival on the mbarrier by this thread (no transaction bytes).
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// Bounded wait for the phase with the given parity; false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint32_t max_polls = 1u << 22) {
  for (uint32_t i = 0; i < max_polls; ++i) {
    if (mbar_try_wait(mbar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory writes become visible to the tensor core.
__device__ __forceinline__ void fence_smem_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 TMEM lanes x 16 consecutive 32-bit columns: thread t of the warp gets
// lane (lane field of taddr) + t, columns col .. col + 15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 TMEM lanes x 8 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Round to TF32 (10 explicit mantissa bits), nearest with ties away.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row, k) of a K-major no-swizzle operand whose MMA
// steps of 8 K-values are stored one after another (rows x 32 bytes each).
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int row, int k, int rows) {
  const int step = k >> 3, kk = k & 7;
  return (uint32_t)step * (uint32_t)rows * 32u + (uint32_t)(row >> 3) * 256u + (uint32_t)(kk >> 2) * 128u +
         (uint32_t)(row & 7) * 16u + (uint32_t)(kk & 3) * 4u;
}

// ---------------------------------------------------------------------------
// Complex FP32 GEMM tile on tcgen05 with FP32-level accuracy.
//
// The complex product C = A B is the real product of
//   A' (rows 2r, 2r+1; inner columns 2l, 2l+1) = [[Re A, -Im A], [Im A, Re A]]
//   B' (inner rows 2l, 2l+1; columns j)         = [Re B ; Im B],
// so row 2r of D holds Re C(r, .) and row 2r+1 holds Im C(r, .).  Each
// operand is split into TF32 hi + lo parts, D = A'_hi B'_hi + A'_hi B'_lo +
// A'_lo B'_hi, accumulated in FP32 in tensor memory.  The CTA (CG_THREADS
// threads) computes complex rows [r0, r0 + 64) x columns [c0, c0 + 128) of C
// (m x ncol, inner k), K in stages of 8 complex values (two MMA steps of 8
// real), double-buffered in shared memory so that the CTA stages block s+1
// while the tensor core multiplies block s.  fa(i, l) and fb(l, j) return the
// operands (zero outside the matrix is supplied here), fe(i, j, acc) consumes
// each in-range result.  smem: cg_smem_bytes().  Returns false (and skips fe)
// if the tensor core did not signal completion within the bounded waits.
constexpr int CG_THREADS = 256;
constexpr int CG_M = 128, CG_N = 128, CG_KC = 8;   // real rows, complex columns, complex K per stage
constexpr int CG_AB = CG_M * 2 * CG_KC * 4;        // bytes of one A' part (hi or lo) per stage
// bytes of one B' part per stage, of one stage, of the tile's shared memory
// for TN complex columns (64 or 128)
template <int TN>
__host__ __device__ constexpr int cg_bb() { return TN * 2 * CG_KC * 4; }
template <int TN>
__host__ __device__ constexpr int cg_stage() { return 2 * CG_AB + 2 * cg_bb<TN>(); }
template <int TN = CG_N>
__host__ __device__ constexpr size_t cg_smem_bytes() { return 2 * (size_t)cg_stage<TN>() + 64; }

// Four values as TF32 hi parts and FP32 remainders, one 16-byte store each.
__device__ __forceinline__ void store_split(unsigned char *hi_base, unsigned char *lo_base, uint32_t off, float a,
                                            float b, float c, float d) {
  const float4 h = make_float4(to_tf32(a), to_tf32(b), to_tf32(c), to_tf32(d));
  *reinterpret_cast<float4 *>(hi_base + off) = h;
  *reinterpret_cast<float4 *>(lo_base + off) = make_float4(a - h.x, b - h.y, c - h.z, d - h.w);
}

// Operands of one K stage as this thread loads them (the staging is
// software-pipelined: the loads of stage s+1 are in flight while stage s is
// split into shared memory and multiplied).
struct CgStage {
  cc a0, a1;   // A task: complex (r, l), (r, l+1)
  cc b[4];     // B tasks
};
static_assert((CG_M / 2) * (CG_KC / 2) == CG_THREADS, "one A task per thread and stage");

// The tile is 64 complex rows x TN complex columns (TN = 64 or 128).
// B_RUNS: fb(l .. l+3, j) lie contiguously in memory for fixed j (one thread
// reads the run); otherwise consecutive j are contiguous for fixed l (one
// thread per column, consecutive threads on consecutive columns).
// RMW: the result updates an existing C; fc(i, j) reads it, and the reads of
// this thread's results are issued before the first stage so that they are in
// flight during the whole product.  fe(i, j, acc, c) receives the old value c
// (zero when !RMW).
template <bool B_RUNS, bool RMW, int TN = CG_N, class FA, class FB, class FC, class FE>
__device__ bool cgemm_tile(int m, int ncol, int k, int r0, int c0, FA fa, FB fb, FC fc, FE fe,
                           unsigned char *smem) {
  static_assert(TN == 64 || TN == 128, "tile width");
  constexpr int BB = cg_bb<TN>(), STAGE = cg_stage<TN>();
  constexpr int BTASKS = B_RUNS ? TN * 2 : TN * (CG_KC / 2);   // B tasks per stage
  constexpr int BPER = (BTASKS + CG_THREADS - 1) / CG_THREADS;  // per thread
  static_assert(BPER * (B_RUNS ? 4 : 2) <= 4, "B staging registers");
  constexpr int NCH = TN / 16;                                  // 8-column chunks per warp
  unsigned char *stage0 = smem;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 2 * STAGE);   // [2]
  uint32_t *slot = reinterpret_cast<uint32_t *>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const cc zero = czero<float>();
  auto load = [&](int s, CgStage &t) {
    const int l0 = s * CG_KC;
    {
      const int rr = tid % (CG_M / 2), lp = tid / (CG_M / 2);
      const int r = r0 + rr, l = l0 + 2 * lp;
      t.a0 = (r < m && l < k) ? fa(r, l) : zero;
      t.a1 = (r < m && l + 1 < k) ? fa(r, l + 1) : zero;
    }
#pragma unroll
    for (int u = 0; u < BPER; ++u) {
      const int e = tid + u * CG_THREADS;
      if (e >= BTASKS) break;
      if (B_RUNS) {
        const int jj = e % TN, half = e / TN;
        const int j = c0 + jj, l = l0 + 4 * half;
#pragma unroll
        for (int q = 0; q < 4; ++q) t.b[q] = (l + q < k && j < ncol) ? fb(l + q, j) : zero;
      } else {
        const int jj = e % TN, lp = e / TN;
        const int j = c0 + jj, l = l0 + 2 * lp;
        t.b[2 * u] = (l < k && j < ncol) ? fb(l, j) : zero;
        t.b[2 * u + 1] = (l + 1 < k && j < ncol) ? fb(l + 1, j) : zero;
      }
    }
  };
  auto store = [&](unsigned char *Ahi, unsigned char *Alo, unsigned char *Bhi, unsigned char *Blo,
                   const CgStage &t) {
    {
      // A': complex (r, l), (r, l+1) -> real rows 2r, 2r+1, one 16-byte chunk each
      const int rr = tid % (CG_M / 2), lp = tid / (CG_M / 2);
      store_split(Ahi, Alo, kmajor_offset(2 * rr, 4 * lp, CG_M), t.a0.re, -t.a0.im, t.a1.re, -t.a1.im);
      store_split(Ahi, Alo, kmajor_offset(2 * rr + 1, 4 * lp, CG_M), t.a0.im, t.a0.re, t.a1.im, t.a1.re);
    }
#pragma unroll
    for (int u = 0; u < BPER; ++u) {
      const int e = tid + u * CG_THREADS;
      if (e >= BTASKS) break;
      if (B_RUNS) {
        const int jj = e % TN, half = e / TN;
        store_split(Bhi, Blo, kmajor_offset(jj, 8 * half, TN), t.b[0].re, t.b[0].im, t.b[1].re, t.b[1].im);
        store_split(Bhi, Blo, kmajor_offset(jj, 8 * half + 4, TN), t.b[2].re, t.b[2].im, t.b[3].re, t.b[3].im);
      } else {
        const int jj = e % TN, lp = e / TN;
        store_split(Bhi, Blo, kmajor_offset(jj, 4 * lp, TN), t.b[2 * u].re, t.b[2 * u].im, t.b[2 * u + 1].re,
                    t.b[2 * u + 1].im);
      }
    }
  };
  // epilogue mapping: warp w reads TMEM lanes 32 (w % 4) .. (real rows) and
  // complex columns (TN / 2) (w / 4) .. + TN / 2 in chunks of 8; of a lane
  // pair (real and imaginary row of one complex row) the real-row lane writes
  // columns 0 .. 3 of each chunk, the imaginary-row lane 4 .. 7
  const int lrow = 32 * (warp & 3) + lane;
  const int er = r0 + (lrow >> 1), eim = lrow & 1;
  auto ecol = [&](int q) { return c0 + (TN / 2) * (warp >> 2) + 8 * q + (eim ? 4 : 0); };
  CgStage cur;
  load(0, cur);
  cc cold[RMW ? NCH : 1][4];
  if constexpr (RMW) {
#pragma unroll
    for (int q = 0; q < NCH; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int j = ecol(q) + i;
        cold[q][i] = (er < m && j < ncol) ? fc(er, j) : zero;
      }
  }
  if (warp == 0) tmem_alloc(slot, TN);
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *slot;
  const int nstage = (k + CG_KC - 1) / CG_KC;
  bool ok = true;
  for (int s = 0; s < nstage; ++s) {
    const int b = s & 1;
    unsigned char *Ahi = stage0 + b * STAGE, *Alo = Ahi + CG_AB;
    unsigned char *Bhi = Alo + CG_AB, *Blo = Bhi + BB;
    if (s >= 2) ok = mbar_wait(&mbar[b], ((s - 2) >> 1) & 1) && ok;   // buffer b is free again
    store(Ahi, Alo, Bhi, Blo, cur);
    if (s + 1 < nstage) load(s + 1, cur);
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      constexpr uint32_t idesc = idesc_tf32(CG_M, TN);
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint64_t ah = smem_desc(Ahi + ks * CG_M * 32, 128, 256);
        const uint64_t al = smem_desc(Alo + ks * CG_M * 32, 128, 256);
        const uint64_t bh = smem_desc(Bhi + ks * TN * 32, 128, 256);
        const uint64_t bl = smem_desc(Blo + ks * TN * 32, 128, 256);
        mma_tf32(tmem, ah, bh, idesc, (s > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, ah, bl, idesc, 1u);
        mma_tf32(tmem, al, bh, idesc, 1u);
      }
      mma_commit(&mbar[b]);
    }
  }
  // the last commit covers every MMA of the tile
  ok = mbar_wait(&mbar[(nstage - 1) & 1], ((nstage - 1) >> 1) & 1) && ok;
  fence_after_sync();
  if (ok) {
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      float vv[8], other[8];
      tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((TN / 2) * (warp >> 2) + 8 * q), vv);
#pragma unroll
      for (int i = 0; i < 8; ++i) other[i] = __shfl_xor_sync(0xffffffffu, vv[i], 1);
      const int jb = ecol(q);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const cc acc = eim ? mkc<float>(other[i + 4], vv[i + 4]) : mkc<float>(vv[i], other[i]);
        if (er < m && jb + i < ncol) fe(er, jb + i, acc, RMW ? cold[RMW ? q : 0][i] : zero);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TN);
  return ok;
}

// ---------------------------------------------------------------------------
// Four complex products sharing one B operand: D_{2h} = A_h B and
// D_{2h+1} = (A_h S_h) B for h = 0, 1, S_h = diag(s_h(l)) a column scaling
// (D_q active when bit q of amask is set), same split, layout and pipeline as
// cgemm_tile with TN = 128; the four accumulators fill the SM's tensor memory
// (4 x 128 columns), so the kernel runs one CTA per SM.  Staging one B tile
// for four A tiles quarters the B staging work per MMA, and A_h is loaded
// once for both of its products.  fa(h, i, l) and fb(l, j) load the operands
// (with ldg_cc: issued where written, so two stages of loads stay in
// flight), fs(h, l) gives s_h(l); fe(i, j, x) receives x[q] = D_q(i, j) (zero
// for inactive q).
constexpr int C4 = 4;
__host__ __device__ constexpr size_t c4_stage() { return (size_t)C4 * 2 * CG_AB + 2 * (size_t)cg_bb<CG_N>(); }
__host__ __device__ constexpr size_t c4_smem_bytes() { return 2 * c4_stage() + 64; }

// One complex FP32 value from global memory, issued at this point of the
// program (the compiler may not sink it towards its use).
__device__ __forceinline__ cc ldg_cc(const cc *p) {
  float re, im;
  asm volatile("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(re), "=f"(im) : "l"(p));
  return mkc<float>(re, im);
}

template <class FA, class FS, class FB, class FE>
__device__ bool cgemm_tile_shared_b(int m, int ncol, int k, int r0, int c0, unsigned amask, FA fa, FS fs, FB fb,
                                    FE fe, unsigned char *smem) {
  constexpr int TN = CG_N, BB = cg_bb<CG_N>();
  constexpr size_t STAGE = c4_stage();
  constexpr int NCH = TN / 16;
  unsigned char *stage0 = smem;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 2 * STAGE);   // [2]
  uint32_t *slot = reinterpret_cast<uint32_t *>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const cc zero = czero<float>();
  struct Stg {
    cc a[2][2];   // A_h (r, l), (r, l+1)
    cc b[4];
  };
  auto load = [&](int s, Stg &t) {
    const int l0 = s * CG_KC;
    const int rr = tid % (CG_M / 2), lp = tid / (CG_M / 2);
    const int r = r0 + rr, l = l0 + 2 * lp;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool on = (amask >> (2 * h)) & 3u;
      t.a[h][0] = (on && r < m && l < k) ? fa(h, r, l) : zero;
      t.a[h][1] = (on && r < m && l + 1 < k) ? fa(h, r, l + 1) : zero;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * CG_THREADS;
      const int jj = e % TN, lq = e / TN;
      const int j = c0 + jj, lb = l0 + 2 * lq;
      t.b[2 * u] = (lb < k && j < ncol) ? fb(lb, j) : zero;
      t.b[2 * u + 1] = (lb + 1 < k && j < ncol) ? fb(lb + 1, j) : zero;
    }
  };
  auto store = [&](unsigned char *base, int s, const Stg &t) {
    const int rr = tid % (CG_M / 2), lp = tid / (CG_M / 2);
    const int l = s * CG_KC + 2 * lp;
#pragma unroll
    for (int q = 0; q < C4; ++q) {
      if (!((amask >> q) & 1u)) continue;
      const int h = q >> 1;
      cc a0 = t.a[h][0], a1 = t.a[h][1];
      if (q & 1) {
        if (l < k) a0 = cmul(a0, fs(h, l));
        if (l + 1 < k) a1 = cmul(a1, fs(h, l + 1));
      }
      unsigned char *Ahi = base + (size_t)q * 2 * CG_AB, *Alo = Ahi + CG_AB;
      store_split(Ahi, Alo, kmajor_offset(2 * rr, 4 * lp, CG_M), a0.re, -a0.im, a1.re, -a1.im);
      store_split(Ahi, Alo, kmajor_offset(2 * rr + 1, 4 * lp, CG_M), a0.im, a0.re, a1.im, a1.re);
    }
    unsigned char *Bhi = base + (size_t)C4 * 2 * CG_AB, *Blo = Bhi + BB;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * CG_THREADS;
      const int jj = e % TN, lq = e / TN;
      store_split(Bhi, Blo, kmajor_offset(jj, 4 * lq, TN), t.b[2 * u].re, t.b[2 * u].im, t.b[2 * u + 1].re,
                  t.b[2 * u + 1].im);
    }
  };
  const int lrow = 32 * (warp & 3) + lane;
  const int er = r0 + (lrow >> 1), eim = lrow & 1;
  // two register stages in flight: the loads of stage s+2 are issued while
  // stage s is split and multiplied (one CTA per SM leaves few warps to hide
  // the memory latency otherwise)
  Stg st0, st1;
  const int nstage = (k + CG_KC - 1) / CG_KC;
  load(0, st0);
  if (nstage > 1) load(1, st1);
  if (warp == 0) tmem_alloc(slot, C4 * TN);
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *slot;
  bool ok = true;
  auto step = [&](int s, Stg &t) {
    const int b = s & 1;
    unsigned char *base = stage0 + b * STAGE;
    if (s >= 2) ok = mbar_wait(&mbar[b], ((s - 2) >> 1) & 1) && ok;   // buffer b is free again
    store(base, s, t);
    if (s + 2 < nstage) load(s + 2, t);
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      constexpr uint32_t idesc = idesc_tf32(CG_M, TN);
      const unsigned char *Bhi = base + (size_t)C4 * 2 * CG_AB, *Blo = Bhi + BB;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint64_t bh = smem_desc(Bhi + ks * TN * 32, 128, 256);
        const uint64_t bl = smem_desc(Blo + ks * TN * 32, 128, 256);
#pragma unroll
        for (int q = 0; q < C4; ++q) {
          if (!((amask >> q) & 1u)) continue;
          const unsigned char *Ahi = base + (size_t)q * 2 * CG_AB, *Alo = Ahi + CG_AB;
          const uint64_t ah = smem_desc(Ahi + ks * CG_M * 32, 128, 256);
          const uint64_t al = smem_desc(Alo + ks * CG_M * 32, 128, 256);
          const uint32_t d = tmem + (uint32_t)(q * TN);
          mma_tf32(d, ah, bh, idesc, (s > 0 || ks > 0) ? 1u : 0u);
          mma_tf32(d, ah, bl, idesc, 1u);
          mma_tf32(d, al, bh, idesc, 1u);
        }
      }
      mma_commit(&mbar[b]);
    }
  };
  for (int s = 0; s < nstage; s += 2) {
    step(s, st0);
    if (s + 1 < nstage) step(s + 1, st1);
  }
  ok = mbar_wait(&mbar[(nstage - 1) & 1], ((nstage - 1) >> 1) & 1) && ok;
  fence_after_sync();
  if (ok) {
#pragma unroll 1
    for (int qq = 0; qq < NCH; ++qq) {
      float vv[C4][8], other[C4][8];
#pragma unroll
      for (int q = 0; q < C4; ++q) {
        if ((amask >> q) & 1u) {
          tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(q * TN + (TN / 2) * (warp >> 2) + 8 * qq),
                   vv[q]);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) vv[q][i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) other[q][i] = __shfl_xor_sync(0xffffffffu, vv[q][i], 1);
      }
      const int jb = c0 + (TN / 2) * (warp >> 2) + 8 * qq + (eim ? 4 : 0);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        cc x[C4];
#pragma unroll
        for (int q = 0; q < C4; ++q)
          x[q] = eim ? mkc<float>(other[q][i + 4], vv[q][i + 4]) : mkc<float>(vv[q][i], other[q][i]);
        if (er < m && jb + i < ncol) fe(er, jb + i, x);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, C4 * TN);
  return ok;
}

// ---------------------------------------------------------------------------
// The four-accumulator tile of cgemm_tile_shared_b with an FP16 split in
// place of the TF32 one.  Each real operand value x becomes hi = fp16(x) and
// lo = fp16(x - hi); A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 carries about
// 22 bits, like the TF32 split, but kind::f16 runs at twice the rate of
// kind::tf32 and the staged operands take half the bytes, so one K stage of 8
// complex values (16 real) is one MMA step and three MMAs per accumulator.
// FP16's range is kept by scaling: row r of accumulator q's A is multiplied by
// 2^(F16_HEAD - fx(q, r)) before the split (fx(q, r) >= log2 of the row's
// largest component) and B, which must be bounded by 1 in magnitude (an
// overlap matrix), by 2^F16_HEAD; the result is scaled back by
// 2^(fx(q, r) - 2 F16_HEAD).  The headroom keeps typical entries (about
// 1/sqrt(n) of the largest) and their remainders in FP16's normal range, so
// the split matches the TF32 split's accuracy relative to each row's scale
// (entries far below it keep an absolute accuracy of 2^-24 of the scaled
// range, FP16's subnormal step); the largest scaled value stays below 2^8.
// Layout: K-major, no swizzle, 16-bit elements: core matrices of 8 rows x 8
// values (16 bytes per row), LBO = 128 between the two K-halves of a step,
// SBO = 256 between 8-row groups.
// ---------------------------------------------------------------------------
constexpr int CG_AB16 = CG_M * 2 * CG_KC * 2;                        // bytes of one A' part per stage
__host__ __device__ constexpr int cg_bb16() { return CG_N * 2 * CG_KC * 2; }   // bytes of one B' part
__host__ __device__ constexpr size_t c4_stage16() { return (size_t)C4 * 2 * CG_AB16 + 2 * (size_t)cg_bb16(); }
__host__ __device__ constexpr size_t c4_smem_bytes16() { return 2 * c4_stage16() + 64; }

// Byte offset of element (row, k), k < 16, of a 16-bit K-major operand stage.
__host__ __device__ __forceinline__ uint32_t kmajor_offset16(int row, int k) {
  return (uint32_t)(row >> 3) * 256u + (uint32_t)((k >> 3) & 1) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 7) * 2u;
}

// Four values (already scaled) as FP16 hi parts and FP16 remainders, 8 bytes each.
__device__ __forceinline__ void store_split16(unsigned char *hi_base, unsigned char *lo_base, uint32_t off, float a,
                                              float b, float c, float d) {
  const __half ha = __float2half_rn(a), hb = __float2half_rn(b), hc = __float2half_rn(c), hd = __float2half_rn(d);
  const __half la = __float2half_rn(a - __half2float(ha)), lb = __float2half_rn(b - __half2float(hb));
  const __half lc = __float2half_rn(c - __half2float(hc)), ld = __float2half_rn(d - __half2float(hd));
  uint2 h, l;
  h.x = (uint32_t)__half_as_ushort(ha) | ((uint32_t)__half_as_ushort(hb) << 16);
  h.y = (uint32_t)__half_as_ushort(hc) | ((uint32_t)__half_as_ushort(hd) << 16);
  l.x = (uint32_t)__half_as_ushort(la) | ((uint32_t)__half_as_ushort(lb) << 16);
  l.y = (uint32_t)__half_as_ushort(lc) | ((uint32_t)__half_as_ushort(ld) << 16);
  *reinterpret_cast<uint2 *>(hi_base + off) = h;
  *reinterpret_cast<uint2 *>(lo_base + off) = l;
}

// 2^e as a float (e within the normal range)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

constexpr int F16_HEAD = 8;   // power-of-two headroom of the FP16 split (see cgemm_tile_shared_b_f16)

template <class FA, class FS, class FB, class FX, class FE>
__device__ bool cgemm_tile_shared_b_f16(int m, int ncol, int k, int r0, int c0, unsigned amask, FA fa, FS fs,
                                        FB fb, FX fx, FE fe, unsigned char *smem) {
  constexpr int TN = CG_N, BB = cg_bb16();
  constexpr size_t STAGE = c4_stage16();
  constexpr int NCH = TN / 16;
  unsigned char *stage0 = smem;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 2 * STAGE);   // [2]
  uint32_t *slot = reinterpret_cast<uint32_t *>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const cc zero = czero<float>();
  struct Stg {
    cc a[2][2];   // A_h (r, l), (r, l+1)
    cc b[4];
  };
  // this thread's staging row and its scales 2^-fx(q, r)
  const int srr = tid % (CG_M / 2), slp = tid / (CG_M / 2);
  float sdown[C4];
#pragma unroll
  for (int q = 0; q < C4; ++q)
    sdown[q] = (r0 + srr < m && ((amask >> q) & 1u)) ? pow2f(F16_HEAD - fx(q, r0 + srr)) : 1.f;
  const float bup = pow2f(F16_HEAD);
  auto load = [&](int s, Stg &t) {
    const int l0 = s * CG_KC;
    const int r = r0 + srr, l = l0 + 2 * slp;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool on = (amask >> (2 * h)) & 3u;
      t.a[h][0] = (on && r < m && l < k) ? fa(h, r, l) : zero;
      t.a[h][1] = (on && r < m && l + 1 < k) ? fa(h, r, l + 1) : zero;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * CG_THREADS;
      const int jj = e % TN, lq = e / TN;
      const int j = c0 + jj, lb = l0 + 2 * lq;
      t.b[2 * u] = (lb < k && j < ncol) ? fb(lb, j) : zero;
      t.b[2 * u + 1] = (lb + 1 < k && j < ncol) ? fb(lb + 1, j) : zero;
    }
  };
  auto store = [&](unsigned char *base, int s, const Stg &t) {
    const int l = s * CG_KC + 2 * slp;
#pragma unroll
    for (int q = 0; q < C4; ++q) {
      if (!((amask >> q) & 1u)) continue;
      const int h = q >> 1;
      cc a0 = t.a[h][0], a1 = t.a[h][1];
      if (q & 1) {
        if (l < k) a0 = cmul(a0, fs(h, l));
        if (l + 1 < k) a1 = cmul(a1, fs(h, l + 1));
      }
      const float sc = sdown[q];
      a0 = mkc<float>(a0.re * sc, a0.im * sc);
      a1 = mkc<float>(a1.re * sc, a1.im * sc);
      unsigned char *Ahi = base + (size_t)q * 2 * CG_AB16, *Alo = Ahi + CG_AB16;
      store_split16(Ahi, Alo, kmajor_offset16(2 * srr, 4 * slp), a0.re, -a0.im, a1.re, -a1.im);
      store_split16(Ahi, Alo, kmajor_offset16(2 * srr + 1, 4 * slp), a0.im, a0.re, a1.im, a1.re);
    }
    unsigned char *Bhi = base + (size_t)C4 * 2 * CG_AB16, *Blo = Bhi + BB;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * CG_THREADS;
      const int jj = e % TN, lq = e / TN;
      store_split16(Bhi, Blo, kmajor_offset16(jj, 4 * lq), t.b[2 * u].re * bup, t.b[2 * u].im * bup,
                    t.b[2 * u + 1].re * bup, t.b[2 * u + 1].im * bup);
    }
  };
  const int lrow = 32 * (warp & 3) + lane;
  const int er = r0 + (lrow >> 1), eim = lrow & 1;
  Stg st0, st1;
  const int nstage = (k + CG_KC - 1) / CG_KC;
  load(0, st0);
  if (nstage > 1) load(1, st1);
  if (warp == 0) tmem_alloc(slot, C4 * TN);
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *slot;
  bool ok = true;
  auto step = [&](int s, Stg &t) {
    const int b = s & 1;
    unsigned char *base = stage0 + b * STAGE;
    if (s >= 2) ok = mbar_wait(&mbar[b], ((s - 2) >> 1) & 1) && ok;   // buffer b is free again
    store(base, s, t);
    if (s + 2 < nstage) load(s + 2, t);
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      constexpr uint32_t idesc = idesc_f16(CG_M, TN);
      const unsigned char *Bhi = base + (size_t)C4 * 2 * CG_AB16, *Blo = Bhi + BB;
      const uint64_t bh = smem_desc(Bhi, 128, 256);
      const uint64_t bl = smem_desc(Blo, 128, 256);
#pragma unroll
      for (int q = 0; q < C4; ++q) {
        if (!((amask >> q) & 1u)) continue;
        const unsigned char *Ahi = base + (size_t)q * 2 * CG_AB16, *Alo = Ahi + CG_AB16;
        const uint32_t d = tmem + (uint32_t)(q * TN);
        mma_f16(d, smem_desc(Ahi, 128, 256), bh, idesc, s > 0 ? 1u : 0u);
        mma_f16(d, smem_desc(Ahi, 128, 256), bl, idesc, 1u);
        mma_f16(d, smem_desc(Alo, 128, 256), bh, idesc, 1u);
      }
      mma_commit(&mbar[b]);
    }
  };
  for (int s = 0; s < nstage; s += 2) {
    step(s, st0);
    if (s + 1 < nstage) step(s + 1, st1);
  }
  ok = mbar_wait(&mbar[(nstage - 1) & 1], ((nstage - 1) >> 1) & 1) && ok;
  fence_after_sync();
  if (ok) {
    float sup[C4];
#pragma unroll
    for (int q = 0; q < C4; ++q) sup[q] = (er < m && ((amask >> q) & 1u)) ? pow2f(fx(q, er) - 2 * F16_HEAD) : 1.f;
#pragma unroll 1
    for (int qq = 0; qq < NCH; ++qq) {
      float vv[C4][8], other[C4][8];
#pragma unroll
      for (int q = 0; q < C4; ++q) {
        if ((amask >> q) & 1u) {
          tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(q * TN + (TN / 2) * (warp >> 2) + 8 * qq),
                   vv[q]);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) vv[q][i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) other[q][i] = __shfl_xor_sync(0xffffffffu, vv[q][i], 1);
      }
      const int jb = c0 + (TN / 2) * (warp >> 2) + 8 * qq + (eim ? 4 : 0);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        cc x[C4];
#pragma unroll
        for (int q = 0; q < C4; ++q) {
          const cc v = eim ? mkc<float>(other[q][i + 4], vv[q][i + 4]) : mkc<float>(vv[q][i], other[q][i]);
          x[q] = mkc<float>(v.re * sup[q], v.im * sup[q]);
        }
        if (er < m && jb + i < ncol) fe(er, jb + i, x);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, C4 * TN);
  return ok;
}

}  // namespace tc
}  // namespace pw
