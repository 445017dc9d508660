// Self-test of the tensor-core path (pw_selftest_tensor_core): one 128 x 64
// TF32 tile product with K = 32 on tcgen05, against an FP64 product on the
// host, for single TF32 and for the three-product split (A_hi B_hi + A_hi B_lo
// + A_lo B_hi) that recovers FP32 accuracy.
#include <math.h>
#include <stdlib.h>

#include <vector>

#include "../../include/pw.h"
#include "pw_internal.h"
#include "pw_tc.cuh"

namespace pw {

namespace {

constexpr int TM = 128, TN = 64, TK = 32;

// One CTA of 128 threads.  split: 0 = one TF32 product, 1 = three-product split.
__global__ void __launch_bounds__(128) k_tc_selftest(const float *A, const float *B, float *C, int split,
                                                     int *err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char *Ahi = smraw;                     // TM x TK
  unsigned char *Alo = Ahi + TM * TK * 4;
  unsigned char *Bhi = Alo + TM * TK * 4;         // TN x TK (B^T, K-major)
  unsigned char *Blo = Bhi + TN * TK * 4;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(Blo + TN * TK * 4);
  uint32_t *slot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // operands: A row-major TM x TK, B row-major TK x TN
  for (int e = tid; e < TM * TK; e += 128) {
    const int r = e / TK, k = e % TK;
    const float a = A[e], hi = tc::to_tf32(a);
    *reinterpret_cast<float *>(Ahi + tc::kmajor_offset(r, k, TM)) = hi;
    *reinterpret_cast<float *>(Alo + tc::kmajor_offset(r, k, TM)) = a - hi;
  }
  for (int e = tid; e < TK * TN; e += 128) {
    const int k = e / TN, c = e % TN;
    const float b = B[e], hi = tc::to_tf32(b);
    *reinterpret_cast<float *>(Bhi + tc::kmajor_offset(c, k, TN)) = hi;
    *reinterpret_cast<float *>(Blo + tc::kmajor_offset(c, k, TN)) = b - hi;
  }
  if (warp == 0) tc::tmem_alloc(slot, 64);
  if (tid == 0) tc::mbar_init(mbar, 1);
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_tf32(TM, TN);
    uint32_t acc = 0;
    for (int s = 0; s < TK / 8; ++s) {
      const uint64_t ah = tc::smem_desc(Ahi + s * TM * 32, 128, 256);
      const uint64_t bh = tc::smem_desc(Bhi + s * TN * 32, 128, 256);
      tc::mma_tf32(tmem, ah, bh, idesc, acc);
      acc = 1;
      if (split) {
        const uint64_t al = tc::smem_desc(Alo + s * TM * 32, 128, 256);
        const uint64_t bl = tc::smem_desc(Blo + s * TN * 32, 128, 256);
        tc::mma_tf32(tmem, ah, bl, idesc, 1);
        tc::mma_tf32(tmem, al, bh, idesc, 1);
      }
    }
    tc::mma_commit(mbar);
  }
  const bool done = tc::mbar_wait(mbar, 0);
  tc::fence_after_sync();
  if (!done) {
    if (lane == 0) atomicOr(err, 1);
  } else {
    // warp w reads TMEM lanes 32w .. 32w+31 (rows of D)
    const int row = warp * 32 + lane;
    for (int c0 = 0; c0 < TN; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) C[row * TN + c0 + i] = v[i];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// One CTA of 128 threads: the same 128 x 64 x 32 product in the FP16 split
// (hi/lo FP16 parts, three kind::f16 MMAs per K step of 16) with A and B
// scaled by the split's headroom 2^F16_HEAD, the layout and descriptors of
// cgemm_tile_shared_b_f16.
__global__ void __launch_bounds__(128) k_tc_selftest16(const float *A, const float *B, float *C, int *err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  constexpr int SA = TM * 32, SB = TN * 32;       // bytes of one 16-value K step
  unsigned char *Ahi = smraw;                     // two K steps each
  unsigned char *Alo = Ahi + 2 * SA;
  unsigned char *Bhi = Alo + 2 * SA;
  unsigned char *Blo = Bhi + 2 * SB;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(Blo + 2 * SB);
  uint32_t *slot = reinterpret_cast<uint32_t *>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float up = tc::pow2f(tc::F16_HEAD);
  // four consecutive K values per task, 8 bytes per hi/lo store
  for (int e = tid; e < TM * (TK / 4); e += 128) {
    const int r = e / (TK / 4), k4 = 4 * (e % (TK / 4));
    const float *a = A + r * TK + k4;
    const uint32_t off = (uint32_t)(k4 >> 4) * SA + tc::kmajor_offset16(r, k4 & 15);
    tc::store_split16(Ahi, Alo, off, a[0] * up, a[1] * up, a[2] * up, a[3] * up);
  }
  for (int e = tid; e < TN * (TK / 4); e += 128) {
    const int c = e / (TK / 4), k4 = 4 * (e % (TK / 4));
    const uint32_t off = (uint32_t)(k4 >> 4) * SB + tc::kmajor_offset16(c, k4 & 15);
    tc::store_split16(Bhi, Blo, off, B[(k4 + 0) * TN + c] * up, B[(k4 + 1) * TN + c] * up,
                      B[(k4 + 2) * TN + c] * up, B[(k4 + 3) * TN + c] * up);
  }
  if (warp == 0) tc::tmem_alloc(slot, 64);
  if (tid == 0) tc::mbar_init(mbar, 1);
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_f16(TM, TN);
    for (int s = 0; s < TK / 16; ++s) {
      const uint64_t ah = tc::smem_desc(Ahi + s * SA, 128, 256), al = tc::smem_desc(Alo + s * SA, 128, 256);
      const uint64_t bh = tc::smem_desc(Bhi + s * SB, 128, 256), bl = tc::smem_desc(Blo + s * SB, 128, 256);
      tc::mma_f16(tmem, ah, bh, idesc, s > 0 ? 1u : 0u);
      tc::mma_f16(tmem, ah, bl, idesc, 1u);
      tc::mma_f16(tmem, al, bh, idesc, 1u);
    }
    tc::mma_commit(mbar);
  }
  const bool done = tc::mbar_wait(mbar, 0);
  tc::fence_after_sync();
  if (!done) {
    if (lane == 0) atomicOr(err, 1);
  } else {
    const int row = warp * 32 + lane;
    const float down = tc::pow2f(-2 * tc::F16_HEAD);
    for (int c0 = 0; c0 < TN; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) C[row * TN + c0 + i] = v[i] * down;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// The bounded completion wait of the tensor-core kernels on an mbarrier that
// nothing completes (no MMA is issued and, unless `signal`, nobody arrives):
// the wait gives up after `polls` polls, the CTA frees the tensor memory it
// holds and reports through out[0] (1: the wait ran out, 0: it completed).
// With signal != 0 thread 0 arrives first, so the same wait completes.
__global__ void __launch_bounds__(128) k_wait_selftest(uint32_t polls, int signal, int *out) {
  __shared__ uint64_t mbar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc::tmem_alloc(&slot, 32);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = slot;
  if (signal && tid == 0) tc::mbar_arrive(&mbar);
  const bool done = tc::mbar_wait(&mbar, 0, polls);
  const bool all = __syncthreads_and(done) != 0;
  if (tid == 0) out[0] = all ? 0 : 1;
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

}  // namespace

}  // namespace pw

extern "C" pw_status pw_selftest_bounded_wait(int polls, int signal) {
  using namespace pw;
  if (polls < 1) return PW_EINVAL;
  int *d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return PW_ENOMEM;
  int h = -1;
  cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 128>>>((uint32_t)polls, signal, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return PW_ECUDA;
  return h == 0 ? PW_OK : h == 1 ? PW_ETIMEOUT : PW_ECUDA;
}

extern "C" pw_status pw_selftest_f16_split(double *rel_err) {
  if (!rel_err) return PW_EINVAL;
  using namespace pw;
  std::vector<float> A(TM * TK), B(TK * TN), C(TM * TN);
  unsigned s = 777u;
  auto rnd = [&]() {
    s = s * 1664525u + 1013904223u;
    return (float)((s >> 8) & 0xFFFF) / 65536.0f - 0.5f;
  };
  for (auto &x : A) x = rnd();
  for (auto &x : B) x = rnd();
  float *dA = nullptr, *dB = nullptr, *dC = nullptr;
  int *derr = nullptr;
  const size_t smem = (size_t)(4 * TM * 32 + 4 * TN * 32) + 64;
  pw_status st = PW_OK;
  if (cudaMalloc(&dA, A.size() * 4) || cudaMalloc(&dB, B.size() * 4) || cudaMalloc(&dC, C.size() * 4) ||
      cudaMalloc(&derr, sizeof(int))) {
    cudaGetLastError();
    st = PW_ENOMEM;
  } else {
    int herr = 0;
    if (cudaMemcpy(dA, A.data(), A.size() * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(dB, B.data(), B.size() * 4, cudaMemcpyHostToDevice) || cudaMemset(derr, 0, sizeof(int)) ||
        cudaMemset(dC, 0, C.size() * 4) ||
        cudaFuncSetAttribute(k_tc_selftest16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) {
      st = PW_ECUDA;
    } else {
      k_tc_selftest16<<<1, 128, smem>>>(dA, dB, dC, derr);
      if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
          cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(C.data(), dC, C.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        st = PW_ECUDA;
      else if (herr)
        st = PW_ETIMEOUT;
    }
    if (st == PW_OK) {
      double num = 0.0, den = 0.0;
      for (int i = 0; i < TM; ++i)
        for (int j = 0; j < TN; ++j) {
          double ref = 0.0;
          for (int k = 0; k < TK; ++k) ref += (double)A[i * TK + k] * (double)B[k * TN + j];
          num = fmax(num, fabs(ref - (double)C[i * TN + j]));
          den = fmax(den, fabs(ref));
        }
      *rel_err = num / fmax(den, 1e-300);
    }
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  cudaFree(derr);
  return st;
}

extern "C" pw_status pw_selftest_tensor_core(double *rel_err_tf32, double *rel_err_split) {
  if (!rel_err_tf32 || !rel_err_split) return PW_EINVAL;
  using namespace pw;
  std::vector<float> A(TM * TK), B(TK * TN), C(TM * TN);
  unsigned s = 12345u;
  auto rnd = [&]() {
    s = s * 1664525u + 1013904223u;
    return (float)((s >> 8) & 0xFFFF) / 65536.0f - 0.5f;
  };
  for (auto &x : A) x = rnd();
  for (auto &x : B) x = rnd();
  float *dA = nullptr, *dB = nullptr, *dC = nullptr;
  int *derr = nullptr;
  const size_t smem = (size_t)(2 * TM * TK + 2 * TN * TK) * 4 + 64;
  pw_status st = PW_OK;
  if (cudaMalloc(&dA, A.size() * 4) || cudaMalloc(&dB, B.size() * 4) || cudaMalloc(&dC, C.size() * 4) ||
      cudaMalloc(&derr, sizeof(int))) {
    st = PW_ENOMEM;
  } else {
    cudaMemcpy(dA, A.data(), A.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, B.data(), B.size() * 4, cudaMemcpyHostToDevice);
    cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    double *outs[2] = {rel_err_tf32, rel_err_split};
    for (int split = 0; split < 2 && st == PW_OK; ++split) {
      cudaMemset(derr, 0, sizeof(int));
      cudaMemset(dC, 0, C.size() * 4);
      k_tc_selftest<<<1, 128, smem>>>(dA, dB, dC, split, derr);
      int herr = 0;
      if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
          cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(C.data(), dC, C.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        st = PW_ECUDA;
        break;
      }
      if (herr) {
        st = PW_ETIMEOUT;
        break;
      }
      double num = 0.0, den = 0.0;
      for (int i = 0; i < TM; ++i)
        for (int j = 0; j < TN; ++j) {
          double ref = 0.0;
          for (int k = 0; k < TK; ++k) ref += (double)A[i * TK + k] * (double)B[k * TN + j];
          num = fmax(num, fabs(ref - (double)C[i * TN + j]));
          den = fmax(den, fabs(ref));
        }
      *outs[split] = num / fmax(den, 1e-300);
    }
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  cudaFree(derr);
  return st;
}
