// Measured arithmetic peaks of the GPU the library runs on (pw_measure_peaks):
// the FP64 FMA rate of the SIMT pipe (DFMA), the FP64 tensor rate of the
// warp-level FP64 MMA (mma.sync m8n8k4, the only FP64 tensor instruction that
// sm_103a offers) and the FP32 FMA rate.  GB300 cut FP64 sharply against
// earlier data-centre parts, so the FP64 form's roofline is taken from these
// numbers rather than from a datasheet.  Each kernel runs enough independent
// dependency chains per thread to hide latency, on every SM, and is timed with
// CUDA events after a warm-up launch.
#include <cuda_runtime.h>

#include "../../include/pw.h"
#include "pw_internal.h"

namespace pw {
namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;   // independent accumulators per thread

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) k_peak_fma(T *out, T x, T y, int iters) {
  T acc[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) acc[c] = x + (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) acc[c] = fma(acc[c], y, x);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += acc[c];
  if (s == (T)1.2345) out[blockIdx.x * PK_THREADS + threadIdx.x] = s;   // keeps the chains live
}

// One warp-level FP64 MMA D(8x8) = A(8x4) B(4x8) + C: 256 multiply-adds.
__device__ __forceinline__ void dmma_8x8x4(double &d0, double &d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_dmma(double *out, double x, double y, int iters) {
  double d[PK_CHAINS][2];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) d[c][0] = d[c][1] = 0.0;
  const double a = x + threadIdx.x * 1e-3, b = y - threadIdx.x * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) dmma_8x8x4(d[c][0], d[c][1], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += d[c][0] + d[c][1];
  if (s == 1.2345) out[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

// Milliseconds of the faster of two timed launches (after one warm-up).
template <typename L>
cudaError_t time_launch(L launch, float *ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
  launch();
  float best = 1e30f;
  for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e == cudaSuccess && t < best) best = t;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = best;
  return e;
}

}  // namespace
}  // namespace pw

extern "C" pw_status pw_measure_peaks(double *tflops) {
  using namespace pw;
  if (!tflops) return PW_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return PW_ECUDA;
  const int blocks = 8 * sms;   // eight 256-thread CTAs per SM
  void *buf = nullptr;
  if (cudaMalloc(&buf, (size_t)blocks * PK_THREADS * sizeof(double)) != cudaSuccess) return PW_ENOMEM;
  double *d64 = static_cast<double *>(buf);
  float *d32 = static_cast<float *>(buf);
  const double threads = (double)blocks * PK_THREADS;
  float ms = 0.f;
  cudaError_t e;
  // DFMA: 2 flop per FMA
  const int it64 = 4096;
  e = time_launch([&] { k_peak_fma<double><<<blocks, PK_THREADS>>>(d64, 1.0000001, 0.9999999, it64); }, &ms);
  if (e == cudaSuccess) tflops[0] = 2.0 * PK_CHAINS * it64 * threads / (ms * 1e-3) / 1e12;
  // DMMA m8n8k4: 2 * 256 flop per warp instruction
  const int itm = 2048;
  if (e == cudaSuccess)
    e = time_launch([&] { k_peak_dmma<<<blocks, PK_THREADS>>>(d64, 1.0000001, 0.9999999, itm); }, &ms);
  if (e == cudaSuccess) tflops[1] = 2.0 * 256.0 * PK_CHAINS * itm * (threads / 32.0) / (ms * 1e-3) / 1e12;
  // FP32 FMA
  const int it32 = 65536;
  if (e == cudaSuccess)
    e = time_launch([&] { k_peak_fma<float><<<blocks, PK_THREADS>>>(d32, 1.0000001f, 0.9999999f, it32); }, &ms);
  if (e == cudaSuccess) tflops[2] = 2.0 * PK_CHAINS * it32 * threads / (ms * 1e-3) / 1e12;
  cudaFree(buf);
  return e == cudaSuccess ? PW_OK : PW_ECUDA;
}
