// Conductance sums of Sec. II B (Eq. T1_d / T2_d) on the device, in FP64:
// the weighted sum of T over a set of (E, k_par) points and the transmission
// per electrode conduction channel, T averaged over the k_par mesh points at
// which the left electrode has an open channel.  One CTA reduces in a fixed
// order (thread-strided partial sums, then a shared-memory tree), so the
// result does not depend on scheduling.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/pw.h"
#include "pw_internal.h"

namespace pw {
namespace {

constexpr int RT = 256;

__global__ void __launch_bounds__(RT) k_reduce_T(int npts, const double *T, const int *nopen, const double *w,
                                                 double *out) {
  __shared__ double s_sum[RT], s_bar[RT], s_cnt[RT];
  double sum = 0.0, bar = 0.0, cnt = 0.0;
  for (int i = threadIdx.x; i < npts; i += RT) {
    const double t = T[i];
    if (isnan(t)) continue;                 // a point at an electrode threshold
    sum += (w ? w[i] : 1.0) * t;
    if (!nopen || nopen[2 * i] > 0) {
      bar += t;
      cnt += 1.0;
    }
  }
  s_sum[threadIdx.x] = sum;
  s_bar[threadIdx.x] = bar;
  s_cnt[threadIdx.x] = cnt;
  __syncthreads();
  for (int h = RT / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s_sum[threadIdx.x] += s_sum[threadIdx.x + h];
      s_bar[threadIdx.x] += s_bar[threadIdx.x + h];
      s_cnt[threadIdx.x] += s_cnt[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s_sum[0];
    out[1] = s_cnt[0] > 0.0 ? s_bar[0] / s_cnt[0] : 0.0;
    out[2] = s_cnt[0];
  }
}

}  // namespace
}  // namespace pw

extern "C" pw_status pw_reduce_transmission(int npts, const double *T_dev, const int *nopen_dev,
                                            const double *weight_dev, double *out_dev, void *cuda_stream) {
  if (npts < 0 || !out_dev || (npts > 0 && !T_dev)) return PW_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  pw::k_reduce_T<<<1, pw::RT, 0, s>>>(npts, T_dev, nopen_dev, weight_dev, out_dev);
  return cudaGetLastError() == cudaSuccess ? PW_OK : PW_ECUDA;
}
