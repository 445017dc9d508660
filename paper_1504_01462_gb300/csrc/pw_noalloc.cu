// Star product of caller-supplied scattering matrices with no device
// allocation at all: the call's scratch is a fixed array in the library's own
// device image instead of memory from cudaMalloc.  See pw_compose_noalloc in
// include/pw.h.
#include <cuda_runtime.h>
#include <string.h>

#include <atomic>

#include "../../include/pw.h"
#include "pw_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB on every device that loads the library
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, per device; filled on the first call on each
// device.  (The host-side name g_scratch is only a stand-in for the symbol and
// must never be handed to a kernel.)  Atomic, so that host threads making
// their first calls on a device together do not race on the slot.
std::atomic<void *> g_scratch_addr[kMaxDevices];

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

constexpr int kMaxChunk = 256;   // status words are read back through a fixed host buffer

// Scratch bytes of one launch over nb points: the work matrices, the pivots and
// one status word per point, each region starting on a 256-byte boundary.
size_t chunk_bytes(size_t nb, size_t work_pp, size_t piv_pp) {
  return round256(nb * work_pp) + round256(nb * piv_pp) + round256(nb * sizeof(int));
}

// The most points one launch can take (0 when not even one point fits).
int max_chunk(size_t work_pp, size_t piv_pp) {
  int nb = (int)(kScratchBytes / (work_pp + piv_pp + sizeof(int)));
  if (nb > kMaxChunk) nb = kMaxChunk;
  while (nb > 0 && chunk_bytes((size_t)nb, work_pp, piv_pp) > kScratchBytes) --nb;
  return nb;
}

}  // namespace

extern "C" pw_status pw_compose_noalloc(int n, int npts, const pw_c128 *Sa_dev, const pw_c128 *Sb_dev,
                                        pw_c128 *Sab_dev, void *cuda_stream) {
  if (n < 1 || npts < 0) return PW_EINVAL;
  if (npts == 0) return PW_OK;
  if (!Sa_dev || !Sb_dev || !Sab_dev) return PW_EINVAL;
  const size_t nn = (size_t)n * n;
  const size_t work_pp = 4 * nn * sizeof(zc), piv_pp = (size_t)n * sizeof(int);
  // points per launch that fit the scratch with the layout below (n <= 362)
  const int chunk = max_chunk(work_pp, piv_pp);
  if (chunk < 1) return PW_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PW_ECUDA;
  void *addr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!addr) {
    if (cudaGetSymbolAddress(&addr, g_scratch) != cudaSuccess || !addr) return PW_ECUDA;
    g_scratch_addr[dev].store(addr, std::memory_order_release);
  }
  unsigned char *base = static_cast<unsigned char *>(addr);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int status_h[kMaxChunk];
  for (int b0 = 0; b0 < npts; b0 += chunk) {
    const int nb = npts - b0 < chunk ? npts - b0 : chunk;
    zc *work = reinterpret_cast<zc *>(base);
    int *piv = reinterpret_cast<int *>(base + round256(nb * work_pp));
    int *status = reinterpret_cast<int *>(base + round256(nb * work_pp) + round256(nb * piv_pp));
    if (cudaMemsetAsync(status, 0, nb * sizeof(int), st) != cudaSuccess) return PW_ECUDA;
    if (pw::launch_compose(reinterpret_cast<const zc *>(Sa_dev) + (size_t)b0 * 4 * nn,
                           reinterpret_cast<const zc *>(Sb_dev) + (size_t)b0 * 4 * nn,
                           reinterpret_cast<zc *>(Sab_dev) + (size_t)b0 * 4 * nn, work, piv,
                           status, n, nb, st) != cudaSuccess)
      return PW_ECUDA;
    if (cudaMemcpyAsync(status_h, status, nb * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return PW_ECUDA;
    for (int i = 0; i < nb; ++i)
      if (status_h[i]) return PW_ESINGULAR;
  }
  return PW_OK;
}
