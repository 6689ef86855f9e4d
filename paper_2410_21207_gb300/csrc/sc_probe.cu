// Copy-bandwidth probe (instrumentation; the paper has no counterpart): the denominator of the
// L2 roofline fractions. One launch copies a buffer pair `reps` times, so that the measured time is
// the copies' own and not the gaps between many short kernels; with both buffers inside L2 the
// rate is the L2 copy bandwidth.
#include "../../include/sc.h"
#include "sc_host.h"
#include "sc_internal.cuh"

namespace sc {

// src and dst are deliberately not __restrict__: every pass reloads src. Each pass xors its index
// into the data, so no pass can be folded into another.
__global__ void k_copy_probe(const uint4 *src, uint4 *dst, size_t n16, int reps) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    const uint32_t x = (uint32_t)r;
#pragma unroll 4
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
      uint4 v = src[i];
      v.x ^= x;
      dst[i] = v;
    }
  }
}

}  // namespace sc

using namespace sc;

#define SC_PROBE_CUDA(call)                                                                        \
  do {                                                                                             \
    const cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                       \
      rc = fail(SC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));                         \
      goto done;                                                                                   \
    }                                                                                              \
  } while (0)

extern "C" int sc_probe_copy_bandwidth(size_t bytes, int reps, double *gbs_out) {
  if (!gbs_out || bytes < 4096 || bytes % 16 != 0 || reps < 1 || reps > 10000)
    return fail(SC_EINVAL, "need bytes >= 4096, a multiple of 16, and 1 <= reps <= 10000");
  *gbs_out = 0.0;
  int rc = SC_OK;
  uint4 *a = nullptr, *b = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int dev = 0, sms = 1;
  float ms = 0.f;
  const size_t n16 = bytes / 16;
  SC_PROBE_CUDA(cudaGetDevice(&dev));
  SC_PROBE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SC_PROBE_CUDA(cudaMalloc(&a, bytes));
  SC_PROBE_CUDA(cudaMalloc(&b, bytes));
  SC_PROBE_CUDA(cudaMemset(a, 1, bytes));
  SC_PROBE_CUDA(cudaEventCreate(&e0));
  SC_PROBE_CUDA(cudaEventCreate(&e1));
  k_copy_probe<<<sms * 8, 256>>>(a, b, n16, 2);   // warm-up: buffers resident where they fit
  SC_PROBE_CUDA(cudaGetLastError());
  SC_PROBE_CUDA(cudaEventRecord(e0));
  k_copy_probe<<<sms * 8, 256>>>(a, b, n16, reps);
  SC_PROBE_CUDA(cudaGetLastError());
  SC_PROBE_CUDA(cudaEventRecord(e1));
  SC_PROBE_CUDA(cudaEventSynchronize(e1));
  SC_PROBE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  *gbs_out = 2.0 * (double)bytes * reps / (ms / 1e3) / 1e9;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (a) cudaFree(a);
  if (b) cudaFree(b);
  return rc;
}
