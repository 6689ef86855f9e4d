// sc_find_seam_static: the seam search of sc_find_seam with every byte of its scratch in one
// fixed array that lives in the library's device image, so the call itself allocates nothing.
//
// Who needs it: programs that must not have a library allocate device memory behind their
// back. cudaMalloc/cudaFree can synchronise the whole device and take an unpredictable time, which
// a latency-critical frame loop cannot afford, and hosts that account for every device byte through
// their own allocator or a fixed memory budget forbid allocations they do not control. Such callers
// pass their own input and output buffers; the scratch (a padded copy of the energy map, the cost
// rows saved for the backtrack, two status words) comes from the array below.
#include <cstdio>
#include <mutex>

#include "../../include/sc.h"
#include "sc_internal.cuh"

namespace sc {

// 32 MiB: enough for a 3840 x 2160 energy map. Every GPU that loads the library holds this
// array until the process exits.
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Host code cannot use the name g_static_scratch as a device address: it is a host-side stand-in.
// The device address is looked up once per device with cudaGetSymbolAddress.
static std::mutex g_static_mu;
static void *g_static_addr[256] = {};

// If the energy-range check rejected the input, report it through the caller's outputs.
__global__ void k_static_reject(int H, int32_t *seam, int64_t *cost, const int *gate) {
  if (!(*gate & ERR_ENERGY_RANGE)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < H; i += gridDim.x * blockDim.x) seam[i] = -1;
  if (cost && blockIdx.x == 0 && threadIdx.x == 0) *cost = -1;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace sc

using namespace sc;

extern "C" int sc_find_seam_static(const uint16_t *energy, int H, int W, int32_t *seam_out, int64_t *cost_out,
                                   void *stream) {
  if (!energy || !seam_out) return SC_EINVAL;
  if (H < 1 || W < 1 || H > SC_MAX_ROWS || W > SC_MAX_COLS) return SC_EINVAL;
  const int pe = pitch_e_for(W);
  const int S = (H + KS - 1) / KS;
  const size_t off_flags = 0;
  const size_t off_E = 256;
  const size_t off_M = off_E + align256((size_t)H * pe * sizeof(uint16_t));
  const size_t need = off_M + align256((size_t)(S + 1) * pe * sizeof(uint32_t));
  if (need > STATIC_SCRATCH_BYTES) {
    fprintf(stderr, "sc_find_seam_static: a %d x %d energy map needs %zu bytes of scratch; the fixed array holds %zu\n",
            H, W, need, STATIC_SCRATCH_BYTES);
    return SC_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SC_ECUDA;
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
      void *ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess || !ptr) return SC_ECUDA;
      g_static_addr[dev] = ptr;
    }
    base = static_cast<unsigned char *>(g_static_addr[dev]);
  }
  cudaStream_t st = (cudaStream_t)stream;
  int *err = reinterpret_cast<int *>(base + off_flags);
  int *gate = err + 1;
  uint16_t *E = reinterpret_cast<uint16_t *>(base + off_E);
  uint32_t *Mrow = reinterpret_cast<uint32_t *>(base + off_M);
  // the array keeps the previous call's contents: the two status words must start at zero
  if (cudaMemsetAsync(err, 0, 2 * sizeof(int), st) != cudaSuccess) return SC_ECUDA;
  if (launch_copy_energy(energy, H, W, E + E_PADL, pe, err, gate, st) != cudaSuccess) return SC_ECUDA;
  DpArgs a;
  a.E = E + E_PADL;
  a.pitch_e = pe;
  a.H = H;
  a.W = W;
  a.Mrow = Mrow + E_PADL;
  a.seam = seam_out;
  a.seam_log = nullptr;
  a.cost = cost_out;
  a.err = err;
  a.gate = gate;
  if (launch_dp(a, st) != cudaSuccess) return SC_ECUDA;
  k_static_reject<<<(H + 255) / 256, 256, 0, st>>>(H, seam_out, cost_out, gate);
  return cudaGetLastError() == cudaSuccess ? SC_OK : SC_ECUDA;
}
