// sc_find_seam_static: the seam search of sc_find_seam with every byte of its scratch in one
// fixed array that lives in the library's device image, so the call itself allocates nothing.
//
// Who needs it: programs that must not have a library allocate device memory behind their
// back. cudaMalloc/cudaFree can synchronise the whole device and take an unpredictable time, which
// a latency-critical frame loop cannot afford, and hosts that account for every device byte through
// their own allocator or a fixed memory budget forbid allocations they do not control. Such callers
// pass their own input and output buffers; the scratch (a padded copy of the energy map, the cost
// rows saved for the backtrack, the wide-cost search's directions and ancestors, three status
// words) comes from the array below.
#include <cstdio>
#include <mutex>

#include "../../include/sc.h"
#include "sc_host.h"
#include "sc_internal.cuh"

namespace sc {

// 32 MiB: enough for a 3840 x 2160 energy map. Every GPU that loads the library holds this
// array until the process exits.
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Status words at the start of the array:
//   [0] the errors of the call in flight (cleared by each call),
//   [1] the call's energy-range gate (cleared by each call),
//   [2] errors not yet reported: every call's errors are added here, and sc_check reads and
//       clears it.
constexpr int ST_CALL_ERR = 0, ST_GATE = 1, ST_PENDING = 2;

// Host code cannot use the name g_static_scratch as a device address: it is a host-side stand-in.
// The device address is looked up once per device with cudaGetSymbolAddress.
static std::mutex g_static_mu;
static void *g_static_addr[256] = {};

static int static_base(unsigned char **out, bool lookup) {
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SC_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 256) return fail(SC_ECUDA, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev] && lookup) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(SC_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    g_static_addr[dev] = ptr;
  }
  *out = static_cast<unsigned char *>(g_static_addr[dev]);
  return SC_OK;
}

// The last step of every static call: the call's error bits join the pending word, and a call
// that recorded any reports it through its outputs too (every seam entry and the cost set to -1).
__global__ void k_static_finish(int H, int32_t *seam, int64_t *cost, int *words) {
  const int e = words[ST_CALL_ERR];
  if (e == 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicOr(&words[ST_PENDING], e);
    if (cost) *cost = -1;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < H; i += gridDim.x * blockDim.x) seam[i] = -1;
}

static int launch_finish(int H, int32_t *seam, int64_t *cost, int *words, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((H + 255) / 256);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_static_finish, H, seam, cost, words);
  if (e != cudaSuccess) return fail(SC_ECUDA, "static search completion launch failed: %s", cudaGetErrorString(e));
  return SC_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int static_pending_errors(int *bits) {
  *bits = 0;
  unsigned char *base = nullptr;
  int rc = static_base(&base, false);
  if (rc || !base) return rc;   // no static call on this device yet: nothing pending
  int *pending = reinterpret_cast<int *>(base) + ST_PENDING;
  cudaError_t e = cudaMemcpy(bits, pending, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && *bits) e = cudaMemset(pending, 0, sizeof(int));
  if (e != cudaSuccess) return fail(SC_ECUDA, "reading the static search's status failed: %s", cudaGetErrorString(e));
  return SC_OK;
}

}  // namespace sc

using namespace sc;

#define SC_STATIC_CUDA(call)                                                                         \
  do {                                                                                               \
    const cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(SC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

extern "C" int sc_find_seam_static(const uint16_t *energy, int H, int W, int32_t *seam_out, int64_t *cost_out,
                                   void *stream) {
  if (!energy || !seam_out) return fail(SC_EINVAL, "null pointer");
  if (H < 1 || W < 1 || H > SC_MAX_ROWS || W > SC_MAX_COLS) return fail(SC_EINVAL, "bad shape %d x %d", H, W);
  const int pe = pitch_e_for(W);
  const int S = (H + KS - 1) / KS;
  const size_t off_E = 256;
  const size_t off_M = off_E + align256((size_t)H * pe * sizeof(uint16_t));
  const size_t off_D = off_M + align256((size_t)(S + 1) * pe * sizeof(uint32_t));
  const size_t off_A = off_D + align256(wide_dirs_words(H, W) * sizeof(uint32_t));
  const size_t need = off_A + align256(wide_anc_elems(H, W) * sizeof(uint16_t));
  if (need > STATIC_SCRATCH_BYTES)
    return fail(SC_EINVAL, "a %d x %d energy map needs %zu bytes of scratch; the static array holds %zu", H, W, need,
                STATIC_SCRATCH_BYTES);
  unsigned char *base = nullptr;
  int rc = static_base(&base, true);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int *words = reinterpret_cast<int *>(base);
  uint16_t *E = reinterpret_cast<uint16_t *>(base + off_E);
  // the array keeps the previous call's contents: this call's error word and gate start at zero
  SC_STATIC_CUDA(cudaMemsetAsync(words, 0, 2 * sizeof(int), st));
  SC_STATIC_CUDA(launch_copy_energy(energy, H, W, E + E_PADL, pe, words + ST_GATE, st));
  DpArgs a;
  a.E = E + E_PADL;
  a.pitch_e = pe;
  a.H = H;
  a.W = W;
  a.Mrow = reinterpret_cast<uint32_t *>(base + off_M) + E_PADL;
  a.seam = seam_out;
  a.seam_log = nullptr;
  a.cost = cost_out;
  a.err = words + ST_CALL_ERR;
  a.gate = words + ST_GATE;
  SC_STATIC_CUDA(launch_dp(a, st));
  SC_STATIC_CUDA(launch_dp_wide(a, reinterpret_cast<uint32_t *>(base + off_D), reinterpret_cast<uint16_t *>(base + off_A),
                                st));
  return launch_finish(H, seam_out, cost_out, words, st);
}

extern "C" int sc_find_seam_static_selftest(int limit_us, int H, int32_t *seam_out, int64_t *cost_out, void *stream) {
  if (limit_us < 1 || limit_us > 1000000) return fail(SC_EINVAL, "limit must be 1 us .. 1 s");
  if (!seam_out || H < 1 || H > SC_MAX_ROWS) return fail(SC_EINVAL, "null seam or H out of range");
  unsigned char *base = nullptr;
  int rc = static_base(&base, true);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int *words = reinterpret_cast<int *>(base);
  SC_STATIC_CUDA(cudaMemsetAsync(words, 0, 2 * sizeof(int), st));
  SC_STATIC_CUDA(launch_wait_selftest((uint64_t)limit_us * 1000u, words + ST_CALL_ERR, st));
  return launch_finish(H, seam_out, cost_out, words, st);
}
