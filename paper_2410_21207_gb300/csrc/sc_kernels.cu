// Whole-image kernels of libsc_gb300: packing, transposition, the e1 energy, and the per-seam
// local energy refresh and row compaction (arXiv 2410.21207, sections "Energy Mapping" and
// "Removal of Seams"; horizontal seams by transposition, section "Design Techniques").
#include "sc_internal.cuh"
#include "sc_ptx.cuh"
#include "sc_rowops.cuh"

namespace sc {

// ---- pack: HWC uint8 (C in {1,3,4}) -> one uint32 word per pixel, channel c in byte c ----
__global__ void k_pack(const uint8_t *__restrict__ src, int H, int W, int C, uint32_t *__restrict__ img,
                       int pitch) {
  const int64_t n = (int64_t)H * W;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(p / W), j = (int)(p % W);
    img[(int64_t)i * pitch + j] = pack_pixel(src + p * C, C);
  }
}

// ---- unpack: words -> HWC uint8 ----
__global__ void k_unpack(const uint32_t *__restrict__ img, int pitch, int H, int W, int C, uint8_t *__restrict__ dst) {
  const int64_t n = (int64_t)H * W;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(p / W), j = (int)(p % W);
    unpack_pixel(img[(int64_t)i * pitch + j], dst + p * C, C);
  }
}

// ---- transpose of a word image through 32x32 shared-memory tiles (coalesced both ways) ----
__global__ void k_transpose(const uint32_t *__restrict__ src, int ps, int H, int W, uint32_t *__restrict__ dst,
                            int pd) {
  __shared__ uint32_t tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int i = by + r, j = bx + threadIdx.x;
    if (i < H && j < W) tile[r][threadIdx.x] = src[(int64_t)i * ps + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int j = bx + r, i = by + threadIdx.x;   // dst row j, column i
    if (i < H && j < W) dst[(int64_t)j * pd + i] = tile[threadIdx.x][r];
  }
}

// ---- e1 energy: sum over the packed channels of |right - left| + |down - up|, clamped ----
__global__ void k_energy(const uint32_t *__restrict__ img, int pitch, int H, int W, uint16_t *__restrict__ E,
                         int pe) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= W || i >= H) return;
  E[(int64_t)i * pe + j] = (uint16_t)energy_at(img, pitch, H, W, i, j);
}

// ---- forward energy: the CU, DL, DR planes (plane p at E + p * pstride) ----
__global__ void k_forward(const uint32_t *__restrict__ img, int pitch, int H, int W, uint16_t *__restrict__ E, int pe,
                          int64_t pstride) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= W || i >= H) return;
  uint32_t cu, dl, dr;
  forward_at([&](int r, int c) { return img[(int64_t)r * pitch + c]; }, W, i, j, cu, dl, dr);
  E[(int64_t)i * pe + j] = (uint16_t)cu;
  E[pstride + (int64_t)i * pe + j] = (uint16_t)dl;
  E[2 * pstride + (int64_t)i * pe + j] = (uint16_t)dr;
}

// ---- caller forward planes -> padded layout. DL in row 0 and column 0 and DR in row 0 and the
// last column are never used (no such predecessor) and are stored as 0. A cell whose
// CU + max(DL, DR) exceeds `limit` sets the map's gate: its seam sums may not fit the 24-bit cost
// field, and the wide-cost search takes the map (one atomic per warp). ----
__global__ void k_copy_planes(const uint16_t *__restrict__ cu, const uint16_t *__restrict__ dl,
                              const uint16_t *__restrict__ dr, int H, int W, uint16_t *__restrict__ E, int pe,
                              int64_t pstride, uint32_t limit, int *gate) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  bool over = false;
  if (j < W && i < H) {
    const int64_t q = (int64_t)i * W + j;
    const uint32_t u = cu[q];
    const uint32_t l = (i >= 1 && j >= 1) ? dl[q] : 0u;
    const uint32_t r = (i >= 1 && j + 1 < W) ? dr[q] : 0u;
    E[(int64_t)i * pe + j] = (uint16_t)u;
    E[pstride + (int64_t)i * pe + j] = (uint16_t)l;
    E[2 * pstride + (int64_t)i * pe + j] = (uint16_t)r;
    over = u + (l > r ? l : r) > limit;
  }
  if (__any_sync(0xffffffffu, over) && (threadIdx.x & 31) == 0) atomicOr(gate, ERR_ENERGY_RANGE);
}

// ---- caller energy -> padded layout; an energy above `limit` sets the map's gate (its seam sums
// may not fit the 24-bit cost field: the wide-cost search takes the map; one atomic per warp) ----
__global__ void k_copy_energy(const uint16_t *__restrict__ src, int H, int W, uint16_t *__restrict__ E, int pe,
                              uint32_t limit, int *gate) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  bool over = false;
  if (j < W && i < H) {
    const uint16_t v = src[(int64_t)i * W + j];
    E[(int64_t)i * pe + j] = v;
    over = v > limit;
  }
  if (__any_sync(0xffffffffu, over) && (threadIdx.x & 31) == 0) atomicOr(gate, ERR_ENERGY_RANGE);
}

__global__ void k_unpad_energy(const uint16_t *__restrict__ E, int pe, int H, int W, uint16_t *__restrict__ dst) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= W || i >= H) return;
  dst[(int64_t)i * W + j] = E[(int64_t)i * pe + j];
}

// ---- lazy image compaction: refresh through the pending-removal lists, then add the removal ----
// one warp per row: refreshed pair (lazy image), list update, energy compaction (refresh_row)
__global__ void k_refresh(const uint32_t *__restrict__ img, int pitch, uint16_t *__restrict__ E, int pe, int H, int W,
                          const int32_t *__restrict__ seam, const int16_t *__restrict__ lists_in,
                          int16_t *__restrict__ lists_out, int m, int *err) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  pdl_launch_dependents();
  pdl_wait_prerequisites();   // the seam of the search that precedes this launch
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < H; i += warps)
    if (!refresh_row(img, pitch, E, pe, H, W, seam, lists_in, lists_out, m, i, lane) && lane == 0)
      atomicOr(err, ERR_BAD_SEAM);
}

__global__ void k_refresh_fwd(const uint32_t *__restrict__ img, int pitch, uint16_t *__restrict__ E, int pe,
                              int64_t pstride, int H, int W, const int32_t *__restrict__ seam,
                              const int16_t *__restrict__ lists_in, int16_t *__restrict__ lists_out, int m, int *err) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  pdl_launch_dependents();
  pdl_wait_prerequisites();
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < H; i += warps)
    if (!refresh_row_fwd(img, pitch, E, pe, pstride, H, W, seam, lists_in, lists_out, m, i, lane) && lane == 0)
      atomicOr(err, ERR_BAD_SEAM);
}

__global__ void k_compact_lazy(uint32_t *__restrict__ img, int pitch, int H, int w, const int16_t *__restrict__ lists,
                               int m) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  pdl_launch_dependents();
  pdl_wait_prerequisites();
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < H; i += warps)
    compact_row_lazy(img + (int64_t)i * pitch, lists + (int64_t)i * RPEND, m, w, lane);
}

// ---- launchers ----
// launch as a programmatic dependent of the previous kernel on the stream (the kernels of the seam
// loop wait for their predecessor with griddepcontrol.wait before touching its results)
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), int blocks, int threads, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

static int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_pack(const uint8_t *src, int H, int W, int C, uint32_t *img, int pitch, cudaStream_t st) {
  k_pack<<<grid_for((int64_t)H * W, 256), 256, 0, st>>>(src, H, W, C, img, pitch);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const uint32_t *img, int pitch, int H, int W, int C, bool transposed, uint8_t *dst,
                          cudaStream_t st) {
  (void)transposed;  // the caller transposes first when needed
  k_unpack<<<grid_for((int64_t)H * W, 256), 256, 0, st>>>(img, pitch, H, W, C, dst);
  return cudaGetLastError();
}

cudaError_t launch_transpose(const uint32_t *src, int ps, int H, int W, uint32_t *dst, int pd, cudaStream_t st) {
  dim3 grid((W + 31) / 32, (H + 31) / 32), block(32, 8);
  k_transpose<<<grid, block, 0, st>>>(src, ps, H, W, dst, pd);
  return cudaGetLastError();
}

cudaError_t launch_energy(const uint32_t *img, int pitch, int H, int W, uint16_t *E, int pe, cudaStream_t st) {
  dim3 grid((W + 127) / 128, H);
  k_energy<<<grid, 128, 0, st>>>(img, pitch, H, W, E, pe);
  return cudaGetLastError();
}

cudaError_t launch_copy_energy(const uint16_t *src, int H, int W, uint16_t *E, int pe, int *gate, cudaStream_t st) {
  // the 24-bit search keeps costs below 2^24: every seam sum must fit
  const uint32_t limit = (uint32_t)((((uint64_t)1 << 24) - 1) / (uint64_t)H);
  dim3 grid((W + 127) / 128, H);
  k_copy_energy<<<grid, 128, 0, st>>>(src, H, W, E, pe, limit, gate);
  return cudaGetLastError();
}

cudaError_t launch_forward(const uint32_t *img, int pitch, int H, int W, uint16_t *E, int pe, int64_t pstride,
                           cudaStream_t st) {
  dim3 grid((W + 127) / 128, H);
  k_forward<<<grid, 128, 0, st>>>(img, pitch, H, W, E, pe, pstride);
  return cudaGetLastError();
}

cudaError_t launch_copy_planes(const uint16_t *cu, const uint16_t *dl, const uint16_t *dr, int H, int W, uint16_t *E,
                               int pe, int64_t pstride, int *gate, cudaStream_t st) {
  const uint32_t limit = (uint32_t)((((uint64_t)1 << 24) - 1) / (uint64_t)H);
  dim3 grid((W + 127) / 128, H);
  k_copy_planes<<<grid, 128, 0, st>>>(cu, dl, dr, H, W, E, pe, pstride, limit, gate);
  return cudaGetLastError();
}

cudaError_t launch_unpad_energy(const uint16_t *E, int pe, int H, int W, uint16_t *dst, cudaStream_t st) {
  dim3 grid((W + 127) / 128, H);
  k_unpad_energy<<<grid, 128, 0, st>>>(E, pe, H, W, dst);
  return cudaGetLastError();
}

}  // namespace sc

namespace sc {

cudaError_t launch_refresh(const uint32_t *img, int pitch, uint16_t *E, int pe, int H, int W, const int32_t *seam,
                           const int16_t *lists_in, int16_t *lists_out, int m, int *err, cudaStream_t st) {
  const int warps_per_block = 8;
  int blocks = (H + warps_per_block - 1) / warps_per_block;
  if (blocks > 152 * 8) blocks = 152 * 8;
  return launch_pdl(k_refresh, blocks, warps_per_block * 32, st, img, pitch, E, pe, H, W, seam, lists_in, lists_out, m,
                    err);
}

cudaError_t launch_refresh_fwd(const uint32_t *img, int pitch, uint16_t *E, int pe, int64_t pstride, int H, int W,
                               const int32_t *seam, const int16_t *lists_in, int16_t *lists_out, int m, int *err,
                               cudaStream_t st) {
  const int warps_per_block = 8;
  int blocks = (H + warps_per_block - 1) / warps_per_block;
  if (blocks > 152 * 8) blocks = 152 * 8;
  return launch_pdl(k_refresh_fwd, blocks, warps_per_block * 32, st, img, pitch, E, pe, pstride, H, W, seam, lists_in,
                    lists_out, m, err);
}

cudaError_t launch_compact_lazy(uint32_t *img, int pitch, int H, int w, const int16_t *lists, int m, cudaStream_t st) {
  const int warps_per_block = 8;
  int blocks = (H + warps_per_block - 1) / warps_per_block;
  if (blocks > 152 * 8) blocks = 152 * 8;
  return launch_pdl(k_compact_lazy, blocks, warps_per_block * 32, st, img, pitch, H, w, lists, m);
}

}  // namespace sc

namespace sc {

// ---- Algorithm 2 (greedy): start at the leftmost minimum of the bottom row, climb by the
// leftmost minimum of the (in-range) upper neighbours. One warp per map: the bottom-row argmin is a
// warp reduction; the climb is serial, so the warp stages the 65-column window it can reach in
// the next 32 rows into shared memory and lane 0 walks it. ----
constexpr int GREEDY_ROWS = 32;
constexpr int GREEDY_COLS = 2 * GREEDY_ROWS + 1;

__global__ void __launch_bounds__(32) k_greedy(const uint16_t *__restrict__ e, int H, int W,
                                               int32_t *__restrict__ seam, int64_t *__restrict__ cost) {
  __shared__ uint32_t win[GREEDY_ROWS][GREEDY_COLS + 1];
  const int lane = threadIdx.x;
  unsigned long long best = ~0ull;   // (energy << 32) | column, leftmost minimum
  const uint16_t *last = e + (int64_t)(H - 1) * W;
  for (int j = lane; j < W; j += 32) {
    const unsigned long long k = ((unsigned long long)last[j] << 32) | (unsigned)j;
    best = k < best ? k : best;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
    best = o < best ? o : best;
  }
  int j = (int)(best & 0xFFFFFFFFu);
  int64_t total = (int64_t)(best >> 32);
  if (lane == 0) seam[H - 1] = j;
  for (int top = H - 1; top > 0; top -= GREEDY_ROWS) {
    const int rows = top < GREEDY_ROWS ? top : GREEDY_ROWS;   // rows top-1 .. top-rows
    const int c0 = j - GREEDY_ROWS;
    // stage 8 rows at a time with all their loads in flight (3 columns per lane per row)
    for (int rb = 0; rb < rows; rb += 8) {
      uint32_t v[8][3];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int r = rb + q;
        const uint16_t *row = e + (int64_t)(top - 1 - (r < rows ? r : 0)) * W;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int c = lane + 32 * u, col = c0 + c;
          v[q][u] = (r < rows && c < GREEDY_COLS && col >= 0 && col < W) ? (uint32_t)row[col] : 0x10000u;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int c = lane + 32 * u;
          if (rb + q < rows && c < GREEDY_COLS) win[rb + q][c] = v[q][u];   // 0x10000: above any energy
        }
      }
    }
    __syncwarp();
    if (lane == 0) {
      int x = j - c0;
      for (int r = 0; r < rows; ++r) {
        int b = x - 1;
        if (win[r][x] < win[r][b]) b = x;
        if (win[r][x + 1] < win[r][b]) b = x + 1;
        x = b;
        total += win[r][x];
        seam[top - 1 - r] = c0 + x;
      }
      j = c0 + x;
    }
    j = __shfl_sync(0xffffffffu, j, 0);
    __syncwarp();
  }
  if (lane == 0 && cost) *cost = total;
}

cudaError_t launch_greedy(const uint16_t *e, int H, int W, int32_t *seam, int64_t *cost, cudaStream_t st) {
  k_greedy<<<1, 32, 0, st>>>(e, H, W, seam, cost);
  return cudaGetLastError();
}

}  // namespace sc

namespace sc {

// ---- self-test of the bounded waits: one thread waits on an mbarrier that nothing completes,
// with a limit of limit_ns, exactly as the search's waits do; when the limit runs out it records
// ERR_TIMEOUT and returns (no trap, no fault), so the host sees SC_ETIMEOUT and the context stays
// usable. ----
__global__ void k_wait_selftest(uint64_t limit_ns, int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);   // one arrival expected; none comes
  fence_mbar_init();
  if (!mbar_wait_bounded(&bar, 0u, limit_ns)) atomicOr(err, ERR_TIMEOUT);
}

cudaError_t launch_wait_selftest(uint64_t limit_ns, int *err, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(limit_ns, err);
  return cudaGetLastError();
}

}  // namespace sc
