// Batched persistent carving: one launch carves many images of uneven sizes. Each CTA repeatedly
// takes the next image from a queue (one atomic counter) and carves it completely on its own: pack,
// e1 energy, every vertical seam (search, local refresh, compaction), the horizontal pass through a
// transposition, and unpack, with CTA barriers between the phases. The seam search is
// seam_search<NW, KT, false> (sc_search.cuh), so an image fits one CTA when every searched width
// is at most NW * (32*V - 2*KT) columns; the host routes wider images to the cluster path.
#pragma once
#include "sc_batch_item.h"
#include "sc_rowops.cuh"
#include "sc_search.cuh"

namespace sc {

// Backtrack-fill warps of the one-CTA kernel: every warp of the CTA (one round of fills for images
// up to 64 * (NW + 1) rows); their direction rows share the idle staging ring.
__host__ __device__ constexpr int batch_fill_warps(int nw, int kt) { return 16; }

__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// rows x cols word image -> its transpose (cols x rows), 32x32 tiles staged in shared memory; `tile`
// holds `ntw` warps' 32x33 tiles.
__device__ inline void cta_transpose(const uint32_t *src, int ps, int rows, int cols, uint32_t *dst, int pd,
                                     uint32_t *tile, int ntw) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= ntw) return;
  uint32_t *t = tile + warp * 32 * 33;
  const int tr = (rows + 31) / 32, tc = (cols + 31) / 32;
  for (int tix = warp; tix < tr * tc; tix += ntw) {
    const int by = (tix / tc) * 32, bx = (tix % tc) * 32;
    for (int r = 0; r < 32; ++r) {
      const int i = by + r, j = bx + lane;
      if (i < rows && j < cols) t[r * 33 + lane] = src[(int64_t)i * ps + j];
    }
    __syncwarp();
    for (int r = 0; r < 32; ++r) {
      const int j = bx + r, i = by + lane;   // dst row j, column i
      if (i < rows && j < cols) dst[(int64_t)j * pd + i] = t[lane * 33 + r];
    }
    __syncwarp();
  }
}

// (count) vertical seams of a rows x cols word image, whose energy is in it.E. Per seam: the
// search, then one warp per row computes the refreshed energy pair through the pending-removal
// lists, adds the removal to the row's list and compacts the energy row; the words are compacted
// every RPEND seams and at the end of the pass.
template <int NW, int KT>
__device__ void batch_seam_pass(const BatchItem &it, uint32_t *words, int rows, int cols, int count,
                                int32_t *log, int64_t *costs, unsigned char *smem, int Smax, SearchState &st,
                                int *err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  int16_t *lb[2] = {it.lists, it.lists + (size_t)rows * RPEND};
  // the staging ring is idle between searches: it holds the rows' refreshed pairs
  const SearchPlan plan = search_plan<NW, KT, false, batch_fill_warps(NW, KT)>(Smax);
  uint32_t *pairs = reinterpret_cast<uint32_t *>(smem + plan.ring);
  const size_t pair_bytes = ((size_t)rows * 4 + 15) & ~(size_t)15;
  uint16_t *sbuf = reinterpret_cast<uint16_t *>(smem + plan.ring + pair_bytes);
  const int sbuf_elems = (int)(((plan.bars - plan.ring - pair_bytes) / nwarps) & ~(size_t)15) / 2;
  uint16_t *const Ecur = it.E + E_PADL;
  int cur = 0, m = 0;
  for (int t = 0; t < count; ++t) {
    const int w = cols - t;
    SearchArgs a;
    a.E = Ecur;
    a.pitch_e = it.pe;
    a.H = rows;
    a.W = w;
    a.Mrow = it.Mrow + E_PADL;
    a.seam = it.seam;
    a.seam_log = log ? log + (size_t)t * rows : nullptr;
    a.cost = costs ? costs + t : nullptr;
    a.err = err;
    a.gated = false;
    seam_search<NW, KT, false, batch_fill_warps(NW, KT)>(a, smem, Smax, st);   // ends with a CTA barrier: the seam is complete
    // every row's refreshed pair and list update, one thread per row (into the idle staging ring)
    if (refresh_pairs(words, it.pitch, rows, w, it.seam, lb[cur], lb[cur ^ 1], m, rows, 0, 1, pairs, threadIdx.x,
                      blockDim.x))
      atomicOr(err, ERR_BAD_SEAM);
    __syncthreads();
    // energy rows compacted past the seam in place, the pair at the new columns s-1 and s; the
    // tails are staged by TMA through the rest of the idle ring, one buffer per warp
    if (!shift_rows_bulk(Ecur, it.pe, rows, 0, 1, w, it.seam, pairs, warp, nwarps, lane,
                         reinterpret_cast<unsigned char *>(sbuf + (size_t)warp * sbuf_elems), sbuf_elems * 2) &&
        lane == 0)
      atomicOr(err, ERR_TIMEOUT);
    cur ^= 1;
    fence_proxy_async_global();   // the next search stages the compacted energy rows with TMA
    __syncthreads();
    if (++m == RPEND) {
      compact_rows_staged(words, it.pitch, rows, 0, 1, lb[cur], m, w - 1, warp, nwarps, lane,
                          reinterpret_cast<uint32_t *>(sbuf + (size_t)warp * sbuf_elems), sbuf_elems / 2);
      m = 0;
      __syncthreads();
    }
  }
  if (m > 0) {
    compact_rows_staged(words, it.pitch, rows, 0, 1, lb[cur], m, cols - count, warp, nwarps, lane,
                        reinterpret_cast<uint32_t *>(sbuf + (size_t)warp * sbuf_elems), sbuf_elems / 2);
    __syncthreads();
  }
}

template <int NW, int KT>
__device__ void batch_energy(const uint32_t *words, int pitch, int rows, int cols, uint16_t *E, int pe) {
  const int64_t n = (int64_t)rows * cols;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
    const int i = (int)(q / cols), j = (int)(q % cols);
    E[(int64_t)i * pe + j] = (uint16_t)energy_at(words, pitch, rows, cols, i, j);
  }
  fence_proxy_async_global();
  __syncthreads();
}

template <int NW, int KT>
__device__ void batch_carve_item(const BatchItem &it, unsigned char *smem, int Smax, SearchState &st, int *err) {
  const int H = it.H, W = it.W, C = it.C, tw = it.tw, th = it.th;
  const int64_t npx = (int64_t)H * W;
  for (int64_t q = threadIdx.x; q < npx; q += blockDim.x) {
    const int i = (int)(q / W), j = (int)(q % W);
    it.img_w[(int64_t)i * it.pitch + j] = pack_pixel(it.img + q * C, C);
  }
  __syncthreads();
  batch_energy<NW, KT>(it.img_w, it.pitch, H, W, it.E + E_PADL, it.pe);
  const int nv = W - tw, nh = H - th;
  batch_seam_pass<NW, KT>(it, it.img_w, H, W, nv, it.seam_log, it.cost_log, smem, Smax, st, err);
  uint32_t *res = it.img_w;
  if (nh > 0) {
    const SearchPlan plan = search_plan<NW, KT, false, batch_fill_warps(NW, KT)>(Smax);
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem + plan.ring);   // the ring is idle between searches
    const int ntw_fit = (int)((plan.bars - plan.ring) / (32 * 33 * 4));
    const int ntw = ntw_fit < NW + 1 ? ntw_fit : NW + 1;
    cta_transpose(it.img_w, it.pitch, H, tw, it.img2_w, it.pitch, tile, ntw);   // tw rows x H columns
    __syncthreads();
    batch_energy<NW, KT>(it.img2_w, it.pitch, tw, H, it.E + E_PADL, it.pe);
    batch_seam_pass<NW, KT>(it, it.img2_w, tw, H, nh, it.seam_log ? it.seam_log + (size_t)nv * H : nullptr,
                            it.cost_log ? it.cost_log + nv : nullptr, smem, Smax, st, err);
    cta_transpose(it.img2_w, it.pitch, tw, th, it.img_w, it.pitch, tile, ntw);  // th rows x tw columns
    __syncthreads();
  }
  const int64_t nout = (int64_t)th * tw;
  for (int64_t q = threadIdx.x; q < nout; q += blockDim.x) {
    const int i = (int)(q / tw), j = (int)(q % tw);
    unpack_pixel(res[(int64_t)i * it.pitch + j], it.out + q * C, C);
  }
  if (it.done) __threadfence_system();   // every thread's output bytes before the completion word
  __syncthreads();
  if (it.done && threadIdx.x == 0) *(volatile int *)it.done = (*(volatile int *)err != 0) ? 2 : 1;
}

template <int NW, int KT>
__global__ void __launch_bounds__(Geo<NW, KT, false>::THREADS, 1)
    k_batch(const BatchItem *__restrict__ items, int n, int Smax, int *queue, int *err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int next;
  // the current image's descriptor lives in shared memory and its fields are read where they are
  // used, so they do not occupy registers across the seam loop
  __shared__ BatchItem cur;
  search_init<NW, KT, false, batch_fill_warps(NW, KT)>(smem, Smax);
  __syncthreads();
  SearchState st;
  for (;;) {
    if (threadIdx.x == 0) {
      next = atomicAdd(queue, 1);
      if (next < n) cur = items[next];
    }
    __syncthreads();
    const int k = next;
    __syncthreads();
    if (k >= n) break;
    batch_carve_item<NW, KT>(cur, smem, Smax, st, err);
    __syncthreads();
  }
  // launched as a programmatic dependent of cluster launches (a batch plan starts them first): this
  // launch does not end before they do, so work after it on the stream follows all of them
  pdl_wait_prerequisites();
}

constexpr size_t BATCH_SMEM_MAX = 232448 - 1024;   // the opt-in limit minus room for static shared memory

template <int NW, int KT>
cudaError_t batch_configure_cfg() {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_batch<NW, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BATCH_SMEM_MAX);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  return cudaSuccess;
}

template <int NW, int KT>
cudaError_t launch_batch_cfg(const BatchItem *items, int n, int Smax, int grid, int *queue, int *err,
                             cudaStream_t st, bool pdl) {
  const size_t smem = search_plan<NW, KT, false, batch_fill_warps(NW, KT)>(Smax).total;
  if (smem > BATCH_SMEM_MAX) return cudaErrorInvalidValue;
  cudaError_t e = batch_configure_cfg<NW, KT>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(Geo<NW, KT, false>::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_batch<NW, KT>, items, n, Smax, queue, err);
}

}  // namespace sc
