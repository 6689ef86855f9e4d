// Batched persistent carving with one thread-block cluster per image (images wider than one CTA,
// and the heaviest images of a batch), templated on the cluster's shape: compute warps NW, tile
// rows KT and backtrack-fill warps FWM; sc_batch_cl.cu and sc_batch_cl_lat.cu instantiate the two
// shapes of sc_batch_cl.h.
// Each cluster repeatedly takes the next image from a queue and carves it completely, like the
// one-CTA batched kernel (sc_batch.cuh), with the cluster-wide seam search (seam_search with CL)
// and the per-seam row work split over the cluster's CTAs: CTA r owns rows r, r + cs, r + 2cs, ...
// Per seam: the search (ends with a cluster barrier); every owned row's refreshed energy pair and
// pending-removal list update, one thread per row; a cluster barrier (the pairs read neighbouring
// rows' words, which the compaction below rewrites); the energy row shifted past the seam with the
// pair written in, one warp per row, and every RPEND seams the image words compacted; a cluster
// barrier. Several clusters run side by side, so a batch of wide images keeps the GPU busy where
// the per-seam cluster path would run one image's latency-bound chain at a time.
#pragma once
#include <atomic>

#include "sc_batch_cl.h"
#include "sc_rowops.cuh"
#include "sc_search.cuh"

namespace sc {

__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// (count) vertical seams of a rows x cols word image whose energy is in it.E
template <int NW, int KT, int FWM>
__device__ void clb_seam_pass(const BatchItem &it, uint32_t *words, int rows, int cols, int count, int32_t *log,
                              int64_t *costs, unsigned char *smem, int Smax, SearchState &st, int *err, int rank,
                              int cs) {
  cg::cluster_group cl = cg::this_cluster();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  int16_t *lb[2] = {it.lists, it.lists + (size_t)rows * RPEND};
  // the staging ring is idle between searches: it holds the owned rows' refreshed pairs
  const SearchPlan plan = search_plan<NW, KT, true, FWM>(Smax);
  uint32_t *pairs = reinterpret_cast<uint32_t *>(smem + plan.ring);
  const int nq = (rows - rank + cs - 1) / cs;   // rows this CTA owns
  const size_t pair_bytes = ((size_t)(nq > 0 ? nq : 0) * 4 + 15) & ~(size_t)15;
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
    seam_search<NW, KT, true, FWM>(a, smem, Smax, st);   // ends with a cluster barrier
    if (refresh_pairs(words, it.pitch, rows, w, it.seam, lb[cur], lb[cur ^ 1], m, nq, rank, cs, pairs, threadIdx.x,
                      blockDim.x))
      atomicOr(err, ERR_BAD_SEAM);
    cl.sync();
    // the owned rows' energy tails, staged through the rest of the idle ring
    if (!shift_rows_bulk(Ecur, it.pe, nq, rank, cs, w, it.seam, pairs, warp, nwarps, lane,
                         reinterpret_cast<unsigned char *>(sbuf + (size_t)warp * sbuf_elems), sbuf_elems * 2) &&
        lane == 0)
      atomicOr(err, ERR_TIMEOUT);
    cur ^= 1;
    if (++m == RPEND) {
      compact_rows_staged(words, it.pitch, nq, rank, cs, lb[cur], m, w - 1, warp, nwarps, lane,
                          reinterpret_cast<uint32_t *>(sbuf + (size_t)warp * sbuf_elems), sbuf_elems / 2);
      m = 0;
    }
    fence_async_global();   // the next search stages the compacted energy rows with TMA
    cl.sync();
  }
  if (m > 0) {
    compact_rows_staged(words, it.pitch, nq, rank, cs, lb[cur], m, cols - count, warp, nwarps, lane,
                        reinterpret_cast<uint32_t *>(sbuf + (size_t)warp * sbuf_elems), sbuf_elems / 2);
    cl.sync();
  }
}

// e1 energy of every owned row (the search's TMA reads it next)
__device__ inline void clb_energy(const uint32_t *words, int pitch, int rows, int cols, uint16_t *E, int pe, int rank, int cs) {
  for (int i = rank; i < rows; i += cs)
    for (int j = threadIdx.x; j < cols; j += blockDim.x)
      E[(int64_t)i * pe + j] = (uint16_t)energy_at(words, pitch, rows, cols, i, j);
  fence_async_global();
  cg::this_cluster().sync();
}

// rows x cols word image -> its transpose, 32 x 32 tiles through shared memory, tiles dealt out
// over the cluster's warps
__device__ inline void clb_transpose(const uint32_t *src, int ps, int rows, int cols, uint32_t *dst, int pd, uint32_t *tile,
                              int ntw, int rank, int cs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < ntw) {
    uint32_t *t = tile + warp * 32 * 33;
    const int tr = (rows + 31) / 32, tc = (cols + 31) / 32;
    for (int tix = rank * ntw + warp; tix < tr * tc; tix += cs * ntw) {
      const int by = (tix / tc) * 32, bx = (tix % tc) * 32;
      for (int r = 0; r < 32; ++r) {
        const int i = by + r, j = bx + lane;
        if (i < rows && j < cols) t[r * 33 + lane] = src[(int64_t)i * ps + j];
      }
      __syncwarp();
      for (int r = 0; r < 32; ++r) {
        const int j = bx + r, i = by + lane;
        if (i < rows && j < cols) dst[(int64_t)j * pd + i] = t[lane * 33 + r];
      }
      __syncwarp();
    }
  }
  cg::this_cluster().sync();
}

template <int NW, int KT, int FWM>
__device__ void clb_carve_item(const BatchItem &it, unsigned char *smem, int Smax, SearchState &st, int *err, int rank,
                               int cs) {
  const int H = it.H, W = it.W, C = it.C, tw = it.tw, th = it.th;
  const int64_t tid = (int64_t)rank * blockDim.x + threadIdx.x, nth = (int64_t)cs * blockDim.x;
  const int64_t npx = (int64_t)H * W;
  for (int64_t q = tid; q < npx; q += nth) {
    const int i = (int)(q / W), j = (int)(q % W);
    it.img_w[(int64_t)i * it.pitch + j] = pack_pixel(it.img + q * C, C);
  }
  cg::this_cluster().sync();
  clb_energy(it.img_w, it.pitch, H, W, it.E + E_PADL, it.pe, rank, cs);
  const int nv = W - tw, nh = H - th;
  clb_seam_pass<NW, KT, FWM>(it, it.img_w, H, W, nv, it.seam_log, it.cost_log, smem, Smax, st, err, rank, cs);
  if (nh > 0) {
    const SearchPlan plan = search_plan<NW, KT, true, FWM>(Smax);
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem + plan.ring);   // the ring is idle between searches
    const int ntw_fit = (int)((plan.bars - plan.ring) / (32 * 33 * 4));
    const int ntw = ntw_fit < NW + 1 ? ntw_fit : NW + 1;
    clb_transpose(it.img_w, it.pitch, H, tw, it.img2_w, it.pitch, tile, ntw, rank, cs);   // tw rows x H columns
    clb_energy(it.img2_w, it.pitch, tw, H, it.E + E_PADL, it.pe, rank, cs);
    clb_seam_pass<NW, KT, FWM>(it, it.img2_w, tw, H, nh, it.seam_log ? it.seam_log + (size_t)nv * H : nullptr,
                  it.cost_log ? it.cost_log + nv : nullptr, smem, Smax, st, err, rank, cs);
    clb_transpose(it.img2_w, it.pitch, tw, th, it.img_w, it.pitch, tile, ntw, rank, cs);   // th rows x tw columns
  }
  const int64_t nout = (int64_t)th * tw;
  for (int64_t q = tid; q < nout; q += nth) {
    const int i = (int)(q / tw), j = (int)(q % tw);
    unpack_pixel(it.img_w[(int64_t)i * it.pitch + j], it.out + q * C, C);
  }
  if (it.done) __threadfence_system();   // every thread's output bytes before the completion word
  cg::this_cluster().sync();
  if (it.done && rank == 0 && threadIdx.x == 0) *(volatile int *)it.done = (*(volatile int *)err != 0) ? 2 : 1;
}

template <int NW, int KT, int FWM>
__global__ void __launch_bounds__(Geo<NW, KT, true, FWM>::THREADS, 1)
    k_batch_cl(const BatchItem *__restrict__ items, int n, int Smax, int *queue, int *err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int next;
  __shared__ BatchItem cur;   // the current image's descriptor, read where its fields are used
  // a launch chained behind this one (programmatic dependent launch) may start once every CTA of
  // this launch is resident: a batch plan places its clusters before the one-CTA launch fills the
  // remaining SMs
  pdl_launch_dependents();
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), cs = (int)cl.num_blocks();
  search_init<NW, KT, true, FWM>(smem, Smax);
  cl.sync();
  SearchState st;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) next = atomicAdd(queue, 1);
    cl.sync();
    const int k = *cl.map_shared_rank(&next, 0);
    cl.sync();   // every CTA has read rank 0's `next` before it can change or its CTA exit
    if (k >= n) break;
    if (threadIdx.x == 0) cur = items[k];
    __syncthreads();
    clb_carve_item<NW, KT, FWM>(cur, smem, Smax, st, err, rank, cs);
  }
  // chained behind another launch: do not end before it does (no-op otherwise)
  pdl_wait_prerequisites();
}

// The host side of one shape: shared memory, capacity and launch (instantiated once per shape).
template <int NW, int KT, int FWM>
struct ClShapeHost {
  using G = Geo<NW, KT, true, FWM>;
  static size_t smem_bytes(int Smax) { return search_plan<NW, KT, true, FWM>(Smax).total; }
  static cudaError_t configure() {
    static std::atomic<bool> done{false};
    if (done.load()) return cudaSuccess;
    auto k = k_batch_cl<NW, KT, FWM>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BATCH_CL_SMEM_MAX);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    done.store(true);
    return cudaSuccess;
  }
  static void cfg_for(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at, int clusters, int cs, int Smax, cudaStream_t st,
                      bool pdl = false) {
    cfg = {};
    cfg.gridDim = dim3(cs * clusters);
    cfg.blockDim = dim3(G::THREADS);
    cfg.dynamicSmemBytes = smem_bytes(Smax);
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 2 : 1;
  }
  static cudaError_t capacity(int cs, int Smax, int *clusters) {
    cudaError_t e = configure();
    if (e != cudaSuccess) return e;
    if (cs < 1 || cs > MAX_CLUSTER || smem_bytes(Smax) > BATCH_CL_SMEM_MAX) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[2];
    cfg_for(cfg, at, 1, cs, Smax, nullptr);
    return cudaOccupancyMaxActiveClusters(clusters, k_batch_cl<NW, KT, FWM>, &cfg);
  }
  static cudaError_t launch(const BatchItem *items, int n, int cs, int Smax, int clusters, int *queue, int *err,
                            cudaStream_t st, bool pdl) {
    cudaError_t e = configure();
    if (e != cudaSuccess) return e;
    if (cs < 1 || cs > MAX_CLUSTER || clusters < 1 || smem_bytes(Smax) > BATCH_CL_SMEM_MAX) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[2];
    cfg_for(cfg, at, clusters, cs, Smax, st, pdl);
    return cudaLaunchKernelEx(&cfg, k_batch_cl<NW, KT, FWM>, items, n, Smax, queue, err);
  }
  static ClOps ops() { return ClOps{G::OWC, &smem_bytes, &capacity, &launch}; }
};

}  // namespace sc
