// Batched persistent carving with one thread-block cluster per image.
#pragma once
#include "sc_batch_item.h"

namespace sc {

constexpr size_t BATCH_CL_SMEM_MAX = 232448 - 1024;   // the opt-in limit minus static shared memory

// Two cluster shapes of the persistent kernel:
//   CL_WIDE: 8 compute warps, 8-row tiles, 768 own columns per CTA. Images wider than one CTA of the
//            one-CTA kernel: few CTAs per image, little redundant halo work (throughput).
//   CL_LAT:  8 compute warps, 32-row tiles, 384 own columns per CTA. The heaviest images of a
//            batch, and the serving form's wide and heavy requests: a quarter of the tile boundaries
//            per seam and twice the CTAs, so one image's seams finish sooner (latency), at more SM
//            time per seam.
enum ClShape { CL_WIDE = 0, CL_LAT = 1 };

struct ClOps {
  int own;                                                     // columns each CTA of a cluster owns
  size_t (*smem)(int Smax);                                    // dynamic shared memory per CTA
  cudaError_t (*capacity)(int cs, int Smax, int *clusters);    // clusters of cs CTAs resident at once
  // `clusters` persistent clusters of cs CTAs carve items[0..n) (a queue counter at *queue, zeroed);
  // every CTA triggers its programmatic dependents at its start; pdl: launched as a programmatic
  // dependent of the launch before it on st, and does not end before that launch does
  cudaError_t (*launch)(const BatchItem *items, int n, int cs, int Smax, int clusters, int *queue, int *err,
                        cudaStream_t st, bool pdl);
};

ClOps cl_ops_wide();
ClOps cl_ops_lat();
inline ClOps cl_ops(int shape) { return shape == CL_LAT ? cl_ops_lat() : cl_ops_wide(); }

// columns each CTA of the cluster owns: an image of searched width w needs ceil(w / own) CTAs
inline int batch_cl_own_cols(int shape = CL_WIDE) { return cl_ops(shape).own; }
inline size_t batch_cl_smem_bytes(int Smax, int shape = CL_WIDE) { return cl_ops(shape).smem(Smax); }
inline cudaError_t batch_cl_capacity(int cs, int Smax, int *clusters, int shape = CL_WIDE) {
  return cl_ops(shape).capacity(cs, Smax, clusters);
}
inline cudaError_t launch_batch_cl(const BatchItem *items, int n, int cs, int Smax, int clusters, int *queue, int *err,
                                   cudaStream_t st, int shape = CL_WIDE, bool pdl = false) {
  return cl_ops(shape).launch(items, n, cs, Smax, clusters, queue, err, st, pdl);
}

}  // namespace sc
