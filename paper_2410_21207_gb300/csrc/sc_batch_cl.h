// Batched persistent carving with one thread-block cluster per image (images wider than a CTA).
#pragma once
#include "sc_batch_item.h"

namespace sc {

constexpr size_t BATCH_CL_SMEM_MAX = 232448 - 1024;   // the opt-in limit minus static shared memory

// columns each CTA of the cluster owns: an image of searched width w needs ceil(w / own) CTAs
int batch_cl_own_cols();
size_t batch_cl_smem_bytes(int Smax);
// clusters of cs CTAs (shared-memory plan for Smax super-tiles) resident on the GPU at once
cudaError_t batch_cl_capacity(int cs, int Smax, int *clusters);
// `clusters` persistent clusters of cs CTAs carve items[0..n) (a queue counter at *queue, zeroed)
cudaError_t launch_batch_cl(const BatchItem *items, int n, int cs, int Smax, int clusters, int *queue, int *err,
                            cudaStream_t st);

}  // namespace sc
