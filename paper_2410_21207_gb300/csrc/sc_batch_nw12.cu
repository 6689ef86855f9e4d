// Batched persistent kernel, 12 compute warps (images up to 1344 / 1152 columns for tile heights
// 8 / 16). Every host function that names these kernels lives in this file, so each kernel has
// exactly one definition.
#include "sc_batch.cuh"

namespace sc {

#define SC_BATCH_CASES(X) X(12, 8) X(12, 16)
#define SC_SMEM(N, K) case K: return search_plan<N, K, false, batch_fill_warps(N, K)>(Smax).total;
#define SC_OCC(N, K) case K: batch_configure_cfg<N, K>(); \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<N, K>, Geo<N, K, false>::THREADS, smem); break;
#define SC_LAUNCH(N, K) case K: return launch_batch_cfg<N, K>(items, n, Smax, grid, queue, err, st, pdl);

size_t batch_smem_nw12(int kt, int Smax) {
  switch (kt) { SC_BATCH_CASES(SC_SMEM) default: return (size_t)1 << 30; }
}
int batch_occ_nw12(int kt, int Smax) {
  const size_t smem = batch_smem_nw12(kt, Smax);
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (kt) { SC_BATCH_CASES(SC_OCC) default: break; }
  return (e == cudaSuccess && n > 0) ? n : 1;
}
cudaError_t launch_batch_nw12(int kt, const BatchItem *items, int n, int Smax, int grid, int *queue, int *err,
                             cudaStream_t st, bool pdl) {
  switch (kt) { SC_BATCH_CASES(SC_LAUNCH) default: return cudaErrorInvalidValue; }
}

}  // namespace sc
