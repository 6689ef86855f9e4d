// Dispatch from a (compute warps, tile height) configuration to the file that instantiates it.
#include "sc_batch_item.h"

namespace sc {

size_t batch_smem_nw8(int kt, int Smax);
size_t batch_smem_nw12(int kt, int Smax);
size_t batch_smem_nw15(int kt, int Smax);
int batch_occ_nw8(int kt, int Smax);
int batch_occ_nw12(int kt, int Smax);
int batch_occ_nw15(int kt, int Smax);
cudaError_t launch_batch_nw8(int kt, const BatchItem *items, int n, int Smax, int grid, int *queue, int *err,
                             cudaStream_t st, bool pdl);
cudaError_t launch_batch_nw12(int kt, const BatchItem *items, int n, int Smax, int grid, int *queue, int *err,
                              cudaStream_t st, bool pdl);
cudaError_t launch_batch_nw15(int kt, const BatchItem *items, int n, int Smax, int grid, int *queue, int *err,
                              cudaStream_t st, bool pdl);

size_t batch_smem_bytes(int nw, int kt, int Smax) {
  return nw == 8 ? batch_smem_nw8(kt, Smax)
         : nw == 12 ? batch_smem_nw12(kt, Smax)
         : nw == 15 ? batch_smem_nw15(kt, Smax) : (size_t)1 << 30;
}

int batch_blocks_per_sm(int nw, int kt, int Smax) {
  return nw == 8 ? batch_occ_nw8(kt, Smax) : nw == 12 ? batch_occ_nw12(kt, Smax) : nw == 15 ? batch_occ_nw15(kt, Smax) : 1;
}

cudaError_t launch_batch(int nw, int kt, const BatchItem *items, int n, int Smax, int grid, int *queue, int *err,
                         cudaStream_t st, bool pdl) {
  if (nw == 8) return launch_batch_nw8(kt, items, n, Smax, grid, queue, err, st, pdl);
  if (nw == 12) return launch_batch_nw12(kt, items, n, Smax, grid, queue, err, st, pdl);
  if (nw == 15) return launch_batch_nw15(kt, items, n, Smax, grid, queue, err, st, pdl);
  return cudaErrorInvalidValue;
}

}  // namespace sc
