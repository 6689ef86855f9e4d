// The CL_WIDE shape of the cluster-per-image persistent kernel (sc_batch_cl.cuh): 8 compute warps,
// 8-row tiles.
#include "sc_batch_cl.cuh"

namespace sc {

ClOps cl_ops_wide() { return ClShapeHost<8, 8, 4>::ops(); }

}  // namespace sc
