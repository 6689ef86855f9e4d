// The CL_LAT shape of the cluster-per-image persistent kernel (sc_batch_cl.cuh): 8 compute warps,
// 32-row tiles.
#include "sc_batch_cl.cuh"

namespace sc {

ClOps cl_ops_lat() { return ClShapeHost<8, 32, 4>::ops(); }

}  // namespace sc
