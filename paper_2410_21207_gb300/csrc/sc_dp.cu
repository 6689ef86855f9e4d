// One seam search per launch on one thread-block cluster (the plain per-seam path and
// sc_find_seam). The search itself is seam_search in sc_search.cuh.
#include "sc_search.cuh"

namespace sc {

using GeoC4 = Geo<4, DP_KT, true>;
using GeoC8 = Geo<8, DP_KT, true>;

DpShape dp_shape_for(int W) {
  DpShape s;
  s.nw = 4;
  s.ow = GeoC4::OWC;
  s.cs = (W + s.ow - 1) / s.ow;
  if (s.cs > MAX_CLUSTER) {
    s.nw = 8;
    s.ow = GeoC8::OWC;
    s.cs = (W + s.ow - 1) / s.ow;
  }
  if (s.cs < 1) s.cs = 1;
  return s;
}

size_t dp_smem_bytes(int nw, int H) {
  const int S = (H + KS - 1) / KS;
  return nw == 4 ? search_plan<4, DP_KT, true>(S).total : search_plan<8, DP_KT, true>(S).total;
}

template <int NW>
__global__ void __launch_bounds__(Geo<NW, DP_KT, true>::THREADS, 1) k_dp(DpArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int S = (p.H + KS - 1) / KS;
  search_init<NW, DP_KT, true>(smem, S);
  // neighbours push into each other's halo buffers: every CTA's barriers must be initialised first
  cg::this_cluster().sync();
  SearchArgs a;
  a.E = p.E;
  a.pitch_e = p.pitch_e;
  a.H = p.H;
  a.W = p.W;
  a.Mrow = p.Mrow;
  a.seam = p.seam;
  a.seam_log = p.seam_log;
  a.cost = p.cost;
  a.err = p.err;
  a.gated = (p.gate != nullptr) && (*p.gate & ERR_ENERGY_RANGE);
  SearchState st;
  seam_search<NW, DP_KT, true>(a, smem, S, st);
}

template <int NW>
static cudaError_t launch_dp_nw(const DpArgs &a, int cs, cudaStream_t st) {
  const size_t smem = dp_smem_bytes(NW, a.H);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_dp<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_dp<NW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (smem > 232448) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(Geo<NW, DP_KT, true>::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_dp<NW>, a);
}

cudaError_t launch_dp(const DpArgs &a, cudaStream_t st) {
  const DpShape s = dp_shape_for(a.W);
  if (s.cs > MAX_CLUSTER) return cudaErrorInvalidValue;
  return s.nw == 4 ? launch_dp_nw<4>(a, s.cs, st) : launch_dp_nw<8>(a, s.cs, st);
}

}  // namespace sc
