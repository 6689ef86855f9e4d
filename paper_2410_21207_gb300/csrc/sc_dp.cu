// One seam search per launch on one thread-block cluster (the plain per-seam path and
// sc_find_seam). The search itself is seam_search in sc_search.cuh.
#include "sc_search.cuh"

namespace sc {

// The search of one map is a chain of H dependent rows, so its shape is chosen for latency: tall
// 32-row tiles cross a tile boundary (strip exchange, staging barrier, bookkeeping) half as often
// as 16-row ones, at the price of more redundant halo columns, which only costs idle SMs. Shapes
// in order of preference; the first whose cluster covers W is used.
struct DpShapeDef {
  int nw, kt, ow;
};
constexpr DpShapeDef kDpShapes[] = {
    {4, 32, Geo<4, 32, true>::OWC}, {8, 32, Geo<8, 32, true>::OWC}, {8, 16, Geo<8, 16, true>::OWC}};

DpShape dp_shape_for(int W) {
  DpShape s{};
  for (const DpShapeDef &d : kDpShapes) {
    s.nw = d.nw;
    s.kt = d.kt;
    s.ow = d.ow;
    s.cs = (W + d.ow - 1) / d.ow;
    if (s.cs < 1) s.cs = 1;
    if (s.cs <= MAX_CLUSTER) break;
  }
  return s;
}

// Super-tile height: KS (32) rows for the 4-warp shape, whose ancestor chain is local (the table is
// gathered in rank 0) and whose serial backtrack fill halves against 64; KS_WIDE (64) for the wide
// shapes and forward energy, whose chain hops cross CTAs through DSMEM and would double.
template <int NW, int KT, bool FWD>
__host__ __device__ constexpr int dp_super_rows() { return (NW == 4 && KT == 32 && !FWD) ? KS : KS_WIDE; }

template <int NW, int KT, bool FWD = false>
__global__ void __launch_bounds__(Geo<NW, KT, true>::THREADS, 1) k_dp(DpArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int KSS = dp_super_rows<NW, KT, FWD>();
  const int S = (p.H + KSS - 1) / KSS;
  search_init<NW, KT, true, FILL_WARPS_MAX, FWD, KSS>(smem, S);
  // neighbours push into each other's halo buffers: every CTA's barriers must be initialised first
  cg::this_cluster().sync();
  // the set-up above overlaps the previous kernel of the seam loop; its results are read below
  pdl_launch_dependents();
  pdl_wait_prerequisites();
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
  a.pstride = p.pstride;
  SearchState st;
  seam_search<NW, KT, true, FILL_WARPS_MAX, FWD, KSS>(a, smem, S, st);
}

template <int NW, int KT, bool FWD = false>
static cudaError_t launch_dp_shape(const DpArgs &a, int cs, cudaStream_t st) {
  constexpr int KSS = dp_super_rows<NW, KT, FWD>();
  const size_t smem = search_plan<NW, KT, true, FILL_WARPS_MAX, FWD, KSS>((a.H + KSS - 1) / KSS).total;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_dp<NW, KT, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_dp<NW, KT, FWD>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (smem > 232448) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(Geo<NW, KT, true>::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // may start before its predecessor ends
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_dp<NW, KT, FWD>, a);
}

// forward energy stages three planes per row: one shape, 4 warps x 16-row tiles (W <= 4096)
int dp_forward_max_width() { return MAX_CLUSTER * Geo<4, 16, true>::OWC; }

cudaError_t launch_dp(const DpArgs &a, cudaStream_t st) {
  if (a.pstride > 0) {
    const int cs = (a.W + Geo<4, 16, true>::OWC - 1) / Geo<4, 16, true>::OWC;
    if (cs > MAX_CLUSTER) return cudaErrorInvalidValue;
    return launch_dp_shape<4, 16, true>(a, cs < 1 ? 1 : cs, st);
  }
  const DpShape s = dp_shape_for(a.W);
  if (s.cs > MAX_CLUSTER) return cudaErrorInvalidValue;
  if (s.nw == 4 && s.kt == 32) return launch_dp_shape<4, 32>(a, s.cs, st);
  if (s.nw == 8 && s.kt == 32) return launch_dp_shape<8, 32>(a, s.cs, st);
  return launch_dp_shape<8, 16>(a, s.cs, st);
}

}  // namespace sc
