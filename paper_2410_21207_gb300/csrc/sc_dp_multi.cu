// Many seam searches of one size in one launch: cluster c searches map c. Each search is the
// cluster-wide seam_search (sc_search.cuh); the clusters run side by side, so with enough maps in
// flight the pass is bound by the GPU's throughput instead of one map's chain of dependent rows.
// The maps are read where the caller keeps them (seam_search's in-place form, which also checks
// each map's cost range), so a call moves no more than the search's own bytes.
// Four tile shapes are built (compute warps per CTA x DP tile rows). The kernel is bound by the
// latency of its dependent chains, so the shapes are compiled for as many resident CTAs per SM as
// registers and shared memory allow (2 of 8 warps, 4 of 4 warps; four backtrack-fill warps keep
// the shared-memory plan small), and 8-row tiles waste fewer columns on the trapezoids' slopes.
#include <atomic>
#include <map>
#include <mutex>
#include "sc_search.cuh"

namespace sc {

// backtrack-fill warps per CTA: 7 (of 9) gives the 68 super-tiles of a 2160-row map two fill rounds
// on a 5-CTA cluster instead of four, with the direction rows still inside the idle staging ring;
// below FILL_WARPS_MAX, so the throughput-bound forms of the search are kept (2-4-row chunks)
constexpr int MULTI_FILL_WARPS = 7;

template <int NW, int KT>
__global__ void __launch_bounds__(Geo<NW, KT, true>::THREADS, NW == 8 ? 2 : 4) k_dp_multi(const DpArgs *__restrict__ ps,
                                                                                          const __grid_constant__ MultiArgs inl) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int img = blockIdx.x / cg::this_cluster().num_blocks();
  const DpArgs p = ps ? ps[img] : inl.a[img];
  const int S = (p.H + KS - 1) / KS;
  search_init<NW, KT, true, MULTI_FILL_WARPS, false, KS, true>(smem, S);
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
  a.pitch_m = p.pitch_m;
  a.gate = p.gate;
  SearchState st;
  seam_search<NW, KT, true, MULTI_FILL_WARPS, false, KS, true>(a, smem, S, st);
}

namespace {

struct MultiShape {
  int nw, kt, ow;
  cudaError_t (*configure)();
  cudaError_t (*launch)(const DpArgs *, const MultiArgs *, int, int, int, cudaStream_t);
  cudaError_t (*capacity)(int, int, int *);
  size_t (*smem)(int);
};

template <int NW, int KT>
size_t multi_smem(int H) {
  return search_plan<NW, KT, true, MULTI_FILL_WARPS, false, KS, true>((H + KS - 1) / KS).total;
}

template <int NW, int KT>
cudaError_t multi_configure() {
  static std::atomic<bool> done{false};
  if (done.load()) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_dp_multi<NW, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_dp_multi<NW, KT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  done.store(true);
  return cudaSuccess;
}

template <int NW, int KT>
void multi_cfg(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at, int n, int H, int cs, cudaStream_t st) {
  cfg = {};
  cfg.gridDim = dim3(cs * n);
  cfg.blockDim = dim3(Geo<NW, KT, true>::THREADS);
  cfg.dynamicSmemBytes = multi_smem<NW, KT>(H);
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
}

template <int NW, int KT>
cudaError_t multi_launch(const DpArgs *dargs, const MultiArgs *inl, int n, int H, int cs, cudaStream_t st) {
  cudaError_t e = multi_configure<NW, KT>();
  if (e != cudaSuccess) return e;
  if (multi_smem<NW, KT>(H) > 232448) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  multi_cfg<NW, KT>(cfg, at, n, H, cs, st);
  static const MultiArgs none{};
  return cudaLaunchKernelEx(&cfg, k_dp_multi<NW, KT>, inl ? nullptr : dargs, inl ? *inl : none);
}

template <int NW, int KT>
cudaError_t multi_capacity(int H, int cs, int *n_out) {
  cudaError_t e = multi_configure<NW, KT>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  multi_cfg<NW, KT>(cfg, at, 1, H, cs, nullptr);
  return cudaOccupancyMaxActiveClusters(n_out, k_dp_multi<NW, KT>, &cfg);
}

#define SC_MULTI_SHAPE(N, K) \
  { N, K, Geo<N, K, true>::OWC, multi_configure<N, K>, multi_launch<N, K>, multi_capacity<N, K>, multi_smem<N, K> }
const MultiShape kShapes[] = {SC_MULTI_SHAPE(8, 8), SC_MULTI_SHAPE(4, 8), SC_MULTI_SHAPE(8, 16), SC_MULTI_SHAPE(4, 16)};
#undef SC_MULTI_SHAPE
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));

std::atomic<int> g_forced{-1};   // index into kShapes, or -1 for the automatic choice

int clusters_for(const MultiShape &sh, int W) { return (W + sh.ow - 1) / sh.ow; }

// Relative time per map of a shape on a GPU full of H x W searches: the columns every lane
// computes per useful column, times a per-tile overhead factor (fit to measurements of 1920- and
// 3840-column maps: one tile boundary costs about as much as 3.75 rows), divided by the compute
// warps resident on an SM.
double shape_cost(const MultiShape &sh, int H, int W) {
  const int cs = clusters_for(sh, W);
  if (cs > MAX_CLUSTER) return -1.0;
  int clusters = 0, dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -1.0;
  if (sh.capacity(H, cs, &clusters) != cudaSuccess || clusters < 1 || sms < 1) return -1.0;
  const double warps_per_sm = (double)clusters * cs * sh.nw / sms;
  const double computed = (double)cs * sh.nw * 32 * V / W;
  return computed * (1.0 + 3.75 / sh.kt) / warps_per_sm;
}

std::mutex g_pick_mu;
std::map<std::pair<int, int>, int> g_pick;   // (super-tile count, W) -> shape index

int pick_shape(int H, int W) {
  const int f = g_forced.load();
  if (f >= 0) return (kShapes[f].ow * MAX_CLUSTER >= W) ? f : -1;
  const std::pair<int, int> key((H + KS - 1) / KS, W);
  std::lock_guard<std::mutex> lk(g_pick_mu);
  auto it = g_pick.find(key);
  if (it != g_pick.end()) return it->second;
  int best = -1;
  double best_cost = 0.0;
  for (int k = 0; k < kNumShapes; ++k) {
    const double c = shape_cost(kShapes[k], H, W);
    if (c > 0.0 && (best < 0 || c < best_cost)) {
      best = k;
      best_cost = c;
    }
  }
  if (best >= 0) g_pick[key] = best;
  return best;
}

}  // namespace

int dp_multi_set_shape(int nw, int kt) {
  if (nw == 0 && kt == 0) {
    g_forced.store(-1);
    return 0;
  }
  for (int k = 0; k < kNumShapes; ++k)
    if (kShapes[k].nw == nw && kShapes[k].kt == kt) {
      g_forced.store(k);
      return 0;
    }
  return -1;
}

cudaError_t dp_multi_capacity(int H, int W, int *n_out) {
  const int k = pick_shape(H, W);
  if (k < 0) return cudaErrorInvalidValue;
  const int cs = clusters_for(kShapes[k], W);
  return kShapes[k].capacity(H, cs, n_out);
}

cudaError_t launch_dp_multi(const DpArgs *dargs_dev, const MultiArgs *inl, int n, int H, int W, cudaStream_t st) {
  const int k = pick_shape(H, W);
  if (k < 0 || n < 1 || (inl && n > MULTI_INLINE) || (!inl && !dargs_dev)) return cudaErrorInvalidValue;
  const int cs = clusters_for(kShapes[k], W);
  return kShapes[k].launch(dargs_dev, inl, n, H, cs, st);
}

}  // namespace sc
