// The minimum-vertical-seam search (arXiv 2410.21207, section "DP Seam Carving": Algorithm 3 and
// the recurrence M(i,j) = e(i,j) + min(M(i-1,j-1), M(i-1,j), M(i-1,j+1)); the paper's "GPU" variant
// parallelises the j loop, this code does that and more) as a device function that one CTA, or
// every CTA of a thread-block cluster, calls together.
//
// Layout of the work
//   * Columns are split over the CTAs (CTA r owns [r*OWC, (r+1)*OWC)) and, inside a CTA, over
//     NW compute warps; a lane holds V = 4 consecutive columns of the current cost row in registers
//     and reads its neighbours' edge values with warp shuffles.
//   * Row-blocked trapezoidal tiles: a warp computes a window of 32*V columns (its strip of
//     Q = 32*V - 2*KT columns plus KT halo columns per side) for KT rows without talking to other
//     warps (the valid part shrinks by one column per row), then the strips' last rows are
//     exchanged through shared memory. One level up (clusters only), each CTA computes K2 halo
//     columns on either side of its own range and every K2 rows pushes its edge columns into the
//     neighbours' shared memory with st.async; there is no cluster-wide barrier in the row loop.
//   * A cost travels with an ancestor: key = (M << 8) | a, with a the column (in the warp's frame)
//     where the cell's optimal path crossed the top of the current super-tile of KSS rows (32; 64
//     for the single-map search of wide maps, whose chain hops cross CTAs through DSMEM). The
//     unsigned minimum of three keys is the minimum M and, among equal M, the smallest ancestor.
//     Optimal predecessors never cross under the leftmost tie-break (pred(j) <= pred(j+1): if
//     pred(j) = j+1 then M(j+1) < M(j), so j+1 cannot pick j), hence ancestors are non-decreasing
//     in the column and the smallest ancestor among tied candidates is the leftmost candidate's:
//     the key minimum carries exactly Algorithm 3's choice. The bottom row of each super-tile
//     records its ancestors; a chain of ceil(H/KSS) lookups gives the seam column at every
//     super-tile boundary, and then the super-tiles are backtracked in parallel by recomputing
//     their KSS rows in a 4*KSS-column window (KSS/8 columns per lane) from a saved cost row with
//     explicit directions.
//   * Energies are staged in shared memory by TMA: a producer warp issues one bulk copy per row
//     (one row per lane) into an NSLOT-slot ring, gated by full/empty mbarriers; a lane reads its 4
//     energies of a row with one 8-byte shared-memory load.
//   * The rows of a tile are branch-free (row 0 initialises from its energies; a ragged last tile
//     runs a counted loop), and per-super-tile bookkeeping runs after the tile, on its last row
//     (the only row of a tile where it can occur, since KSS is a multiple of KT).
// The result is Algorithm 3's seam exactly (leftmost ties, leftmost last-row minimum).
// With DIRECT the map is the caller's own H x W array (any row pitch that is a multiple of 8
// elements, 16-byte aligned rows), read in place: the row copies are clipped to the map's columns,
// the backtrack's loads outside it are skipped, and the 24-bit cost range is checked here instead
// of by a copy kernel (a per-row maximum of the staged energies, reduced over the cluster; a map
// that fails it is left to the wide-cost search through its gate).
// With FWD (forward energy) the map has three planes, CU, DL and DR, and a cell's cost depends on
// the direction it is reached from: M(i,j) = CU(i,j) + min(M(i-1,j-1) + DL(i,j), M(i-1,j),
// M(i-1,j+1) + DR(i,j)). Optimal predecessors still never cross (a crossing pair would need
// DL + DR < 0), so the ancestor keys keep their meaning; the planes are staged side by side.
#pragma once
#include <cooperative_groups.h>
#include <type_traits>

#include "sc_internal.cuh"
#include "sc_ptx.cuh"

namespace sc {

namespace cg = cooperative_groups;

constexpr uint32_t SENT = 0xFFFFFFFFu;   // excluded (outside the image): above every key
constexpr int FILL_WARPS_MAX = 8;        // warps that run backtrack fills
constexpr int NSLOT = 3;                 // energy staging ring: tiles in flight
constexpr size_t SEARCH_SMEM_LIMIT = 232448;   // opt-in dynamic shared memory per CTA

template <int NW, int KT, bool CL, int FWM = FILL_WARPS_MAX, int KSS = KS>
struct Geo {
  static constexpr int Q = 32 * V - 2 * KT;              // warp strip
  static constexpr int K2E = CL ? K2 : 0;                // CTA-level halo (clusters only)
  static constexpr int BW = NW * Q + 2 * KT;             // boundary / staged row width
  static constexpr int OWC = NW * Q - 2 * K2E;           // CTA-own columns
  static constexpr int FW = (NW + 1) < FWM ? (NW + 1) : FWM;   // backtrack-fill warps
  static constexpr int THREADS = (NW + 1) * 32;          // compute warps + the producer warp
  static constexpr int FV = KSS / 8;                     // backtrack-fill columns per lane
  static constexpr int FILLW = 32 * FV;                  // backtrack-fill window (4 * KSS columns)
  static_assert(Q > 0 && KSS % KT == 0 && K2 % KT == 0, "tile geometry");
  static_assert(KSS == 32 || KSS == 64, "super-tile height");
  static_assert(Q + 2 * KSS <= 256, "the ancestor frame must fit 8 bits");
};

// offsets of the dynamic shared-memory regions used by seam_search
struct SearchPlan {
  size_t bnd, hbuf, anc, wmin, cmin, jb, misc, emx, fdir, ring, bars, gat, total;
  int gw;   // row stride (bytes) of the gathered ancestor table in rank 0; 0: not gathered
};

template <int NW, int KT, bool CL, int FWM = FILL_WARPS_MAX, bool FWD = false, int KSS = KS, bool DIRECT = false>
__host__ __device__ inline SearchPlan search_plan(int S) {
  using G = Geo<NW, KT, CL, FWM, KSS>;
  SearchPlan p;
  size_t o = 0;
  p.bnd = o;  o += (size_t)2 * G::BW * 4;  o = (o + 15) & ~(size_t)15;
  p.hbuf = o; o += CL ? (size_t)2 * 2 * K2 * 4 : 0;
  p.anc = o;  o += (size_t)S * G::OWC;  o = (o + 15) & ~(size_t)15;
  p.wmin = o; o += (size_t)(NW + 1) * 8;
  p.cmin = o; o += CL ? (size_t)MAX_CLUSTER * 8 : 8;   // every CTA's minimum, pushed to rank 0
  p.jb = o;   o += (size_t)(S + 1) * 4;  o = (o + 15) & ~(size_t)15;
  p.misc = o; o += 16;
  p.emx = o;  o += DIRECT ? (size_t)(NW + 1 + MAX_CLUSTER) * 4 : 0;   // energy maxima: per warp, per CTA
  o = (o + 15) & ~(size_t)15;
  // the backtrack fill's direction rows live in the staging ring, which is idle by then (every
  // staged tile has been consumed before the argmin), unless the ring is the smaller of the two
  const size_t fdir_sz = (size_t)G::FW * KSS * 32 * (G::FV == 4 ? 4 : 2), ring_sz = (size_t)NSLOT * (FWD ? 3 : 1) * KT * G::BW * 2;
  if (fdir_sz > ring_sz) { p.fdir = o; o += fdir_sz;  o = (o + 15) & ~(size_t)15; }
  p.ring = o; o += ring_sz;  o = (o + 15) & ~(size_t)15;
  if (fdir_sz <= ring_sz) p.fdir = p.ring;
  p.bars = o; o += (size_t)(2 * NSLOT + 2) * 8;   // full[NSLOT], empty[NSLOT], halo[2]
  o = (o + 15) & ~(size_t)15;
  // single-map cluster search: every CTA writes its super-tile ancestors straight into rank 0's
  // table (remote stores during the row loop), so the chain after the argmin is all local loads;
  // only where the table fits
  p.gat = o;
  p.gw = 0;
  const size_t gat_sz = (size_t)S * MAX_CLUSTER * G::OWC;
  if (CL && FWM >= FILL_WARPS_MAX && o + gat_sz <= SEARCH_SMEM_LIMIT) {
    p.gw = MAX_CLUSTER * G::OWC;
    o += gat_sz;
  }
  p.total = (o + 15) & ~(size_t)15;
  return p;
}

struct SearchArgs {
  const uint16_t *E;   // row 0, column 0 (already offset by E_PADL unless DIRECT)
  int pitch_e;
  int H, W;
  uint32_t *Mrow;      // super-tile boundary cost rows, row s at Mrow + s*pitch_m (offset by E_PADL)
  int pitch_m = 0;     // row stride of Mrow (0: pitch_e)
  int *gate = nullptr; // DIRECT: receives ERR_ENERGY_RANGE when the map fails the 24-bit range check
  int32_t *seam;       // out [H]
  int32_t *seam_log;   // nullable, out [H]
  int64_t *cost;       // nullable, out [1]
  int *err;            // device error word
  bool gated;          // skip the search (energy range failure)
  int64_t pstride;     // forward energy: elements from one cost plane (CU, DL, DR) to the next
};

// Running counters of the mbarrier phases, identical in every thread of the CTA.
struct SearchState {
  uint32_t tiles = 0;  // tiles staged so far (ring slot and phase)
  uint32_t exch = 0;   // inter-CTA exchanges so far (halo buffer and phase)
};

__device__ __forceinline__ uint32_t min3u(uint32_t a, uint32_t b, uint32_t c) { return __vimin3_u32(a, b, c); }

// (uint16 pair) -> value << 8 for the low / high half
__device__ __forceinline__ uint32_t lo8(uint32_t x) { return __byte_perm(x, 0u, 0x4104); }
__device__ __forceinline__ uint32_t hi8(uint32_t x) { return __byte_perm(x, 0u, 0x4324); }

// Bookkeeping after row i (keys k of this lane's V columns, warp frame base fb):
//  - bottom of a super-tile: record the ancestors of the CTA-own columns (one byte: a - col + 128),
//    in rank 0's gathered table (row stride gw) when there is one, else in this CTA's table;
//  - last row before a super-tile: save the raw cost row for the backtrack fill;
//  - last row of the image: fold the lane's (M << 32 | column) minimum.
template <int KSS>
__device__ __forceinline__ void row_events(int i, const uint32_t (&k)[V], int H, int W, int c0, int fb, bool cta_own,
                                           int A, uint32_t *__restrict__ Mrow, int pitch_e,
                                           uint8_t *__restrict__ ancT, int OWC, uint8_t *gat, int gw,
                                           unsigned long long &lastmin) {
  if (!cta_own) return;
  if (((i + 1) % KSS == 0) || (i == H - 1)) {
    const uint32_t d = (uint32_t)(fb - c0 + 128);
    const uint32_t a = ((k[0] + d) & 0xFFu) | (((k[1] + d - 1u) & 0xFFu) << 8) | (((k[2] + d - 2u) & 0xFFu) << 16) |
                       (((k[3] + d - 3u) & 0xFFu) << 24);
    if (gw) *reinterpret_cast<uint32_t *>(gat + (size_t)(i / KSS) * gw + c0) = a;
    else *reinterpret_cast<uint32_t *>(ancT + (size_t)(i / KSS) * OWC + (c0 - A)) = a;
  }
  if (((i + 1) % KSS == 0) && (i + 1 < H)) {
    uint4 m;
    m.x = k[0] >> 8; m.y = k[1] >> 8; m.z = k[2] >> 8; m.w = k[3] >> 8;
    *reinterpret_cast<uint4 *>(Mrow + (size_t)((i + 1) / KSS) * pitch_e + c0) = m;
  }
  if (i == H - 1) {
#pragma unroll
    for (int u = 0; u < V; ++u) {
      if (c0 + u < W) {
        const unsigned long long c = ((unsigned long long)(k[u] >> 8) << 32) | (unsigned)(c0 + u);
        lastmin = c < lastmin ? c : lastmin;
      }
    }
  }
}

// key + energy, forced to SENT where the mask is SENT (outside the image). max(x + e, mask) equals
// (x + e) | mask for a mask of 0 or SENT, and the fused add-max keeps the mask off the row chain's
// critical path better than a separate OR.
template <bool MASK>
__device__ __forceinline__ uint32_t add_mask(uint32_t x, uint32_t e, uint32_t mask) {
  if (MASK) return __viaddmax_u32(x, e, mask);
  return x + e;
}

// One DP row for a lane: keys k (previous row) -> next row; energies ev (4 x uint16).
// LAT (a latency-bound search, one compute warp per SM sub-partition) takes, in warps without
// excluded columns, the instruction forms that shorten the row's dependent chain at the price of
// a few more instructions: the pairwise minima of the lane's own columns first (independent of
// the neighbours' shuffled values), then the neighbour and the energy in one add-min
// (min(a + e, b + e) = min(a, b) + e, exact: keys stay below 2^32 - e there). The
// throughput-bound kernels (several warps per sub-partition) and the masked warps keep the
// 3-input minimum.
template <bool MASK, bool LAT = false>
__device__ __forceinline__ void dp_row(uint32_t (&k)[V], uint2 ev, const uint32_t (&oobm)[V]) {
  const uint32_t e0 = lo8(ev.x), e1 = hi8(ev.x), e2 = lo8(ev.y), e3 = hi8(ev.y);
  const uint32_t L = __shfl_up_sync(0xffffffffu, k[V - 1], 1);
  const uint32_t R = __shfl_down_sync(0xffffffffu, k[0], 1);
  uint32_t n0, n1, n2, n3;
  if (LAT && !MASK) {
    const uint32_t p01 = min(k[0], k[1]), p23 = min(k[2], k[3]);
    n0 = __viaddmin_u32(L, e0, p01 + e0);
    n1 = __viaddmin_u32(k[2], e1, p01 + e1);
    n2 = __viaddmin_u32(k[1], e2, p23 + e2);
    n3 = __viaddmin_u32(R, e3, p23 + e3);
  } else {
    n0 = add_mask<MASK>(min3u(L, k[0], k[1]), e0, oobm[0]);
    n1 = add_mask<MASK>(min3u(k[0], k[1], k[2]), e1, oobm[1]);
    n2 = add_mask<MASK>(min3u(k[1], k[2], k[3]), e2, oobm[2]);
    n3 = add_mask<MASK>(min3u(k[2], k[3], R), e3, oobm[3]);
  }
  k[0] = n0; k[1] = n1; k[2] = n2; k[3] = n3;
}

// Running maximum of a lane's energies (two uint16 pairs; columns outside the map masked to 0 by
// cm in warps that hold such columns) for the DIRECT range check; off the row's dependent chain.
template <bool CHK, bool MASK>
__device__ __forceinline__ void emax_acc(uint32_t &acc, uint2 ev, uint2 cm) {
  if (CHK) acc = __vimax3_u16x2(acc, MASK ? (ev.x & cm.x) : ev.x, MASK ? (ev.y & cm.y) : ev.y);
}

// KT rows of a full tile from the staged energies er (row stride BW); MASK applies oobm.
template <int KT, int BW, bool MASK, bool LAT = false, bool CHK = false>
__device__ __forceinline__ void dp_rows(uint32_t (&k)[V], const uint16_t *er, const uint32_t (&oobm)[V],
                                        uint32_t &acc, uint2 cm) {
  uint2 a = *reinterpret_cast<const uint2 *>(er);
  uint2 b = *reinterpret_cast<const uint2 *>(er + BW);
#pragma unroll
  for (int r = 0; r < KT; ++r) {
    const uint2 ev = a;
    a = b;
    if (r + 2 < KT) b = *reinterpret_cast<const uint2 *>(er + (r + 2) * BW);
    dp_row<MASK, LAT>(k, ev, oobm);
    emax_acc<CHK, MASK>(acc, ev, cm);
  }
}

// Rows rb .. n-1 (n <= KT) of a tile: the first tile (rb = 1, row 0 initialises) or a ragged
// last tile, at the pace of a full tile.
template <int KT, int BW, bool MASK, bool LAT = false, bool CHK = false>
__device__ __forceinline__ void dp_rows_n(uint32_t (&k)[V], const uint16_t *er, const uint32_t (&oobm)[V], int rb,
                                          int n, uint32_t &acc, uint2 cm) {
  uint2 a = *reinterpret_cast<const uint2 *>(er + rb * BW);
  uint2 b = a;
  if (rb + 1 < n) b = *reinterpret_cast<const uint2 *>(er + (rb + 1) * BW);
#pragma unroll 2
  for (int r = rb; r < n; ++r) {
    const uint2 ev = a;
    a = b;
    if (r + 2 < n) b = *reinterpret_cast<const uint2 *>(er + (r + 2) * BW);
    dp_row<MASK, LAT>(k, ev, oobm);
    emax_acc<CHK, MASK>(acc, ev, cm);
  }
}

// One forward-energy row: keys k (previous row) -> next row; cu, dl, dr: 4 x uint16 each.
template <bool MASK>
__device__ __forceinline__ void dp_row_fwd(uint32_t (&k)[V], uint2 cu, uint2 dl, uint2 dr, const uint32_t (&oobm)[V]) {
  const uint32_t L = __shfl_up_sync(0xffffffffu, k[V - 1], 1);
  const uint32_t R = __shfl_down_sync(0xffffffffu, k[0], 1);
  const uint32_t n0 = add_mask<MASK>(min3u(L + lo8(dl.x), k[0], k[1] + lo8(dr.x)), lo8(cu.x), oobm[0]);
  const uint32_t n1 = add_mask<MASK>(min3u(k[0] + hi8(dl.x), k[1], k[2] + hi8(dr.x)), hi8(cu.x), oobm[1]);
  const uint32_t n2 = add_mask<MASK>(min3u(k[1] + lo8(dl.y), k[2], k[3] + lo8(dr.y)), lo8(cu.y), oobm[2]);
  const uint32_t n3 = add_mask<MASK>(min3u(k[2] + hi8(dl.y), k[3], R + hi8(dr.y)), hi8(cu.y), oobm[3]);
  k[0] = n0; k[1] = n1; k[2] = n2; k[3] = n3;
}

// KT forward-energy rows of a full tile; the three planes are KT rows apart in the staging ring.
template <int KT, int BW, bool MASK>
__device__ __forceinline__ void dp_rows_fwd(uint32_t (&k)[V], const uint16_t *er, const uint32_t (&oobm)[V]) {
  constexpr int PL = KT * BW;
  uint2 a0 = *reinterpret_cast<const uint2 *>(er), a1 = *reinterpret_cast<const uint2 *>(er + PL),
        a2 = *reinterpret_cast<const uint2 *>(er + 2 * PL);
#pragma unroll
  for (int r = 0; r < KT; ++r) {
    const uint2 c0 = a0, c1 = a1, c2 = a2;
    if (r + 1 < KT) {
      a0 = *reinterpret_cast<const uint2 *>(er + (r + 1) * BW);
      a1 = *reinterpret_cast<const uint2 *>(er + PL + (r + 1) * BW);
      a2 = *reinterpret_cast<const uint2 *>(er + 2 * PL + (r + 1) * BW);
    }
    dp_row_fwd<MASK>(k, c0, c1, c2, oobm);
  }
}

// Forward-energy rows rb .. n-1 (n <= KT) of a first or ragged last tile.
template <int KT, int BW, bool MASK>
__device__ __forceinline__ void dp_rows_n_fwd(uint32_t (&k)[V], const uint16_t *er, const uint32_t (&oobm)[V], int rb,
                                              int n) {
  constexpr int PL = KT * BW;
  for (int r = rb; r < n; ++r)
    dp_row_fwd<MASK>(k, *reinterpret_cast<const uint2 *>(er + r * BW),
                     *reinterpret_cast<const uint2 *>(er + PL + r * BW),
                     *reinterpret_cast<const uint2 *>(er + 2 * PL + r * BW), oobm);
}

// Initialise the staging and halo mbarriers (thread 0; the caller then synchronises the CTA, and
// the cluster when CL).
template <int NW, int KT, bool CL, int FWM = FILL_WARPS_MAX, bool FWD = false, int KSS = KS, bool DIRECT = false>
__device__ inline void search_init(unsigned char *smem, int S) {
  const SearchPlan plan = search_plan<NW, KT, CL, FWM, FWD, KSS, DIRECT>(S);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + plan.bars);
  uint64_t *empty = full + NSLOT;
  uint64_t *hbar = empty + NSLOT;
  if (threadIdx.x == 0) {
    for (int q = 0; q < NSLOT; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], NW);
    }
    mbar_init(&hbar[0], 1);
    mbar_init(&hbar[1], 1);
    fence_mbar_init();
  }
}

template <bool CL>
__device__ __forceinline__ void group_sync() {
  if (CL) cg::this_cluster().sync(); else __syncthreads();
}

// The search. Every thread of the CTA (of every CTA of the cluster when CL) calls it with the same
// arguments; `Smax` is the super-tile count the shared-memory plan was sized for.
// The parallel backtrack of seam_search: each fill warp recomputes its super-tiles (rows s*KSS ..
// s*KSS+KSS-1, s = warp*cs + rank, + FW*cs, ...) in a FILLW-column window from the saved cost row
// above them, with explicit directions, and walks them up from the chain's column at the bottom.
// A path cell r rows into a super-tile lies within KSS - 1 - r columns of the bottom column jb[s],
// and its three predecessors depend on the saved row only within KSS columns of jb[s]: the window
// [x0, x0 + FILLW) with x0 = jb[s] - FILLW / 2 (rounded down to FV) holds them all. Energies are
// read in chunks of CH rows, the next chunk loaded ahead of the current one's rows.
struct FillCtx {
  const uint16_t *E;
  const uint32_t *Mrow;
  const int *jb0;      // the chain's columns (rank 0's jb)
  uint16_t *fdir;      // direction rows of the fill warps
  int32_t *seam, *seam_log;
  int *err;
  int64_t pstride;
  int pitch_e, pitch_m, H, W, Wa, S, rank, cs;
  uint32_t best_m;     // the argmin's cost, checked against the recomputed one
};

template <int NW, int KT, bool CL, int FWM, bool FWD, int KSS, bool DIRECT, int CH>
__device__ __forceinline__ void backtrack_fill(const FillCtx &f, int warp, int lane) {
  using G = Geo<NW, KT, CL, FWM, KSS>;
  constexpr int NP = FWD ? 3 : 1;   // cost planes per row
  constexpr int FV = G::FV, FILLW = G::FILLW;
  // direction rows: 2 bits per column (FV = 8), or one byte per column (FV = 4: the walk then
  // reads its column's byte directly)
  using DirT = typename std::conditional<FV == 8, uint16_t, uint32_t>::type;
  using EVec = typename std::conditional<FV == 8, uint4, uint2>::type;        // FV uint16 energies
  constexpr int PST = 32 * (int)sizeof(DirT) / 4;   // 32-bit words per direction row
  DirT *fd = reinterpret_cast<DirT *>(f.fdir) + (size_t)warp * KSS * 32;
  const uint16_t *const Ef = f.E;
  int32_t *const seam_out = f.seam;
  int32_t *const seam_log = f.seam_log;
  int *const errw = f.err;
  const uint32_t *const Mrow = f.Mrow;
  const int *const jb0 = f.jb0;
  const int64_t pstride = f.pstride;
  const int pitch_e = f.pitch_e, pitch_m = f.pitch_m, H = f.H, W = f.W, Wa = f.Wa, S = f.S, rank = f.rank, cs = f.cs;
  const uint32_t best_m = f.best_m;
  // the energies of a super-tile's window (KSS rows, two rows per lane at most) are prefetched
  // into L2 one super-tile ahead: the map has usually left L2 since the DP pass read it. The
  // prefetch starts on a 16-byte boundary and covers the window.
  auto prefetch_window = [&](int s) {
    if (s >= S) return;
    int x0 = jb0[s] - FILLW / 2;
    x0 -= ((x0 % 8) + 8) % 8;
    int x1 = x0 + FILLW + 8;
    if (DIRECT) {   // only the caller's columns
      x0 = max(x0, 0);
      x1 = min(x1, Wa);
      if (x1 <= x0) return;
    }
    for (int i = s * KSS + lane; i < s * KSS + KSS && i < H; i += 32)
#pragma unroll
      for (int pl = 0; pl < NP; ++pl)
        bulk_prefetch_l2(Ef + pl * pstride + (size_t)i * pitch_e + x0, (uint32_t)(x1 - x0) * 2);
  };
  auto unpack = [](const EVec &v, uint32_t (&x)[FV]) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(&v);
#pragma unroll
    for (int q = 0; q < FV / 2; ++q) {
      x[2 * q] = w[q] & 0xFFFFu;
      x[2 * q + 1] = w[q] >> 16;
    }
  };
  prefetch_window(warp * cs + rank);
  for (int s = warp * cs + rank; s < S; s += G::FW * cs) {
    prefetch_window(s + G::FW * cs);
    const int jbs = jb0[s];
    const int jprev = (s > 0) ? jb0[s - 1] : jb0[S];
    int x0 = jbs - FILLW / 2;
    x0 -= ((x0 % FV) + FV) % FV;
    const int xc = x0 + lane * FV;
    const int rs = s * KSS, re = (rs + KSS < H) ? rs + KSS : H;
    const int first = (s == 0) ? 1 : rs;
    uint32_t m[FV], oob[FV];
#pragma unroll
    for (int u = 0; u < FV; ++u) oob[u] = (xc + u < 0 || xc + u >= W) ? SENT : 0u;
    // DIRECT: a lane's FV columns lie wholly inside or wholly outside the caller's [0, Wa)
    const bool xin = !DIRECT || (xc >= 0 && xc + FV <= Wa);
    if (s == 0) {
      EVec v0{};
      if (xin) v0 = *reinterpret_cast<const EVec *>(Ef + xc);
      unpack(v0, m);
    } else {
#pragma unroll
      for (int q = 0; q < FV / 4; ++q) {
        const uint4 a = *reinterpret_cast<const uint4 *>(Mrow + (size_t)s * pitch_m + xc + 4 * q);
        m[4 * q] = a.x; m[4 * q + 1] = a.y; m[4 * q + 2] = a.z; m[4 * q + 3] = a.w;
      }
    }
#pragma unroll
    for (int u = 0; u < FV; ++u) m[u] |= oob[u];
    // rows first..re-1 in chunks of CH rows, the next chunk's energies loaded ahead
    EVec eb0[NP][CH], eb1[NP][CH];
    auto load_chunk = [&](EVec (&eb)[NP][CH], int rbeg) {
#pragma unroll
      for (int r = 0; r < CH; ++r) {
        const int i = rbeg + r;
#pragma unroll
        for (int pl = 0; pl < NP; ++pl)
          if (i < re) {
            if (xin) eb[pl][r] = *reinterpret_cast<const EVec *>(Ef + pl * pstride + (size_t)i * pitch_e + xc);
            else eb[pl][r] = EVec{};
          }
      }
    };
    auto run_chunk = [&](const EVec (&eb)[NP][CH], int rbeg) {
#pragma unroll
      for (int r = 0; r < CH; ++r) {
        const int i = rbeg + r;
        if (i >= re) break;
        uint32_t ee[FV], dl[FV], dr[FV];
#pragma unroll
        for (int u = 0; u < FV; ++u) dl[u] = dr[u] = 0u;
        unpack(eb[0][r], ee);
        if (FWD) {
          unpack(eb[NP > 1 ? 1 : 0][r], dl);
          unpack(eb[NP > 2 ? 2 : 0][r], dr);
        }
        const uint32_t L = __shfl_up_sync(0xffffffffu, m[FV - 1], 1);
        const uint32_t R = __shfl_down_sync(0xffffffffu, m[0], 1);
        uint32_t nm[FV];
        uint32_t dirs = 0;
#pragma unroll
        for (int u = 0; u < FV; ++u) {
          const uint32_t a = ((u == 0) ? L : m[u - 1]) + dl[u];
          const uint32_t b = m[u];
          const uint32_t c = ((u == FV - 1) ? R : m[u + 1]) + dr[u];
          const uint32_t mn = min3u(a, b, c);
          const uint32_t dd = (a == mn) ? 0u : ((b == mn) ? 1u : 2u);
          dirs |= dd << ((FV == 4 ? 8 : 2) * u);
          nm[u] = add_mask<true>(mn, ee[u], oob[u]);
        }
#pragma unroll
        for (int u = 0; u < FV; ++u) m[u] = nm[u];
        fd[(i - rs) * 32 + lane] = (DirT)dirs;
      }
    };
    int rb = first;
    load_chunk(eb0, rb);
    while (rb < re) {
      if (rb + CH < re) load_chunk(eb1, rb + CH);
      run_chunk(eb0, rb);
      rb += CH;
      if (rb >= re) break;
      if (rb + CH < re) load_chunk(eb0, rb + CH);
      run_chunk(eb1, rb);
      rb += CH;
    }
    if (s == S - 1) {
      // the recomputed cost at the bottom of the seam must be the argmin's
      const int rel = jbs - x0;
      if (rel / FV == lane) {
        uint32_t v = 0;
#pragma unroll
        for (int u = 0; u < FV; ++u) if (u == rel % FV) v = m[u];
        if (v != best_m) atomicOr(errw, ERR_COST_MISMATCH);
      }
    }
    __syncwarp();
    // lane 0 follows the directions up the window (relative columns, kept in the direction rows it
    // has read: a row's entry is not needed again), then the warp writes the seam rows
    uint32_t *path = reinterpret_cast<uint32_t *>(fd);   // path[(i - rs) * PST] holds the column of row i
    if (lane == 0) {
      int rel = jbs - x0;
      bool okp = true;
      if constexpr (FV == 4) {
        // one byte per column; a step leaving the window is clamped (every read stays in this
        // warp's rows) and recorded as a failure
        const uint8_t *fb = reinterpret_cast<const uint8_t *>(fd) + (size_t)(re - 1 - rs) * FILLW;
        for (int i = re - 1; i >= first; --i, fb -= FILLW) {
          const int nr = rel + (int)fb[rel] - 1;
          path[(i - rs) * PST] = (uint32_t)rel;   // the first 4 bytes of row i's direction words
          okp &= (unsigned)nr < (unsigned)FILLW;
          rel = min(max(nr, 0), FILLW - 1);
        }
      } else {
        for (int i = re - 1; i >= first; --i) {
          if (rel < 0 || rel >= FILLW) { okp = false; break; }
          const uint32_t dd = ((uint32_t)fd[(i - rs) * 32 + rel / FV] >> (2 * (rel % FV))) & 3u;
          path[(i - rs) * PST] = (uint32_t)rel;   // the first 4 bytes of row i's direction words
          rel += (int)dd - 1;
        }
      }
      if (!okp) {
        atomicOr(errw, ERR_FILL_MISMATCH);
        rel = -1 - x0;
      }
      path[KSS * PST - 1] = (uint32_t)rel;    // the column above row `first` (row 0's seam when s == 0)
      if (x0 + rel != jprev) atomicOr(errw, ERR_FILL_MISMATCH);
    }
    __syncwarp();
    const bool path_ok = (int)path[KSS * PST - 1] + x0 >= 0;
    if (path_ok) {
      for (int i = first + lane; i < re; i += 32) {
        const int j = x0 + (int)path[(i - rs) * PST];
        seam_out[i] = j;
        if (seam_log) seam_log[i] = j;
      }
      if (s == 0 && lane == 0) {
        const int j = x0 + (int)path[KSS * PST - 1];
        seam_out[0] = j;
        if (seam_log) seam_log[0] = j;
      }
    }
    __syncwarp();
  }
}

// backtrack_fill as a function of its own (not inlined): it gets its own register allocation, so
// the one-CTA batched kernel, whose 512 threads have at most 128 registers each, can load deeper
// energy chunks
template <int NW, int KT, bool CL, int FWM, bool FWD, int KSS, bool DIRECT, int CH>
static __device__ __noinline__ void backtrack_fill_call(FillCtx f, int warp, int lane) {
  backtrack_fill<NW, KT, CL, FWM, FWD, KSS, DIRECT, CH>(f, warp, lane);
}

template <int NW, int KT, bool CL, int FWM = FILL_WARPS_MAX, bool FWD = false, int KSS = KS, bool DIRECT = false>
__device__ void seam_search(const SearchArgs &p, unsigned char *smem, int Smax, SearchState &st) {
  static_assert(!DIRECT || (CL && !FWD), "the in-place form is built for the cluster search of e1 maps");
  constexpr int NP = FWD ? 3 : 1;   // cost planes staged per row
  // the single-map search: one cluster, a CTA per SM, every compute warp alone on its SM
  // sub-partition with 4 warps (latency-bound)
  constexpr bool LAT = CL && FWM >= FILL_WARPS_MAX && NW == 4;
  using G = Geo<NW, KT, CL, FWM, KSS>;
  constexpr int Q = G::Q, BW = G::BW, OWC = G::OWC, K2E = G::K2E;
  const int rank = CL ? (int)cg::this_cluster().block_rank() : 0;
  const int cs = CL ? (int)cg::this_cluster().num_blocks() : 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool producer = (warp == NW);
  const int H = p.H, W = p.W;
  const int S = (H + KSS - 1) / KSS;
  const SearchPlan plan = search_plan<NW, KT, CL, FWM, FWD, KSS, DIRECT>(Smax);
  uint32_t *bnd = reinterpret_cast<uint32_t *>(smem + plan.bnd);
  uint32_t *hbuf = reinterpret_cast<uint32_t *>(smem + plan.hbuf);
  uint8_t *ancT = reinterpret_cast<uint8_t *>(smem + plan.anc);
  unsigned long long *wmin = reinterpret_cast<unsigned long long *>(smem + plan.wmin);
  unsigned long long *cmin = reinterpret_cast<unsigned long long *>(smem + plan.cmin);
  int *jb = reinterpret_cast<int *>(smem + plan.jb);
  int *misc = reinterpret_cast<int *>(smem + plan.misc);
  uint32_t *emx = reinterpret_cast<uint32_t *>(smem + plan.emx);   // DIRECT: [NW + 1] per warp, then per CTA
  uint16_t *fdir = reinterpret_cast<uint16_t *>(smem + plan.fdir);
  uint16_t *ring = reinterpret_cast<uint16_t *>(smem + plan.ring);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + plan.bars);
  uint64_t *empty = full + NSLOT;
  uint64_t *hbar = empty + NSLOT;
  const int gw = plan.gw;
  uint8_t *const gat = smem + plan.gat;
  uint8_t *const gat0 = (CL && gw) ? cg::this_cluster().map_shared_rank(gat, 0) : gat;

  // geometry
  const int A = rank * OWC, B = A + OWC;
  const int ext0 = A - K2E;                     // extended range start
  const int own0 = ext0 + warp * Q;             // warp strip start
  const int c0 = own0 - KT + lane * V;          // this lane's first column
  const int frame_base = own0 - KSS;            // ancestor frame of this warp
  const bool strip_lane = !producer && (lane * V >= KT) && (lane * V < KT + Q);
  const bool cta_own = strip_lane && c0 >= A && c0 < B;   // A, B, c0 are multiples of 4
  uint32_t oobm[V];
#pragma unroll
  for (int u = 0; u < V; ++u) oobm[u] = (c0 + u < 0 || c0 + u >= W) ? SENT : 0u;
  const bool edge = __any_sync(0xffffffffu, (oobm[0] | oobm[V - 1]) != 0u);
  const int bidx0 = c0 - (ext0 - KT);           // index of c0 in bnd and in a staged energy row

  unsigned long long lastmin = ~0ull;
  const int nt = p.gated ? 0 : (H + KT - 1) / KT;
  // single CTA: only the warps whose strips reach into [0, W) compute, and only their columns are
  // staged (a cluster is sized to W, so all its warps work)
  const int nwa = CL ? NW : min(NW, (W + Q - 1) / Q);
  const bool active = warp < nwa;
  const uint32_t ROW_BYTES = CL ? (uint32_t)BW * 2 : (uint32_t)(nwa * Q + 2 * KT) * 2;
  // fields used inside the loops, held in registers (stores through the map pointers could
  // otherwise force reloads of the argument struct)
  const int pitch_e = p.pitch_e;
  const int pitch_m = p.pitch_m ? p.pitch_m : p.pitch_e;
  const int64_t pstride = FWD ? p.pstride : 0;
  uint32_t *const Mrow = p.Mrow;
  // DIRECT: the columns that exist in the caller's array, [0, Wa); rows are copied only there
  const int Wa = (W + 7) & ~7;
  const int cbeg = ext0 - KT;   // first staged column (a multiple of 8)
  const int clo = DIRECT ? max(cbeg, 0) : cbeg;
  const int chi = DIRECT ? min(cbeg + (int)(ROW_BYTES / 2), Wa) : cbeg + (int)(ROW_BYTES / 2);
  const uint32_t COPY_BYTES = (uint32_t)(chi - clo) * 2;

  if (producer) {
    // ---- energy staging: rows of columns [ext0 - KT, ext0 - KT + BW), one bulk copy per lane ----
    const uint16_t *Estage = p.E + (ext0 - KT);
    for (int tt = 0; tt < nt; ++tt) {
      const uint32_t g = st.tiles + tt;
      const int slot = (int)(g % NSLOT);
      if (g >= NSLOT && !mbar_wait_bounded(&empty[slot], ((g / NSLOT) - 1) & 1u, WAIT_TIMEOUT_NS)) {
        if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
      }
      const int rbeg = tt * KT;
      const int nrows = (H - rbeg < KT) ? H - rbeg : KT;
      if (lane == 0) mbar_arrive_expect_tx(&full[slot], (uint32_t)(NP * nrows) * COPY_BYTES);
      __syncwarp();
      if (lane < nrows) {
#pragma unroll
        for (int pl = 0; pl < NP; ++pl)
          bulk_g2s(ring + (size_t)((slot * NP + pl) * KT + lane) * BW + (clo - cbeg),
                   Estage + pl * pstride + (size_t)(rbeg + lane) * pitch_e + (clo - cbeg), COPY_BYTES, &full[slot]);
      }
    }
  } else if (!active) {
    // outside the image: release every slot at once and keep the barrier count
    for (int t = 0; t < nt; ++t) {
      const uint32_t g = st.tiles + t;
      if (lane == 0) mbar_arrive(&empty[g % NSLOT]);
      if (t * KT + KT < H) named_bar_sync(NW * 32);
    }
  } else {
    uint32_t k[V] = {0u, 0u, 0u, 0u};
    uint32_t emax = 0u;   // DIRECT: running maximum of this lane's in-map energies (two uint16 halves)
    const uint2 cm = make_uint2((oobm[0] ? 0u : 0xFFFFu) | (oobm[1] ? 0u : 0xFFFF0000u),
                                (oobm[2] ? 0u : 0xFFFFu) | (oobm[3] ? 0u : 0xFFFF0000u));
    // The tile loop, compiled twice: EDGE warps hold columns outside the image and apply the
    // exclusion mask on every row; the others never test it.
    auto tiles = [&](auto edge_tag) {
      constexpr bool EDGE = decltype(edge_tag)::value;
      const uint32_t own_a = (uint32_t)(c0 - frame_base);   // this lane's first column, warp frame
      for (int t = 0; t < nt; ++t) {
        const int r0 = t * KT;
        const bool more = r0 + KT < H;
        const uint32_t g = st.tiles + t;
        const int slot = (int)(g % NSLOT);
        // one barrier test per tile: the tile was issued NSLOT - 1 tiles ago and has landed by now
        // (an earlier test of the next tile, overlapped with this tile's rows, found it still in
        // flight every time and cost more than it saved)
        if (!mbar_wait_bounded(&full[slot], (g / NSLOT) & 1u, WAIT_TIMEOUT_NS)) {
          if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
        }
        const uint16_t *er = ring + (size_t)slot * NP * KT * BW + bidx0;
        if (t > 0) {
          // window of the previous row from the boundary buffer (relative ancestors -> warp frame).
          // At a new super-tile every cell becomes its own ancestor; the old ancestor field is
          // dropped without arithmetic (it may lie outside this warp's frame).
          const uint4 v = *reinterpret_cast<const uint4 *>(bnd + ((t - 1) & 1) * BW + bidx0);
          const bool fresh = (r0 % KSS) == 0;
          const uint32_t d = own_a - 128u;
          k[0] = fresh ? ((v.x & ~0xFFu) | own_a) : (v.x + d);
          k[1] = fresh ? ((v.y & ~0xFFu) | (own_a + 1u)) : (v.y + d + 1u);
          k[2] = fresh ? ((v.z & ~0xFFu) | (own_a + 2u)) : (v.z + d + 2u);
          k[3] = fresh ? ((v.w & ~0xFFu) | (own_a + 3u)) : (v.w + d + 3u);
          if (EDGE) { k[0] |= oobm[0]; k[1] |= oobm[1]; k[2] |= oobm[2]; k[3] |= oobm[3]; }
        }
        if (t > 0 && r0 + KT <= H) {
          // full tile: KT branch-free rows (the energies of the next rows are loaded ahead of
          // the row that needs them, off the dependent chain); bookkeeping only where a
          // super-tile or the image ends on its last row
          if (FWD) dp_rows_fwd<KT, BW, EDGE>(k, er, oobm);
          else dp_rows<KT, BW, EDGE, LAT, DIRECT>(k, er, oobm, emax, cm);
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[slot]);   // this warp is done with the staged rows
          if (((r0 + KT) % KSS) == 0 || r0 + KT == H)
            row_events<KSS>(r0 + KT - 1, k, H, W, c0, frame_base, cta_own, A, Mrow, pitch_m, ancT, OWC, gat0, gw, lastmin);
        } else {
          // first tile (row 0 has no predecessor) or a ragged last tile. Neither holds a row with
          // bookkeeping except the image's last row and the first tile's last row when KSS = KT:
          // a super-tile ends on a multiple of KSS (a multiple of KT), which is never inside
          // these tiles' rows 0 .. n-2
          const int n = (H - r0 < KT) ? H - r0 : KT;
          if (t == 0) {
            const uint2 ev = *reinterpret_cast<const uint2 *>(er);   // CU with FWD
            k[0] = (lo8(ev.x) | own_a) | oobm[0];
            k[1] = (hi8(ev.x) | (own_a + 1u)) | oobm[1];
            k[2] = (lo8(ev.y) | (own_a + 2u)) | oobm[2];
            k[3] = (hi8(ev.y) | (own_a + 3u)) | oobm[3];
            emax_acc<DIRECT, EDGE>(emax, ev, cm);
          }
          if (FWD) dp_rows_n_fwd<KT, BW, EDGE>(k, er, oobm, t == 0 ? 1 : 0, n);
          else dp_rows_n<KT, BW, EDGE, LAT, DIRECT>(k, er, oobm, t == 0 ? 1 : 0, n, emax, cm);
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[slot]);
          if (((r0 + n) % KSS) == 0 || r0 + n == H)
            row_events<KSS>(r0 + n - 1, k, H, W, c0, frame_base, cta_own, A, Mrow, pitch_m, ancT, OWC, gat0, gw, lastmin);
        }
        if (more) {
          const bool exch = CL && ((r0 + KT) % K2 == 0) && cs > 1;
          const uint32_t d = own_a - 128u;
          uint4 v;
          v.x = k[0] - d; v.y = k[1] - d - 1u; v.z = k[2] - d - 2u; v.w = k[3] - d - 3u;
          // publish this warp's strip (relative ancestor encoding); at an exchange the CTA's halo
          // columns come from the neighbours instead
          if (strip_lane && (!exch || (c0 >= A && c0 < B)))
            *reinterpret_cast<uint4 *>(bnd + (t & 1) * BW + bidx0) = v;
          if constexpr (CL) if (exch) {
            const uint32_t xg = st.exch + (uint32_t)((r0 + KT) / K2 - 1);
            const int par = (int)(xg & 1);
            // my first K2 own columns are the left neighbour's right halo, my last K2 the right's left
            if (strip_lane && rank > 0 && c0 >= A && c0 < A + K2)
              st_async_v4(mapa_u32(hbuf + par * 2 * K2 + K2 + (c0 - A), rank - 1), v, mapa_u32(&hbar[par], rank - 1));
            if (strip_lane && rank < cs - 1 && c0 >= B - K2 && c0 < B)
              st_async_v4(mapa_u32(hbuf + par * 2 * K2 + (c0 - (B - K2)), rank + 1), v, mapa_u32(&hbar[par], rank + 1));
            if (threadIdx.x == 0)
              mbar_arrive_expect_tx(&hbar[par], (uint32_t)(((rank > 0) + (rank < cs - 1)) * K2 * 4));
            if (!mbar_wait_bounded(&hbar[par], (xg >> 1) & 1u, WAIT_TIMEOUT_NS)) {
              if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
            }
            uint32_t *mine = bnd + (t & 1) * BW;
            for (int q = threadIdx.x; q < 2 * K2; q += NW * 32) {
              if (q < K2) {
                if (rank > 0) mine[(A - K2 + q) - (ext0 - KT)] = hbuf[par * 2 * K2 + q];
              } else {
                if (rank < cs - 1) mine[(B + (q - K2)) - (ext0 - KT)] = hbuf[par * 2 * K2 + q];
              }
            }
          }
          named_bar_sync(NW * 32);
        }
      }
    };
    if (edge) tiles(std::integral_constant<bool, true>());
    else tiles(std::integral_constant<bool, false>());
    if (DIRECT) {
      const uint32_t m = __reduce_max_sync(0xffffffffu, max(emax & 0xFFFFu, emax >> 16));
      if (lane == 0) emx[warp] = m;
    }
  }
  if (DIRECT && lane == 0 && (producer || !active)) emx[warp] = 0u;
  st.tiles += (uint32_t)nt;
  if (CL && nt > 0) st.exch += (uint32_t)((cs > 1) ? ((H - 1) / K2) : 0);

  // ---- last-row argmin: the leftmost minimum (min of (M << 32) | column) ----
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, lastmin, off);
    lastmin = o < lastmin ? o : lastmin;
  }
  if (lane == 0) wmin[warp] = lastmin;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = ~0ull;
    for (int w = 0; w <= NW; ++w) m = wmin[w] < m ? wmin[w] : m;
    if (CL) cg::this_cluster().map_shared_rank(cmin, 0)[rank] = m;   // pushed to rank 0
    else cmin[0] = m;
    if (DIRECT) {
      uint32_t e = 0u;
      for (int w = 0; w <= NW; ++w) e = max(e, emx[w]);
      cg::this_cluster().map_shared_rank(emx, 0)[NW + 1 + rank] = e;
    }
  }
  group_sync<CL>();

  // ---- ancestor chain (rank 0, one thread): seam column at every super-tile bottom ----
  if (rank == 0 && threadIdx.x == 0) {
    int ok = !p.gated;
    unsigned long long best = ~0ull;
    for (int r = 0; r < cs; ++r) best = cmin[r] < best ? cmin[r] : best;
    if (DIRECT && ok) {
      // the 24-bit keys hold the seam sums only while H * max(e) < 2^24; otherwise this result is
      // void and the wide-cost search, launched next, takes the map
      uint32_t e = 0u;
      for (int r = 0; r < cs; ++r) e = max(e, emx[NW + 1 + r]);
      if ((uint64_t)e * (uint64_t)H >= ((uint64_t)1 << 24)) {
        ok = 0;
        if (p.gate) atomicOr(p.gate, ERR_ENERGY_RANGE);
      }
    }
    int j = (int)(best & 0xFFFFFFFFull);
    if (ok && (j < 0 || j >= W)) { ok = 0; atomicOr(p.err, ERR_BAD_SEAM); }
    if (ok && gw) {
      // branch-free hops: a column outside the map is clamped (every table read stays inside
      // the table) and recorded as a failure
      bool bad = false;
      for (int s = S - 1; s >= 0; --s) {
        jb[s] = j;
        const int nj = j + (int)gat[(size_t)s * gw + j] - 128;
        bad |= (unsigned)nj >= (unsigned)W;
        j = min(max(nj, 0), W - 1);
      }
      if (bad) { ok = 0; atomicOr(p.err, ERR_BAD_SEAM); }
    }
    for (int s = S - 1; ok && !gw && s >= 0; --s) {
      jb[s] = j;
      const int c = j / OWC;
      if (c < 0 || c >= cs) { ok = 0; atomicOr(p.err, ERR_BAD_SEAM); break; }
      const uint8_t *ra = CL ? cg::this_cluster().map_shared_rank(ancT, c) : ancT;
      j = j + (int)ra[(size_t)s * OWC + (j - c * OWC)] - 128;
      if (j < 0 || j >= W) { ok = 0; atomicOr(p.err, ERR_BAD_SEAM); }
    }
    jb[S] = j;          // the seam's column in row 0
    misc[0] = ok;
    misc[1] = (int)(best >> 32);
    if (ok && p.cost) *p.cost = (int64_t)(best >> 32);
  }
  group_sync<CL>();

  // ---- parallel backtrack: each super-tile recomputed in a FILLW-column window ----
  const int *jb0 = CL ? cg::this_cluster().map_shared_rank(jb, 0) : jb;
  const int *misc0 = CL ? cg::this_cluster().map_shared_rank(misc, 0) : misc;
  const int ok = misc0[0];
  const uint32_t best_m = (uint32_t)misc0[1];
  if (ok && warp < G::FW) {
    const FillCtx f{p.E, Mrow, jb0, fdir, p.seam, p.seam_log, p.err, pstride, pitch_e, pitch_m, H, W, Wa, S, rank, cs,
                    best_m};
    // energy chunks: the single-map search (all fill warps, one CTA per SM, latency-bound) has
    // registers to spare for chunks whose compute covers an L2 round trip (16 rows of 4 columns per
    // lane, 8 rows of 8); the multi-map and cluster batched kernels, whose latency other CTAs hide
    // and whose registers are capped, use 4- or 2-row chunks; the one-CTA batched kernel calls the
    // fill as a function of its own, with 4-row chunks (config 4: 46.9 -> 45.3 ms; the same call in
    // the cluster batched kernel made its largest image 37.1 -> 46.1 ms, so that one stays inline).
    constexpr int FV = G::FV;
    if constexpr (!CL && !FWD) {
      backtrack_fill_call<NW, KT, CL, FWM, FWD, KSS, DIRECT, 4>(f, warp, lane);
    } else {
      constexpr int CH = FWD ? 2 : ((CL && FWM >= FILL_WARPS_MAX) ? (FV == 4 ? 16 : 8) : (CL && FV == 4 ? 4 : 2));
      backtrack_fill<NW, KT, CL, FWM, FWD, KSS, DIRECT, CH>(f, warp, lane);
    }
  }
  group_sync<CL>();   // rank 0's shared memory is read above; the seam is complete after this
}

}  // namespace sc
