// Minimum vertical seam on one GB300 thread-block cluster (arXiv 2410.21207, section "DP Seam
// Carving": Algorithm 3 and the recurrence M(i,j) = e(i,j) + min(M(i-1,j-1), M(i-1,j), M(i-1,j+1));
// the paper's "GPU" variant runs the j loop in parallel, this kernel does that and more).
//
// Layout of the work
//   * The columns are split over the CTAs of one cluster (CTA r owns [r*OW, (r+1)*OW)) and,
//     inside a CTA, over warps; a lane holds V = 4 consecutive columns of the current cost row in
//     registers and reads its neighbours' edge values with warp shuffles.
//   * Row-blocked trapezoidal tiles: a warp computes a window of 32*V columns, its own strip of
//     Q columns plus KT halo columns on each side, for KT rows without talking to other warps (the
//     halo shrinks by one column per row), then the strips' last rows are exchanged through shared
//     memory. The same idea one level up: each CTA computes K2 halo columns on either side of its
//     own range and the CTAs exchange edge columns through distributed shared memory every K2 rows
//     (one cluster barrier per K2 rows instead of one per row).
//   * A cost value travels with an ancestor: key = (M << 8) | a, with a the column (relative to
//     the warp's frame) where the cell's optimal path crossed the top of the current super-tile of
//     KS rows. Taking the unsigned minimum of three keys gives the minimum M and, among equal M, the
//     smallest ancestor; because optimal predecessors never cross (pred(j) <= pred(j+1) under the
//     leftmost tie-break), the smallest ancestor among tied candidates is the ancestor of the
//     leftmost one, so the key minimum carries exactly Algorithm 3's choice. The last row of each
//     super-tile records the ancestors; a chain of ceil(H/KS) lookups then gives the seam column at
//     every super-tile boundary, and the super-tiles are backtracked in parallel by recomputing
//     their KS rows in a 256-column window from a saved cost row (leftmost tie-break, explicit
//     directions).
//   * Energies are staged in shared memory by TMA: one thread issues a bulk copy per row of the
//     CTA's columns two tiles ahead into a three-slot ring (mbarrier completion, bounded waits);
//     a lane reads its 4 energies of a row with one 8-byte shared-memory load.
//   * The row loop of a full tile is branch-free (16 rows unrolled); the first tile (row 0) and
//     a ragged last tile take a general path, and the per-super-tile bookkeeping runs after the
//     tile, on its last row, which is the only row of a full tile where it can occur.
// The result is Algorithm 3's seam exactly (leftmost ties, leftmost last-row minimum).
#include <cooperative_groups.h>

#include "sc_internal.cuh"
#include "sc_ptx.cuh"

namespace cg = cooperative_groups;

namespace sc {

constexpr uint32_t SENT = 0xFFFFFFFFu;   // excluded (outside the image) — larger than any key
constexpr int FILL_W = 256;              // fill window (8 columns per lane)

template <int NW>
struct DpSmem {
  static constexpr int BW = NW * Q + 2 * KT;     // boundary row: extended range + window pads
  static constexpr int OWC = NW * Q - 2 * K2;    // CTA-own columns
};

DpShape dp_shape_for(int W) {
  DpShape s;
  s.nw = 4;
  s.ow = 4 * Q - 2 * K2;
  s.cs = (W + s.ow - 1) / s.ow;
  if (s.cs > MAX_CLUSTER) {
    s.nw = 8;
    s.ow = 8 * Q - 2 * K2;
    s.cs = (W + s.ow - 1) / s.ow;
  }
  if (s.cs < 1) s.cs = 1;
  return s;
}

// offsets of the dynamic shared-memory regions
constexpr int NSLOT = 3;   // energy staging ring: tiles in flight

struct SmemPlan {
  size_t bnd, hbuf, anc, wmin, cmin, jb, misc, fdir, ring, bars, total;
};
// bars: full[NSLOT], empty[NSLOT], halo[2]  (uint64 mbarriers)
static __host__ __device__ SmemPlan smem_plan(int nw, int S) {
  SmemPlan p;
  const int BW = nw * Q + 2 * KT, OWC = nw * Q - 2 * K2;
  const int nwarps = nw + 1;   // compute warps + the energy producer warp
  size_t o = 0;
  p.bnd = o;  o += (size_t)2 * BW * 4;  o = (o + 15) & ~(size_t)15;
  p.hbuf = o; o += (size_t)2 * 2 * K2 * 4;
  p.anc = o;  o += (size_t)S * OWC;  o = (o + 15) & ~(size_t)15;
  p.wmin = o; o += (size_t)nwarps * 8;
  p.cmin = o; o += 8;
  p.jb = o;   o += (size_t)(S + 1) * 4;  o = (o + 15) & ~(size_t)15;
  p.misc = o; o += 16;
  p.fdir = o; o += (size_t)nwarps * KS * 32 * 2;  o = (o + 15) & ~(size_t)15;
  p.ring = o; o += (size_t)NSLOT * KT * BW * 2;  o = (o + 15) & ~(size_t)15;
  p.bars = o; o += (size_t)(2 * NSLOT + 2) * 8;
  p.total = (o + 15) & ~(size_t)15;
  return p;
}

size_t dp_smem_bytes(int nw, int H) { return smem_plan(nw, (H + KS - 1) / KS).total; }

__device__ __forceinline__ uint32_t min3u(uint32_t a, uint32_t b, uint32_t c) { return __vimin3_u32(a, b, c); }

// (uint16 pair) -> value << 8 for the low / high half
__device__ __forceinline__ uint32_t lo8(uint32_t x) { return __byte_perm(x, 0u, 0x4104); }
__device__ __forceinline__ uint32_t hi8(uint32_t x) { return __byte_perm(x, 0u, 0x4324); }

// Bookkeeping after row i (keys k of this lane's V columns, warp frame base `fb`):
//  - bottom of a super-tile: record the ancestors (absolute columns) of the CTA-own columns;
//  - last row before a super-tile: save the raw cost row for the backtrack fill;
//  - last row of the image: fold the lane's (M << 32 | column) minimum.
__device__ __forceinline__ void row_events(int i, const uint32_t (&k)[V], int H, int W, int c0, int fb, bool cta_own,
                                           int A, uint32_t *__restrict__ Mrow, int pitch_e,
                                           uint8_t *__restrict__ ancT, int OWC, unsigned long long &lastmin) {
  if (!cta_own) return;
  if (((i + 1) % KS == 0) || (i == H - 1)) {
    // ancestor - column + 128, one byte per column (|ancestor - column| <= KS)
    const uint32_t d = (uint32_t)(fb - c0 + 128);
    const uint32_t a = ((k[0] + d) & 0xFFu) | (((k[1] + d - 1u) & 0xFFu) << 8) | (((k[2] + d - 2u) & 0xFFu) << 16) |
                       (((k[3] + d - 3u) & 0xFFu) << 24);
    *reinterpret_cast<uint32_t *>(ancT + (size_t)(i / KS) * OWC + (c0 - A)) = a;
  }
  if (((i + 1) % KS == 0) && (i + 1 < H)) {
    uint4 m;
    m.x = k[0] >> 8; m.y = k[1] >> 8; m.z = k[2] >> 8; m.w = k[3] >> 8;
    *reinterpret_cast<uint4 *>(Mrow + (size_t)((i + 1) / KS) * pitch_e + c0) = m;
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

// One DP row for a lane: keys k (previous row) -> next row, energies ev (4 x uint16).
__device__ __forceinline__ void dp_row(uint32_t (&k)[V], uint2 ev, const uint32_t (&oobm)[V]) {
  const uint32_t e0 = lo8(ev.x), e1 = hi8(ev.x), e2 = lo8(ev.y), e3 = hi8(ev.y);
  const uint32_t L = __shfl_up_sync(0xffffffffu, k[V - 1], 1);
  const uint32_t R = __shfl_down_sync(0xffffffffu, k[0], 1);
  const uint32_t n0 = (min3u(L, k[0], k[1]) + e0) | oobm[0];
  const uint32_t n1 = (min3u(k[0], k[1], k[2]) + e1) | oobm[1];
  const uint32_t n2 = (min3u(k[1], k[2], k[3]) + e2) | oobm[2];
  const uint32_t n3 = (min3u(k[2], k[3], R) + e3) | oobm[3];
  k[0] = n0; k[1] = n1; k[2] = n2; k[3] = n3;
}

template <int NW>
__global__ void __launch_bounds__((NW + 1) * 32, 1) k_dp(DpArgs p) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int cs = (int)cl.num_blocks();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool producer = (warp == NW);           // the last warp only stages energies
  const int H = p.H, W = p.W;
  const int S = (H + KS - 1) / KS;
  constexpr int BW = DpSmem<NW>::BW, OWC = DpSmem<NW>::OWC;
  const SmemPlan plan = smem_plan(NW, S);
  uint32_t *bnd = reinterpret_cast<uint32_t *>(smem + plan.bnd);
  uint32_t *hbuf = reinterpret_cast<uint32_t *>(smem + plan.hbuf);
  uint8_t *ancT = reinterpret_cast<uint8_t *>(smem + plan.anc);
  unsigned long long *wmin = reinterpret_cast<unsigned long long *>(smem + plan.wmin);
  unsigned long long *cmin = reinterpret_cast<unsigned long long *>(smem + plan.cmin);
  int *jb = reinterpret_cast<int *>(smem + plan.jb);
  int *misc = reinterpret_cast<int *>(smem + plan.misc);
  uint16_t *fdir = reinterpret_cast<uint16_t *>(smem + plan.fdir);
  uint16_t *ring = reinterpret_cast<uint16_t *>(smem + plan.ring);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + plan.bars);
  uint64_t *empty = full + NSLOT;
  uint64_t *hbar = empty + NSLOT;

  const bool gated = (p.gate != nullptr) && (*p.gate & ERR_ENERGY_RANGE);

  // geometry
  const int A = rank * OWC, B = A + OWC;
  const int ext0 = A - K2;                      // extended range start
  const int own0 = ext0 + warp * Q;             // warp strip start
  const int wa = own0 - KT;                     // warp window start
  const int c0 = wa + lane * V;                 // this lane's first column
  const int frame_base = own0 - KS;             // ancestor frame of this warp
  const bool strip_lane = !producer && (lane * V >= KT) && (lane * V < KT + Q);
  const bool cta_own = strip_lane && c0 >= A && c0 < B;   // A, B, c0 are multiples of 4
  uint32_t oobm[V];
#pragma unroll
  for (int u = 0; u < V; ++u) oobm[u] = (c0 + u < 0 || c0 + u >= W) ? SENT : 0u;
  const int bidx0 = c0 - (ext0 - KT);           // index of c0 in bnd and in a staged energy row

  unsigned long long lastmin = ~0ull;
  if (threadIdx.x <= NW) wmin[threadIdx.x] = ~0ull;
  const int nt = gated ? 0 : (H + KT - 1) / KT;
  constexpr uint32_t ROW_BYTES = BW * 2;

  if (threadIdx.x == 0) {
    for (int q = 0; q < NSLOT; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], NW);
    }
    mbar_init(&hbar[0], 1);
    mbar_init(&hbar[1], 1);
    fence_mbar_init();
  }
  // neighbours push into hbuf/hbar: their initialisation must be visible cluster-wide first
  cl.sync();

  if (producer) {
    // ---- energy staging: rows of columns [ext0 - KT, ext0 - KT + BW), one bulk copy per lane ----
    const uint16_t *Estage = p.E + (ext0 - KT);
    for (int tt = 0; tt < nt; ++tt) {
      const int slot = tt % NSLOT;
      if (tt >= NSLOT && !mbar_wait_bounded(&empty[slot], (uint32_t)(((tt / NSLOT) - 1) & 1), WAIT_TIMEOUT_NS)) {
        if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
      }
      const int rbeg = tt * KT;
      const int nrows = (H - rbeg < KT) ? H - rbeg : KT;
      if (lane == 0) mbar_arrive_expect_tx(&full[slot], (uint32_t)nrows * ROW_BYTES);
      __syncwarp();
      if (lane < nrows)
        bulk_g2s(ring + (size_t)(slot * KT + lane) * BW, Estage + (size_t)(rbeg + lane) * p.pitch_e, ROW_BYTES,
                 &full[slot]);
    }
  } else {
    uint32_t k[V] = {0u, 0u, 0u, 0u};
    for (int t = 0; t < nt; ++t) {
      const int r0 = t * KT;
      const bool more = r0 + KT < H;
      const int slot = t % NSLOT;
      if (!mbar_wait_bounded(&full[slot], (uint32_t)((t / NSLOT) & 1), WAIT_TIMEOUT_NS)) {
        if (lane == 0) atomicOr(p.err, ERR_TIMEOUT);
      }
      const uint16_t *er = ring + (size_t)slot * KT * BW + bidx0;
      if (t > 0) {
        // window of the previous row from the boundary buffer (relative ancestors -> warp frame)
        const uint4 v = *reinterpret_cast<const uint4 *>(bnd + ((t - 1) & 1) * BW + bidx0);
        if (r0 % KS == 0) {
          // a new super-tile: every cell becomes its own ancestor. The old ancestor field is
          // dropped without arithmetic: it may lie outside this warp's frame.
          const uint32_t a = (uint32_t)(c0 - frame_base);
          k[0] = (v.x & ~0xFFu) | a; k[1] = (v.y & ~0xFFu) | (a + 1);
          k[2] = (v.z & ~0xFFu) | (a + 2); k[3] = (v.w & ~0xFFu) | (a + 3);
        } else {
          // relative ancestor -> this warp's frame (exact for every cell that can reach the strip)
          const uint32_t d = (uint32_t)(c0 - frame_base) - 128u;
          k[0] = v.x + d; k[1] = v.y + d + 1u; k[2] = v.z + d + 2u; k[3] = v.w + d + 3u;
        }
        k[0] |= oobm[0]; k[1] |= oobm[1]; k[2] |= oobm[2]; k[3] |= oobm[3];
      }
      if (t > 0 && !(r0 + KT > H)) {
        // full tile: 16 branch-free rows, bookkeeping only on its last row
#pragma unroll
        for (int r = 0; r < KT; ++r) dp_row(k, *reinterpret_cast<const uint2 *>(er + r * BW), oobm);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);   // this warp is done with the staged rows
        row_events(r0 + KT - 1, k, H, W, c0, frame_base, cta_own, A, p.Mrow, p.pitch_e, ancT, OWC, lastmin);
      } else {
        // first tile (row 0 has no predecessor) or a ragged last tile
        for (int r = 0; r < KT; ++r) {
          const int i = r0 + r;
          if (i >= H) break;
          const uint2 ev = *reinterpret_cast<const uint2 *>(er + r * BW);
          if (i == 0) {
            const uint32_t a = (uint32_t)(c0 - frame_base);
            k[0] = (lo8(ev.x) | a) | oobm[0];
            k[1] = (hi8(ev.x) | (a + 1)) | oobm[1];
            k[2] = (lo8(ev.y) | (a + 2)) | oobm[2];
            k[3] = (hi8(ev.y) | (a + 3)) | oobm[3];
          } else {
            dp_row(k, ev, oobm);
          }
          row_events(i, k, H, W, c0, frame_base, cta_own, A, p.Mrow, p.pitch_e, ancT, OWC, lastmin);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
      }
      if (more) {
        const bool exch = ((r0 + KT) % K2 == 0) && cs > 1;
        const uint32_t d = (uint32_t)(c0 - frame_base) - 128u;
        uint4 v;
        v.x = k[0] - d; v.y = k[1] - d - 1u; v.z = k[2] - d - 2u; v.w = k[3] - d - 3u;
        // publish this warp's strip (relative ancestor encoding); at an exchange the CTA's halo
        // columns come from the neighbours instead
        if (strip_lane && (!exch || (c0 >= A && c0 < B)))
          *reinterpret_cast<uint4 *>(bnd + (t & 1) * BW + bidx0) = v;
        if (exch) {
          const int x = (r0 + KT) / K2 - 1;
          const int par = x & 1;
          // my first K2 own columns are the left neighbour's right halo, my last K2 the right's left halo
          if (strip_lane && rank > 0 && c0 >= A && c0 < A + K2)
            st_async_v4(mapa_u32(hbuf + par * 2 * K2 + K2 + (c0 - A), rank - 1), v, mapa_u32(&hbar[par], rank - 1));
          if (strip_lane && rank < cs - 1 && c0 >= B - K2 && c0 < B)
            st_async_v4(mapa_u32(hbuf + par * 2 * K2 + (c0 - (B - K2)), rank + 1), v, mapa_u32(&hbar[par], rank + 1));
          if (threadIdx.x == 0)
            mbar_arrive_expect_tx(&hbar[par], (uint32_t)(((rank > 0) + (rank < cs - 1)) * K2 * 4));
          if (!mbar_wait_bounded(&hbar[par], (uint32_t)((x >> 1) & 1), WAIT_TIMEOUT_NS)) {
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
  }
  __syncthreads();

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
    *cmin = m;
  }
  cl.sync();

  // ---- ancestor chain (rank 0, one thread): seam column at every super-tile bottom ----
  if (rank == 0 && threadIdx.x == 0) {
    int ok = !gated;
    unsigned long long best = ~0ull;
    for (int r = 0; r < cs; ++r) {
      const unsigned long long *rm = cl.map_shared_rank(cmin, r);
      best = *rm < best ? *rm : best;
    }
    int j = (int)(best & 0xFFFFFFFFull);
    if (ok && (j < 0 || j >= W)) { ok = 0; atomicOr(p.err, ERR_BAD_SEAM); }
    for (int s = S - 1; ok && s >= 0; --s) {
      jb[s] = j;
      const int c = j / OWC;
      if (c < 0 || c >= cs) { ok = 0; atomicOr(p.err, ERR_BAD_SEAM); break; }
      const uint8_t *ra = cl.map_shared_rank(ancT, c);
      j = j + (int)ra[(size_t)s * OWC + (j - c * OWC)] - 128;
      if (j < 0 || j >= W) { ok = 0; atomicOr(p.err, ERR_BAD_SEAM); }
    }
    jb[S] = j;          // the seam's column in row 0
    misc[0] = ok;
    misc[1] = (int)(best >> 32);
    if (ok && p.cost) *p.cost = (int64_t)(best >> 32);
  }
  cl.sync();

  // ---- parallel backtrack: each super-tile recomputed in a 256-column window ----
  const int *jb0 = cl.map_shared_rank(jb, 0);
  const int *misc0 = cl.map_shared_rank(misc, 0);
  const int ok = misc0[0];
  const uint32_t best_m = (uint32_t)misc0[1];
  uint16_t *fd = fdir + (size_t)warp * KS * 32;
  for (int s = warp * cs + rank; ok && s < S; s += (NW + 1) * cs) {
    const int jbs = jb0[s];
    const int jprev = (s > 0) ? jb0[s - 1] : jb0[S];
    int x0 = jbs - 128;
    x0 -= ((x0 % 8) + 8) % 8;
    const int xc = x0 + lane * 8;
    const int rs = s * KS, re = (rs + KS < H) ? rs + KS : H;
    const int first = (s == 0) ? 1 : rs;
    uint32_t m[8], oob[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) oob[u] = (xc + u < 0 || xc + u >= W) ? SENT : 0u;
    if (s == 0) {
      const uint4 ev = *reinterpret_cast<const uint4 *>(p.E + xc);
      m[0] = ev.x & 0xFFFFu; m[1] = ev.x >> 16; m[2] = ev.y & 0xFFFFu; m[3] = ev.y >> 16;
      m[4] = ev.z & 0xFFFFu; m[5] = ev.z >> 16; m[6] = ev.w & 0xFFFFu; m[7] = ev.w >> 16;
    } else {
      const uint4 a = *reinterpret_cast<const uint4 *>(p.Mrow + (size_t)s * p.pitch_e + xc);
      const uint4 b = *reinterpret_cast<const uint4 *>(p.Mrow + (size_t)s * p.pitch_e + xc + 4);
      m[0] = a.x; m[1] = a.y; m[2] = a.z; m[3] = a.w; m[4] = b.x; m[5] = b.y; m[6] = b.z; m[7] = b.w;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] |= oob[u];
    // rows first..re-1 in chunks of 8 with the next chunk's energies loaded ahead
    constexpr int CH = 8;
    uint4 eb0[CH], eb1[CH];
    auto load_chunk = [&](uint4 (&eb)[CH], int rbeg) {
#pragma unroll
      for (int r = 0; r < CH; ++r) {
        const int i = rbeg + r;
        if (i < re) eb[r] = __ldg(reinterpret_cast<const uint4 *>(p.E + (size_t)i * p.pitch_e + xc));
      }
    };
    auto run_chunk = [&](const uint4 (&eb)[CH], int rbeg) {
#pragma unroll
      for (int r = 0; r < CH; ++r) {
        const int i = rbeg + r;
        if (i >= re) break;
        const uint32_t ee[8] = {eb[r].x & 0xFFFFu, eb[r].x >> 16, eb[r].y & 0xFFFFu, eb[r].y >> 16,
                                eb[r].z & 0xFFFFu, eb[r].z >> 16, eb[r].w & 0xFFFFu, eb[r].w >> 16};
        const uint32_t L = __shfl_up_sync(0xffffffffu, m[7], 1);
        const uint32_t R = __shfl_down_sync(0xffffffffu, m[0], 1);
        uint32_t nm[8];
        uint32_t dirs = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const uint32_t a = (u == 0) ? L : m[u - 1];
          const uint32_t b = m[u];
          const uint32_t c = (u == 7) ? R : m[u + 1];
          const uint32_t mn = min3u(a, b, c);
          const uint32_t d = (a == mn) ? 0u : ((b == mn) ? 1u : 2u);
          dirs |= d << (2 * u);
          nm[u] = (mn + ee[u]) | oob[u];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) m[u] = nm[u];
        fd[(i - rs) * 32 + lane] = (uint16_t)dirs;
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
      if ((rel >> 3) == lane) {
        uint32_t v = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) if (u == (rel & 7)) v = m[u];
        if (v != best_m) atomicOr(p.err, ERR_COST_MISMATCH);
      }
    }
    __syncwarp();
    if (lane == 0) {
      int j = jbs;
      for (int i = re - 1; i >= first; --i) {
        p.seam[i] = j;
        if (p.seam_log) p.seam_log[i] = j;
        const int rel = j - x0;
        if (rel < 0 || rel >= FILL_W) { atomicOr(p.err, ERR_FILL_MISMATCH); j = -1; break; }
        const uint32_t d = (fd[(i - rs) * 32 + (rel >> 3)] >> (2 * (rel & 7))) & 3u;
        j += (int)d - 1;
      }
      if (s == 0 && j >= 0) {
        p.seam[0] = j;
        if (p.seam_log) p.seam_log[0] = j;
      }
      if (j != jprev) atomicOr(p.err, ERR_FILL_MISMATCH);
    }
    __syncwarp();
  }
  cl.sync();   // rank 0's shared memory is read above; keep every CTA alive until all are done
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
  cfg.blockDim = dim3((NW + 1) * 32);
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
