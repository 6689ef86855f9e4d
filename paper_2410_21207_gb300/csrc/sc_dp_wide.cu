// The seam search for maps whose seam sums do not fit the 24-bit cost field of seam_search
// (arXiv 2410.21207, section "DP Seam Carving": Algorithm 3 and the recurrence
// M(i,j) = e(i,j) + min(M(i-1,j-1), M(i-1,j), M(i-1,j+1))).
//
// Any uint16 map is a valid input (the paper's DP has no bound on the energies), but seam_search
// packs a 24-bit cost with an 8-bit ancestor into one 32-bit key. The energy copy kernels check
// H * max(e) < 2^24 per map and, when it fails, set that map's gate; seam_search then skips the
// map and this kernel, launched right after it on the same stream, searches it instead (it returns
// at once for maps whose gate is clear). M stays exact in 32 bits: H <= 8192 rows of energies
// <= 65535 (forward energy: <= 131070 per row) sum to less than 2^31.
//
// One CTA of 1024 threads per map, one row after another:
//   * thread t owns the column pairs q = t, t + 1024, ... (columns 2q, 2q + 1); the previous and
//     the current cost row live in shared memory (double buffered), one CTA barrier per row;
//   * every cell picks the leftmost minimum of its in-range predecessors, exactly as Algorithm 3
//     reads (ties to j-1, then j, then j+1); its direction (2 bits) goes to global memory by four
//     warp ballots per 64 columns;
//   * beside M, every cell carries the column where its optimal path left the previous super-tile
//     of KW ~ sqrt(H) rows (its own column in row 0); the bottom row of each super-tile stores
//     them, so after the last-row argmin one thread follows ceil(H/KW) of them to the seam's
//     column at every super-tile bottom, and then one thread per super-tile walks its KW rows of
//     directions in parallel;
//   * self-checks: every walk must end on the column the chain gave, and the energies along the
//     seam must add up to the argmin.
// The energies of the next rows are loaded into registers WIDE_D rows ahead of their use.
#include "sc_internal.cuh"

namespace sc {

constexpr int WIDE_THREADS = 1024;
constexpr int WIDE_D = 4;           // rows of energies in flight per thread
constexpr uint32_t WINF = 0xFFFFFFFFu;

__host__ __device__ inline int wide_super_rows(int H) {
  int k = 1;
  while (k * k < H) ++k;
  return k < 16 ? 16 : k;
}

size_t wide_dirs_words(int H, int W) { return (size_t)H * (size_t)((W + 63) / 64) * 4; }

size_t wide_anc_elems(int H, int W) {
  const int k = wide_super_rows(H);
  return (size_t)((H + k - 1) / k) * (size_t)W;
}

static size_t wide_smem_bytes(int H, int W) {
  const int k = wide_super_rows(H);
  const int S = (H + k - 1) / k;
  const size_t WP = (size_t)2 * ((W + 1) / 2);
  size_t o = 2 * WP * 4;           // cost rows
  o += 2 * WP * 2;                 // ancestor rows
  o = (o + 15) & ~(size_t)15;
  o += (size_t)(S + 1) * 4;        // seam column at every super-tile bottom (+ row 0)
  o = (o + 15) & ~(size_t)15;
  o += 33 * 8;                     // argmin partials, cost sum
  return o;
}

// direction (0: from j-1, 1: from j, 2: from j+1) of column c in row i
__device__ __forceinline__ int wide_dir(const uint32_t *dirs, int npb, int i, int c) {
  const uint4 w = *reinterpret_cast<const uint4 *>(dirs + ((size_t)i * npb + (c >> 6)) * 4);
  const int lane = (c >> 1) & 31;
  const uint32_t b0 = (c & 1) ? w.z : w.x, b1 = (c & 1) ? w.w : w.y;
  return (int)(((b0 >> lane) & 1u) | (((b1 >> lane) & 1u) << 1));
}

template <bool FWD>
__device__ void wide_search(const DpArgs &p, uint32_t *__restrict__ dirs, uint16_t *__restrict__ ancg,
                            unsigned char *smem) {
  if (!(p.gate && (*p.gate & ERR_ENERGY_RANGE))) return;   // the 24-bit search handled this map
  constexpr int MAXP = FWD ? 2 : 4;                        // column pairs per thread (W <= 4096 / 8192)
  constexpr int NP = FWD ? 3 : 1;                          // cost planes (CU, DL, DR)
  const int H = p.H, W = p.W;
  const int KW = wide_super_rows(H), S = (H + KW - 1) / KW;
  const int np = (W + 1) / 2, WP = 2 * np, npb = (W + 63) / 64;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int nu = (np + WIDE_THREADS - 1) / WIDE_THREADS;   // pair slots per thread (uniform)
  uint32_t *Mb = reinterpret_cast<uint32_t *>(smem);
  uint16_t *Ab = reinterpret_cast<uint16_t *>(Mb + 2 * WP);
  size_t o = ((size_t)2 * WP * 4 + (size_t)2 * WP * 2 + 15) & ~(size_t)15;
  int *jb = reinterpret_cast<int *>(smem + o);
  o = (o + (size_t)(S + 1) * 4 + 15) & ~(size_t)15;
  unsigned long long *red = reinterpret_cast<unsigned long long *>(smem + o);
  const uint16_t *E = p.E;
  const int pe = p.pitch_e;
  const int64_t ps = FWD ? p.pstride : 0;

  // row 0: M = e (CU), every cell its own ancestor
  for (int u = 0; u < nu; ++u) {
    const int q = t + u * WIDE_THREADS;
    if (q >= np || u >= MAXP) continue;
    const int a = 2 * q;
    const uint32_t ev = *reinterpret_cast<const uint32_t *>(E + a);
    Mb[a] = ev & 0xFFFFu;
    Mb[a + 1] = (a + 1 < W) ? (ev >> 16) : WINF;
    Ab[a] = (uint16_t)a;
    Ab[a + 1] = (uint16_t)(a + 1);
    if (H == 1) {
      ancg[a] = (uint16_t)a;
      if (a + 1 < W) ancg[a + 1] = (uint16_t)(a + 1);
    }
  }
  // energies of rows 1 .. WIDE_D, one 4-byte pair per plane and pair slot
  uint32_t eb[WIDE_D][MAXP][NP];
  auto load_row = [&](uint32_t (&dst)[MAXP][NP], int i) {
#pragma unroll
    for (int u = 0; u < MAXP; ++u) {
      const int q = t + u * WIDE_THREADS;
      if (u < nu && q < np) {
#pragma unroll
        for (int pl = 0; pl < NP; ++pl)
          dst[u][pl] = *reinterpret_cast<const uint32_t *>(E + pl * ps + (size_t)i * pe + 2 * q);
      }
    }
  };
#pragma unroll
  for (int r = 0; r < WIDE_D; ++r)
    if (1 + r < H) load_row(eb[r], 1 + r);
  __syncthreads();

  int rin = 1;   // row index inside the current super-tile
  for (int i0 = 1; i0 < H; i0 += WIDE_D) {
#pragma unroll
    for (int r = 0; r < WIDE_D; ++r) {
      const int i = i0 + r;
      if (i >= H) break;
      if (rin == KW) rin = 0;
      const uint32_t *Mp = Mb + ((i - 1) & 1) * WP;
      uint32_t *Mn = Mb + (i & 1) * WP;
      const uint16_t *Ap = Ab + ((i - 1) & 1) * WP;
      uint16_t *An = Ab + (i & 1) * WP;
      const bool fresh = (rin == 0);              // first row of a super-tile: ancestor = predecessor
      const bool store = (rin == KW - 1) || (i == H - 1);
      const int s = i / KW;
#pragma unroll
      for (int u = 0; u < MAXP; ++u) {
        if (u >= nu) break;
        const int q = t + u * WIDE_THREADS;
        int da = 0, db = 0;
        if (q < np) {
          const int a = 2 * q, b = a + 1;
          const uint32_t e2 = eb[r][u][0];
          const uint32_t dl2 = FWD ? eb[r][u][NP > 1 ? 1 : 0] : 0u;
          const uint32_t dr2 = FWD ? eb[r][u][NP > 2 ? 2 : 0] : 0u;
          const uint32_t m0 = Mp[a];
          const uint32_t m1 = (b < W) ? Mp[b] : WINF;
          // column a: predecessors a-1, a, a+1
          uint32_t mn = (a > 0) ? Mp[a - 1] + (dl2 & 0xFFFFu) : WINF;
          if (m0 < mn) { mn = m0; da = 1; }
          if (b < W) {
            const uint32_t c = m1 + (dr2 & 0xFFFFu);
            if (c < mn) { mn = c; da = 2; }
          }
          Mn[a] = mn + (e2 & 0xFFFFu);
          const int pa = a + da - 1;
          const uint16_t anc_a = fresh ? (uint16_t)pa : Ap[pa];
          An[a] = anc_a;
          if (store) ancg[(size_t)s * W + a] = anc_a;
          if (b < W) {
            // column b: predecessors a, b, b+1
            uint32_t mb = m0 + (dl2 >> 16);
            if (m1 < mb) { mb = m1; db = 1; }
            if (b + 1 < W) {
              const uint32_t c = Mp[b + 1] + (dr2 >> 16);
              if (c < mb) { mb = c; db = 2; }
            }
            Mn[b] = mb + (e2 >> 16);
            const int pb = b + db - 1;
            const uint16_t anc_b = fresh ? (uint16_t)pb : Ap[pb];
            An[b] = anc_b;
            if (store) ancg[(size_t)s * W + b] = anc_b;
          } else {
            Mn[b] = WINF;
          }
        }
        // directions of the warp's 64 columns: four bit planes
        const uint32_t w0 = __ballot_sync(0xffffffffu, da & 1), w1 = __ballot_sync(0xffffffffu, da >> 1);
        const uint32_t w2 = __ballot_sync(0xffffffffu, db & 1), w3 = __ballot_sync(0xffffffffu, db >> 1);
        const int pbk = warp + u * (WIDE_THREADS / 32);
        if (lane == 0 && pbk < npb)
          *reinterpret_cast<uint4 *>(dirs + ((size_t)i * npb + pbk) * 4) = make_uint4(w0, w1, w2, w3);
      }
      if (i + WIDE_D < H) load_row(eb[r], i + WIDE_D);
      ++rin;
      __syncthreads();
    }
  }

  // leftmost minimum of the last row: min of (M << 32) | column
  const uint32_t *Ml = Mb + ((H - 1) & 1) * WP;
  unsigned long long best = ~0ull;
  for (int c = t; c < W; c += WIDE_THREADS) {
    const unsigned long long k = ((unsigned long long)Ml[c] << 32) | (unsigned)c;
    best = k < best ? k : best;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, best, off);
    best = x < best ? x : best;
  }
  if (lane == 0) red[warp] = best;
  __syncthreads();
  if (t == 0) {
    unsigned long long m = ~0ull;
    for (int w = 0; w < WIDE_THREADS / 32; ++w) m = red[w] < m ? red[w] : m;
    red[0] = m;
    red[32] = 0ull;   // energy sum along the seam
    // ancestor chain: the seam's column at the bottom of every super-tile, then in row 0
    int j = (int)(m & 0xFFFFFFFFull);
    bool bad = (unsigned)j >= (unsigned)W;
    j = min(max(j, 0), W - 1);
    for (int s = S - 1; s >= 0; --s) {
      jb[s] = j;
      const int nj = ancg[(size_t)s * W + j];
      bad |= (unsigned)nj >= (unsigned)W;
      j = min(max(nj, 0), W - 1);
    }
    jb[S] = j;
    if (bad) atomicOr(p.err, ERR_BAD_SEAM);
    if (p.cost) *p.cost = (int64_t)(m >> 32);
  }
  __syncthreads();

  // every super-tile walked up its directions in parallel, one thread each
  if (t < S) {
    const int rs = t * KW, re = min(H, rs + KW);
    int c = jb[t];
    unsigned long long sum = 0;
    bool ok = true;
    for (int i = re - 1; i >= rs; --i) {
      p.seam[i] = c;
      if (p.seam_log) p.seam_log[i] = c;
      const uint32_t cu = E[(size_t)i * pe + c];
      if (i == 0) {
        sum += cu;
        ok &= (c == jb[S]);
        break;
      }
      const int d = wide_dir(dirs, npb, i, c);
      if (FWD) sum += cu + (d == 0 ? E[ps + (size_t)i * pe + c] : (d == 2 ? E[2 * ps + (size_t)i * pe + c] : 0u));
      else sum += cu;
      const int nc = c + d - 1;
      ok &= (unsigned)nc < (unsigned)W;
      c = min(max(nc, 0), W - 1);
      if (i == rs) ok &= (c == jb[t - 1]);   // the walk leaves on the previous super-tile's bottom column
    }
    if (!ok) atomicOr(p.err, ERR_FILL_MISMATCH);
    atomicAdd(&red[32], sum);
  }
  __syncthreads();
  if (t == 0 && red[32] != (red[0] >> 32)) atomicOr(p.err, ERR_COST_MISMATCH);
}

template <bool FWD>
__global__ void __launch_bounds__(WIDE_THREADS, 1) k_dp_wide(DpArgs p, uint32_t *dirs, uint16_t *anc) {
  extern __shared__ __align__(16) unsigned char smem[];
  wide_search<FWD>(p, dirs, anc, smem);
}

// map blockIdx.x of n, each with its own scratch slices
template <bool FWD>
__global__ void __launch_bounds__(WIDE_THREADS, 1) k_dp_wide_multi(const DpArgs *__restrict__ ps,
                                                                   const __grid_constant__ MultiArgs inl,
                                                                   uint32_t *dirs, uint16_t *anc, size_t dirs_stride,
                                                                   size_t anc_stride) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DpArgs p = ps ? ps[blockIdx.x] : inl.a[blockIdx.x];
  wide_search<FWD>(p, dirs + blockIdx.x * dirs_stride, anc + blockIdx.x * anc_stride, smem);
}

template <typename K>
static cudaError_t wide_configure(K kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_dp_wide(const DpArgs &a, uint32_t *dirs, uint16_t *anc, cudaStream_t st) {
  const size_t smem = wide_smem_bytes(a.H, a.W);
  if (a.pstride > 0) {
    if (a.W > 2 * 2 * WIDE_THREADS) return cudaErrorInvalidValue;
    cudaError_t e = wide_configure(k_dp_wide<true>, smem);
    if (e != cudaSuccess) return e;
    k_dp_wide<true><<<1, WIDE_THREADS, smem, st>>>(a, dirs, anc);
  } else {
    if (a.W > 4 * 2 * WIDE_THREADS) return cudaErrorInvalidValue;
    cudaError_t e = wide_configure(k_dp_wide<false>, smem);
    if (e != cudaSuccess) return e;
    k_dp_wide<false><<<1, WIDE_THREADS, smem, st>>>(a, dirs, anc);
  }
  return cudaGetLastError();
}

cudaError_t launch_dp_wide_multi(const DpArgs *dargs_dev, const MultiArgs *inl, int n, int H, int W, uint32_t *dirs,
                                 uint16_t *anc, cudaStream_t st) {
  if (n < 1 || W > 4 * 2 * WIDE_THREADS || (inl && n > MULTI_INLINE) || (!inl && !dargs_dev))
    return cudaErrorInvalidValue;
  const size_t smem = wide_smem_bytes(H, W);
  cudaError_t e = wide_configure(k_dp_wide_multi<false>, smem);
  if (e != cudaSuccess) return e;
  static const MultiArgs none{};
  k_dp_wide_multi<false><<<n, WIDE_THREADS, smem, st>>>(inl ? nullptr : dargs_dev, inl ? *inl : none, dirs, anc,
                                                        wide_dirs_words(H, W), wide_anc_elems(H, W));
  return cudaGetLastError();
}

}  // namespace sc
