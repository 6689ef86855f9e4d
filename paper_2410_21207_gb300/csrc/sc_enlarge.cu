// Seam insertion (enlargement): widen an image by k seams. The first k seams that the carve would
// remove are found by the carve itself (their log, each seam in its own shrinking image's
// columns); k_enlarge_map turns them into the set of input columns they delete, row by row, and
// k_insert writes every input pixel followed, where its column is in that set, by a pixel holding
// the rounded-up mean (a + b + 1) / 2 of it and its right neighbour (itself at the last column).
#include "../../include/sc.h"
#include "sc_internal.cuh"

namespace sc {

// position of the r-th (0-based) set bit of m (m has more than r set bits)
__device__ __forceinline__ int select_bit(uint32_t m, int r) {
  int p = 0;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const int c = __popc(m & ((1u << w) - 1u));
    if (r >= c) {
      r -= c;
      p += w;
      m >>= w;
    }
  }
  return p;
}

constexpr int MAP_WARPS = 8;                          // rows per block
constexpr int MAP_WORDS = (SC_MAX_COLS + 31) / 32;    // bitmap words of the widest row (256)
constexpr int MAP_WPL = MAP_WORDS / 32;               // words per lane (8)

// One warp per row. The row's deleted input columns are a bitmap in shared memory; lane l keeps
// the counts of columns still present in its words 8l .. 8l+7. For seam t, whose column c counts
// the columns still present, a warp prefix sum over the lanes' counts finds the lane, the word and
// (by a bit select) the input column, which is then marked deleted.
__global__ void __launch_bounds__(MAP_WARPS * 32) k_enlarge_map(const int32_t *__restrict__ log, int H, int W, int k,
                                                               uint32_t *__restrict__ bits, int nwords,
                                                               int32_t *__restrict__ cols, int *err) {
  __shared__ uint32_t del[MAP_WARPS][MAP_WORDS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * MAP_WARPS + warp;
  if (i >= H) return;
  uint32_t *d = del[warp];
  int cnt[MAP_WPL];
  int mine = 0;
#pragma unroll
  for (int q = 0; q < MAP_WPL; ++q) {
    const int w = lane * MAP_WPL + q;
    const int valid = W - 32 * w;   // columns of this word inside the row
    const uint32_t m = valid >= 32 ? 0u : (valid <= 0 ? 0xFFFFFFFFu : (0xFFFFFFFFu << valid));
    d[w] = m;                       // columns beyond the row count as deleted
    cnt[q] = 32 - __popc(m);
    mine += cnt[q];
  }
  __syncwarp();
  for (int t = 0; t < k; ++t) {
    const int c = log[(int64_t)t * H + i];
    int incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    const int excl = incl - mine;
    const bool owner = (c >= excl) && (c < incl);
    const unsigned who = __ballot_sync(0xffffffffu, owner);
    if (who == 0u) {   // c outside the present columns: a corrupt log
      if (lane == 0) atomicOr(err, ERR_BAD_SEAM);
      return;
    }
    if (owner) {
      int r = c - excl;
      bool found = false;
#pragma unroll
      for (int q = 0; q < MAP_WPL; ++q) {
        if (!found) {
          if (r < cnt[q]) {
            const int w = lane * MAP_WPL + q;
            const int b = select_bit(~d[w], r);
            d[w] |= 1u << b;
            cnt[q] -= 1;
            if (cols) cols[(int64_t)t * H + i] = 32 * w + b;
            found = true;
          } else {
            r -= cnt[q];
          }
        }
      }
      mine -= 1;
    }
    __syncwarp();
  }
  // the deleted columns inside the row are the columns that get an inserted pixel
  for (int w = lane; w < nwords; w += 32) {
    const int valid = W - 32 * w;
    const uint32_t inside = valid >= 32 ? 0xFFFFFFFFu : ((1u << valid) - 1u);
    bits[(int64_t)i * nwords + w] = d[w] & inside;
  }
}

// One block per row, one bitmap word (32 input columns) per thread: an exclusive block scan of the
// words' populations gives every input pixel its output column.
__global__ void __launch_bounds__(256) k_insert(const uint8_t *__restrict__ img, int H, int W, int C,
                                                const uint32_t *__restrict__ bits, int nwords,
                                                uint8_t *__restrict__ out, int tw) {
  __shared__ int wsum[8];
  const int i = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t m = (t < nwords) ? bits[(int64_t)i * nwords + t] : 0u;
  const int n = __popc(m);
  int incl = n;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += o;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int base = incl - n;
  for (int w = 0; w < warp; ++w) base += wsum[w];
  if (t >= nwords) return;
  const uint8_t *row = img + (int64_t)i * W * C;
  uint8_t *o = out + (int64_t)i * tw * C;
  for (int b = 0; b < 32; ++b) {
    const int j = 32 * t + b;
    if (j >= W) break;
    const int pos = j + base + __popc(m & ((1u << b) - 1u));
    for (int ch = 0; ch < C; ++ch) o[(int64_t)pos * C + ch] = row[(int64_t)j * C + ch];
    if ((m >> b) & 1u) {
      const int jr = j + 1 < W ? j + 1 : W - 1;
      for (int ch = 0; ch < C; ++ch)
        o[(int64_t)(pos + 1) * C + ch] =
            (uint8_t)(((int)row[(int64_t)j * C + ch] + (int)row[(int64_t)jr * C + ch] + 1) >> 1);
    }
  }
}

cudaError_t launch_enlarge_map(const int32_t *log, int H, int W, int k, uint32_t *bits, int32_t *cols, int *err,
                               cudaStream_t st) {
  if (W > SC_MAX_COLS) return cudaErrorInvalidValue;
  const int nwords = (W + 31) / 32;
  k_enlarge_map<<<(H + MAP_WARPS - 1) / MAP_WARPS, MAP_WARPS * 32, 0, st>>>(log, H, W, k, bits, nwords, cols, err);
  return cudaGetLastError();
}

cudaError_t launch_insert(const uint8_t *img, int H, int W, int C, const uint32_t *bits, uint8_t *out, int tw,
                          cudaStream_t st) {
  const int nwords = (W + 31) / 32;
  if (nwords > 256) return cudaErrorInvalidValue;
  k_insert<<<H, 256, 0, st>>>(img, H, W, C, bits, nwords, out, tw);
  return cudaGetLastError();
}

}  // namespace sc
