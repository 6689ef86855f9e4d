// Per-pixel and per-row operations shared by the whole-image kernels (sc_kernels.cu) and the
// batched persistent kernel (sc_batch.cuh): the e1 energy of a pixel ("Energy Mapping", item e1),
// the two refreshed energies of a row after a removal, and the row compactions ("Removal of
// Seams"). Pixels are uint32 words, channel c in byte c (unused bytes 0).
#pragma once
#include <cstdint>

#include "sc_ptx.cuh"

namespace sc {

// sum over the four bytes of |a_b - b_b|
__device__ __forceinline__ uint32_t sad4(uint32_t a, uint32_t b) { return __vsadu4(a, b); }

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

// e1 energy of pixel (i, j) of a rows x cols word image with edge replication
__device__ __forceinline__ uint32_t energy_at(const uint32_t *img, int pitch, int rows, int cols, int i, int j) {
  const uint32_t *row = img + (int64_t)i * pitch;
  const int jl = j > 0 ? j - 1 : 0, jr = j + 1 < cols ? j + 1 : cols - 1;
  const int iu = i > 0 ? i - 1 : 0, id = i + 1 < rows ? i + 1 : rows - 1;
  return sad4(row[jr], row[jl]) + sad4(img[(int64_t)id * pitch + j], img[(int64_t)iu * pitch + j]);
}

// In-place left shift by one of a 16-byte-aligned uint16 row, row[s+1 .. W-1] -> row[s .. W-2],
// by one warp, 8 elements (one 16-byte load and store) at a time: chunk c of the result is chunk c of the input moved down one element, with the first
// element of chunk c+1 shifted in; every lane reads its chunks and the element after each chunk
// before any lane of the warp writes. The first chunk keeps its elements left of s. Elements from
// W-1 to the end of the last chunk are left undefined (they lie in the row's padding or in the
// column that the shift drops).
// `between` runs once, after the first block of loads is issued and before any store (work that
// overlaps their latency; it must not touch the row).
template <typename F>
__device__ __forceinline__ void shift_row_u16(uint16_t *row, int s, int W, int lane, F &&between) {
  constexpr int R = 4;
  if (s >= W - 1) {
    between();
    return;
  }
  const int c_lo = s >> 3, c_hi = (W - 2) >> 3;
  for (int cb = c_lo; cb <= c_hi; cb += 32 * R) {
    uint4 x[R];
    uint32_t nx[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = cb + r * 32 + lane;
      if (c <= c_hi) {
        x[r] = *reinterpret_cast<const uint4 *>(row + 8 * c);
        nx[r] = row[8 * c + 8];
      }
    }
    if (cb == c_lo) between();
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int c = cb + r * 32 + lane;
      if (c <= c_hi) {
        uint4 o;
        o.x = __funnelshift_r(x[r].x, x[r].y, 16);
        o.y = __funnelshift_r(x[r].y, x[r].z, 16);
        o.z = __funnelshift_r(x[r].z, x[r].w, 16);
        o.w = __funnelshift_r(x[r].w, nx[r], 16);
        if (c == c_lo) {
          const int keep = s - 8 * c;   // leading elements of this chunk that stay
          auto merge = [keep](uint32_t in, uint32_t sh, int q) {
            const uint32_t m = (2 * q < keep ? 0x0000FFFFu : 0u) | (2 * q + 1 < keep ? 0xFFFF0000u : 0u);
            return (in & m) | (sh & ~m);
          };
          o.x = merge(x[r].x, o.x, 0);
          o.y = merge(x[r].y, o.y, 1);
          o.z = merge(x[r].z, o.z, 2);
          o.w = merge(x[r].w, o.w, 3);
        }
        *reinterpret_cast<uint4 *>(row + 8 * c) = o;
      }
    }
    __syncwarp();
  }
}

__device__ __forceinline__ void shift_row_u16(uint16_t *row, int s, int W, int lane) {
  shift_row_u16(row, s, W, lane, [] {});
}

__device__ __forceinline__ uint32_t pack_pixel(const uint8_t *s, int C) {
  uint32_t w = s[0];
  if (C >= 3) w |= ((uint32_t)s[1] << 8) | ((uint32_t)s[2] << 16);
  if (C == 4) w |= (uint32_t)s[3] << 24;
  return w;
}

__device__ __forceinline__ void unpack_pixel(uint32_t w, uint8_t *d, int C) {
  d[0] = (uint8_t)w;
  if (C >= 3) {
    d[1] = (uint8_t)(w >> 8);
    d[2] = (uint8_t)(w >> 16);
  }
  if (C == 4) d[3] = (uint8_t)(w >> 24);
}

}  // namespace sc

namespace sc {

// ---- lazy compaction of the image words ----
// The stored words of a row are compacted only every RPEND seams. Between compactions each row
// keeps the sorted stored columns o_0 < o_1 < ... < o_(m-1) of its m removed pixels. Current column
// j (after the m removals) is stored column j + #{q : o_q - q <= j}: o_q - q is the number of kept
// pixels left of o_q, so the q-th removal is passed exactly when j reaches it.
constexpr int RPEND = 16;

// A row's pending removals in registers: the thresholds t_q = o_q - q, two 16-bit values per word,
// from two 16-byte loads (the lists are 32-byte rows); entries q >= m get t_q = 0x7FFF, above every
// column (columns stay below 2^15). Current column j is stored column j + #{q : t_q <= j}. A count
// is four instructions per word: for 16-bit halves a = 0x8000 + j and b = t_q <= 0x7FFF, a - b
// stays in [1, 0xFFFF] (no borrow between halves) and has bit 15 set exactly when t_q <= j.
// No load per entry on the way to a pixel.
struct LazyRow {
  uint32_t t[RPEND / 2];
};

__device__ __forceinline__ LazyRow lazy_row(const int16_t *list, int m) {
  const uint4 a = *reinterpret_cast<const uint4 *>(list);
  const uint4 b = *reinterpret_cast<const uint4 *>(list + 8);
  const uint32_t w[RPEND / 2] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  LazyRow r;
#pragma unroll
  for (int k = 0; k < RPEND / 2; ++k) {
    // entries past m become 0x7FFF + q before the subtraction (o_q >= q for the others: no borrow)
    const uint32_t lo = (2 * k < m) ? (w[k] & 0xFFFFu) : 0x7FFFu + 2 * k;
    const uint32_t hi = (2 * k + 1 < m) ? (w[k] >> 16) : 0x7FFFu + 2 * k + 1;
    r.t[k] = (lo | (hi << 16)) - ((uint32_t)(2 * k) | ((uint32_t)(2 * k + 1) << 16));
  }
  return r;
}

// removals passed by current column j (0 <= j < 2^15)
__device__ __forceinline__ int lazy_count(const LazyRow &r, int j) {
  const uint32_t jj = ((uint32_t)j * 0x10001u) | 0x80008000u;
  int c = 0;
#pragma unroll
  for (int k = 0; k < RPEND / 2; ++k) c += __popc((jj - r.t[k]) & 0x80008000u);
  return c;
}

// The two energies of row i that the removal of `seam` changes. After deleting seam s from a
// W-wide image, the energy of the (W-1)-wide image equals the old energy shifted left past s_i,
// except at the new columns s_i - 1 and s_i (their left/right neighbour changed, and, since
// |s_i - s_(i+-1)| <= 1, they are the only pixels whose upper/lower neighbour can change). They
// are computed from the old image seen through the removal: new pixel (r, j) = old (r, j + [j >= s_r]).
// Returns (e(s-1) | e(s) << 16); a value is 0 when its column does not exist. The image is read
// through the pending-removal lists of the width-W image the seam was found in: lc is row i's (seam
// column s), lu and ld those of the rows above and below, iu and id (edge rows replicated), whose
// seam columns are su and sd.
__device__ __forceinline__ uint32_t patch_pair(const uint32_t *img, int pitch, int W, int i, int s, int iu, int su,
                                               const LazyRow &lu, const LazyRow &lc, int id, int sd,
                                               const LazyRow &ld) {
  const int Wn = W - 1;
  // new pixel (r, j), j clamped to the new width, of a row r whose seam column is sr and list L
  auto pix = [&](int r, const LazyRow &L, int sr, int j) -> uint32_t {
    j = clampi(j, 0, Wn - 1);
    const int x = j + (j >= sr ? 1 : 0);                    // column in the width-W image
    return img[(int64_t)r * pitch + x + lazy_count(L, x)];
  };
  // columns s-1 and s of the rows above and below (edge rows replicated)
  const uint32_t up0 = pix(iu, lu, su, s - 1), up1 = pix(iu, lu, su, s);
  const uint32_t dn0 = pix(id, ld, sd, s - 1), dn1 = pix(id, ld, sd, s);
  const uint32_t p0 = (s >= 1) ? sad4(pix(i, lc, s, s), pix(i, lc, s, s - 2)) + sad4(dn0, up0) : 0u;
  const uint32_t p1 = (s <= Wn - 1) ? sad4(pix(i, lc, s, s + 1), pix(i, lc, s, s - 1)) + sad4(dn1, up1) : 0u;
  return p0 | (p1 << 16);
}

// patch_pair of row i, its seam columns and lists read here (lists: row r at lists + r*RPEND, m
// entries each); row i's list comes back in *li for the insertion that follows, and *bad is set
// when the seam column is out of range.
__device__ __forceinline__ uint32_t patch_row_lazy(const uint32_t *img, int pitch, int H, int W, const int32_t *seam,
                                                   const int16_t *lists, int m, int i, bool *bad, LazyRow *li) {
  const int s = seam[i];
  *li = lazy_row(lists + (int64_t)i * RPEND, m);
  if (s < 0 || s >= W) {
    *bad = true;
    return 0u;
  }
  const int iu = i > 0 ? i - 1 : 0, id = i + 1 < H ? i + 1 : H - 1;
  const LazyRow lu = lazy_row(lists + (int64_t)iu * RPEND, m);
  const LazyRow ld = lazy_row(lists + (int64_t)id * RPEND, m);
  return patch_pair(img, pitch, W, i, s, iu, seam[iu], lu, *li, id, seam[id], ld);
}

// Add a row's removal at current column s to its sorted list (L: the row's m entries): the removals
// it passes are exactly the first c = lazy_count(s) (t_q never decreases with q), so the stored
// column o = s + c goes in at position c. out gets m + 1 entries (two 16-byte stores).
__device__ __forceinline__ void list_insert(const LazyRow &L, int16_t *out, int s) {
  const int c = lazy_count(L, s);
  const uint32_t o = (uint32_t)(s + c);
  uint32_t raw[RPEND / 2], v[RPEND / 2];
#pragma unroll
  for (int k = 0; k < RPEND / 2; ++k) raw[k] = L.t[k] + ((uint32_t)(2 * k) | ((uint32_t)(2 * k + 1) << 16));   // o_q
#pragma unroll
  for (int k = 0; k < RPEND / 2; ++k) {
    const uint32_t up = k > 0 ? __funnelshift_l(raw[k - 1], raw[k], 16) : (raw[0] << 16);   // entries moved up one
    uint32_t x = 0u;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = 2 * k + h;
      const uint32_t keep = (raw[k] >> (16 * h)) & 0xFFFFu, moved = (up >> (16 * h)) & 0xFFFFu;
      x |= (q < c ? keep : (q == c ? o : moved)) << (16 * h);
    }
    v[k] = x;
  }
  *reinterpret_cast<uint4 *>(out) = make_uint4(v[0], v[1], v[2], v[3]);
  *reinterpret_cast<uint4 *>(out + 8) = make_uint4(v[4], v[5], v[6], v[7]);
}

// The refreshed pairs and pending-removal list updates of the rows one thread handles (local rows
// q = t0, t0 + tstride, ... of nq; image row row0 + q * rstride): pairs[q] gets row q's pair (as
// patch_row_lazy) and lists_out its list with this seam's removal added. Returns true when a seam
// column was out of range (the rows after it are left alone).
__device__ __forceinline__ bool refresh_pairs(const uint32_t *img, int pitch, int H, int W, const int32_t *seam,
                                           const int16_t *lists_in, int16_t *lists_out, int m, int nq, int row0,
                                           int rstride, uint32_t *pairs, int t0, int tstride) {
  bool bad = false;
#pragma unroll 1
  for (int q = t0; q < nq; q += tstride) {
    const int i = row0 + q * rstride;
    LazyRow li;
    pairs[q] = patch_row_lazy(img, pitch, H, W, seam, lists_in, m, i, &bad, &li);
    if (!bad) list_insert(li, lists_out + (size_t)i * RPEND, seam[i]);
  }
  return bad;
}

// Compact one row of stored words in place by one warp: current column j <- its stored column, for
// j < w. Sources never lie left of their destination and the row is processed left to right in
// chunks read completely before they are written, so nothing is overwritten before it is read.
__device__ __forceinline__ void compact_row_lazy(uint32_t *row, const int16_t *list, int m, int w, int lane) {
  constexpr int R = 4;
  int l[RPEND];   // o_q - q (the output column where the q-th removal is passed), padded high
#pragma unroll
  for (int q = 0; q < RPEND; ++q) l[q] = q < m ? (int)list[q] - q : 0x7FFFFFFF;
  int first = w;   // columns left of the first removal keep their place
  if (m > 0) first = l[0];
  for (int base = first; base < w; base += 32 * R) {
    uint32_t x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int j = base + r * 32 + lane;
      if (j < w) {
        int c = 0;
#pragma unroll
        for (int q = 0; q < RPEND; ++q) c += (l[q] <= j) ? 1 : 0;
        x[r] = row[j + c];
      }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int j = base + r * 32 + lane;
      if (j < w) row[j] = x[r];
    }
    __syncwarp();
  }
}

}  // namespace sc

namespace sc {

// One warp, row i, after seam `seam` was found in the width-W energy map E (and image words read
// through the pending-removal lists_in with m entries): the row's refreshed energy pair (lane 0,
// through the lazy map), the row's list with this removal added (lists_out), then the energy row's
// tail shifted left past the seam and the pair written at the new columns s-1 and s.
// Returns false when the seam column is out of range (nothing is changed then).
__device__ __forceinline__ bool refresh_row(const uint32_t *img, int pitch, uint16_t *E, int pe, int H, int W,
                                            const int32_t *seam, const int16_t *lists_in, int16_t *lists_out, int m,
                                            int i, int lane) {
  // lane 0's pending-removal lists of rows i-1, i, i+1 and the neighbours' seam columns depend on i
  // alone: loaded beside seam[i], they take a round trip off the refreshed pair's path
  const int iu = i > 0 ? i - 1 : 0, id = i + 1 < H ? i + 1 : H - 1;
  LazyRow lu{}, lc{}, ld{};
  int su = 0, sd = 0;
  if (lane == 0) {
    lc = lazy_row(lists_in + (int64_t)i * RPEND, m);
    lu = lazy_row(lists_in + (int64_t)iu * RPEND, m);
    ld = lazy_row(lists_in + (int64_t)id * RPEND, m);
    su = seam[iu];
    sd = seam[id];
  }
  const int s = seam[i];
  if (s < 0 || s >= W) return false;
  uint32_t p = 0;
  uint16_t *er = E + (int64_t)i * pe;
  // lane 0 computes the refreshed pair (image words through the lists, not the energy row) while
  // the warp's loads of the energy tail are in flight
  shift_row_u16(er, s, W, lane, [&] {
    if (lane == 0) {
      p = patch_pair(img, pitch, W, i, s, iu, su, lu, lc, id, sd, ld);
      list_insert(lc, lists_out + (int64_t)i * RPEND, s);
    }
  });
  if (lane == 0) {
    if (s >= 1) er[s - 1] = (uint16_t)(p & 0xFFFFu);
    if (s <= W - 2) er[s] = (uint16_t)(p >> 16);
  }
  return true;
}

// The energy shift of every row this warp owns (local rows q = warp, warp + nwarps, ... of nq; image
// row row0 + q * rstride), each followed by its refreshed pair (pairs[q]: e(s-1) | e(s) << 16), staged
// by TMA. In rounds, the warp takes as many of its next rows as its buffer holds (a prefix sum of
// their tail sizes over the lanes); lane l copies row l's tail (the 16-byte chunks from the one
// holding s to the one after the new last column) with one bulk copy, all completing on one
// mbarrier at the head of the buffer; then each row is written back one element to the left, 32
// lanes over its chunks, reading only the staged copy (so nothing is overwritten before it is read).
// buf: this warp's buffer, 16-byte aligned, buf_bytes of it (the first 16 hold the mbarrier). Rows
// whose seam is out of range are skipped (the caller records the error). Returns false when a wait
// ran out (the caller records ERR_TIMEOUT). Not inlined (nor is compact_rows_staged): a separate
// function gets its own register allocation, and inlined the two phases cost the one-CTA batched
// kernel ~160 bytes of spills.
static __device__ __noinline__ bool shift_rows_bulk(uint16_t *E, int pe, int nq, int row0, int rstride, int w, const int32_t *seam,
                                       const uint32_t *pairs, int warp, int nwarps, int lane, unsigned char *buf,
                                       int buf_bytes) {
  uint64_t *bar = reinterpret_cast<uint64_t *>(buf);
  unsigned char *data = buf + 16;
  const int cap = buf_bytes - 16;
  const int c_last = (w - 2) >> 3;   // the chunk holding the new last column
  const int nk = warp < nq ? (nq - warp + nwarps - 1) / nwarps : 0;
  if (nk == 0) return true;
  if (lane == 0) mbar_init(bar, 1);
  fence_mbar_init();
  __syncwarp();
  uint32_t parity = 0;
  bool ok = true;
  for (int k0 = 0; k0 < nk;) {
    const int k = k0 + lane;
    const int q = warp + k * nwarps;
    const int s = k < nk ? seam[row0 + q * rstride] : -1;
    uint16_t *er = E + (size_t)(row0 + (k < nk ? q : 0) * rstride) * pe;
    const int bytes = (k < nk && s >= 0 && s < w - 1) ? 16 * (c_last - (s >> 3) + 2) : 0;
    int incl = bytes;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += t;
    }
    // the rows taken are a prefix of the lanes (incl never decreases)
    const int n = __popc(__ballot_sync(0xffffffffu, k < nk && incl <= cap));
    if (n == 0) {   // the next row's tail alone exceeds the buffer: shifted in place, chunk by chunk
      const int s0 = __shfl_sync(0xffffffffu, s, 0);
      uint16_t *e0 = E + (size_t)(row0 + warp * rstride + k0 * nwarps * rstride) * pe;
      const uint32_t pr = pairs[warp + k0 * nwarps];
      shift_row_u16(e0, s0, w, lane);
      __syncwarp();
      if (lane == 0) {
        if (s0 >= 1) e0[s0 - 1] = (uint16_t)(pr & 0xFFFFu);
        e0[s0] = (uint16_t)(pr >> 16);
      }
      k0 += 1;
      continue;
    }
    const int total = __shfl_sync(0xffffffffu, incl, n - 1);
    const int off = incl - bytes;
    if (total > 0) {
      fence_proxy_async_smem();   // this warp's reads of the buffer's previous round come first
      __syncwarp();
      if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)total);
      __syncwarp();
      if (lane < n && bytes > 0) bulk_g2s(data + off, er + 8 * (s >> 3), (uint32_t)bytes, bar);
      ok = mbar_wait_bounded(bar, parity, WAIT_TIMEOUT_NS);
      parity ^= 1u;
      if (!__all_sync(0xffffffffu, ok)) return false;   // copies may be in flight: the barrier stays
    }
    // a seam in the last column: nothing to shift, only the left refreshed value
    if (lane < n && s == w - 1 && s >= 1) er[s - 1] = (uint16_t)(pairs[q] & 0xFFFFu);
    for (int t = 0; t < n; ++t) {
      const int bt = __shfl_sync(0xffffffffu, bytes, t);
      if (bt == 0) continue;
      const int st = __shfl_sync(0xffffffffu, s, t), ot = __shfl_sync(0xffffffffu, off, t);
      const int qt = warp + (k0 + t) * nwarps;
      uint16_t *et = E + (size_t)(row0 + qt * rstride) * pe;
      const uint16_t *b = reinterpret_cast<const uint16_t *>(data + ot);
      const int c_lo = st >> 3;
      for (int c = c_lo + lane; c <= c_last; c += 32) {
        const uint4 x = *reinterpret_cast<const uint4 *>(b + 8 * (c - c_lo));
        const uint32_t nx = b[8 * (c - c_lo) + 8];
        uint4 o;
        o.x = __funnelshift_r(x.x, x.y, 16);
        o.y = __funnelshift_r(x.y, x.z, 16);
        o.z = __funnelshift_r(x.z, x.w, 16);
        o.w = __funnelshift_r(x.w, nx, 16);
        if (c == c_lo) {
          const int keep = st - 8 * c;   // leading elements of this chunk that stay
          auto merge = [keep](uint32_t in, uint32_t sh, int j) {
            const uint32_t m = (2 * j < keep ? 0x0000FFFFu : 0u) | (2 * j + 1 < keep ? 0xFFFF0000u : 0u);
            return (in & m) | (sh & ~m);
          };
          o.x = merge(x.x, o.x, 0);
          o.y = merge(x.y, o.y, 1);
          o.z = merge(x.z, o.z, 2);
          o.w = merge(x.w, o.w, 3);
        }
        *reinterpret_cast<uint4 *>(et + 8 * c) = o;
        if (c == c_lo) {   // this lane wrote the chunk holding s: the refreshed pair goes over it
          const uint32_t pr = pairs[qt];
          if (st >= 1) et[st - 1] = (uint16_t)(pr & 0xFFFFu);
          et[st] = (uint16_t)(pr >> 16);
        }
      }
    }
    __syncwarp();   // the buffer is reused by the next round
    k0 += n;
  }
  __syncwarp();
  if (lane == 0) mbar_inval(bar);   // the buffer holds other data next
  return ok;
}

// compact_row_lazy for every row this warp owns (local rows q = warp, warp + nwarps, ... of nq;
// image row row0 + q * rstride), staged through a shared-memory buffer of buf_words words
// (16-byte aligned): the stored tail of a row is copied in with cp.async in pieces, then every
// output word is gathered from the buffer. The removals are held one per lane (o_q - q in lane q);
// for 32 consecutive outputs one ballot counts those left of the first and a second finds the few
// that fall inside, instead of comparing every output with every removal.
static __device__ __noinline__ void compact_rows_staged(uint32_t *img, int pitch, int nq, int row0, int rstride,
                                           const int16_t *lists, int m, int w, int warp, int nwarps, int lane,
                                           uint32_t *buf, int buf_words) {
  const int piece = ((buf_words - 24) / 32) * 32;   // outputs per staged piece
  for (int q = warp; q < nq; q += nwarps) {
    const int r = row0 + q * rstride;
    uint32_t *row = img + (int64_t)r * pitch;
    const int16_t *list = lists + (int64_t)r * RPEND;
    if (piece < 32) {   // no room to stage: the direct form
      compact_row_lazy(row, list, m, w, lane);
      continue;
    }
    const int lq = lane < m ? (int)list[lane] - lane : 0x7FFFFFFF;
    const int first = m > 0 ? __shfl_sync(0xffffffffu, lq, 0) : w;   // the list is sorted
    for (int j0 = first; j0 < w; j0 += piece) {
      const int j1 = min(w, j0 + piece);
      const int a = j0 & ~3, b = (j1 + m + 3) & ~3;   // stored words j0 .. j1 + m - 1, 16-byte aligned
      for (int x = a + 4 * lane; x < b; x += 128) cp_async16(buf + (x - a), row + x);
      cp_async_wait_all();
      __syncwarp();
      for (int jb = j0; jb < j1; jb += 32) {
        const int j = jb + lane;
        int c = __popc(__ballot_sync(0xffffffffu, lq <= jb));
        unsigned in = __ballot_sync(0xffffffffu, lq > jb && lq < jb + 32);
        while (in) {
          const int bq = __ffs(in) - 1;
          in &= in - 1;
          const int lv = __shfl_sync(0xffffffffu, lq, bq);
          c += (j >= lv) ? 1 : 0;
        }
        const uint32_t v = (j < j1) ? buf[j + c - a] : 0u;
        __syncwarp();
        if (j < j1) row[j] = v;
      }
      __syncwarp();   // the buffer is reused by the next piece
    }
  }
}

// ---- forward energy ----
// The three cost planes of pixel (i, j) of a rows x cols word image: CU = |P(i,j+1) - P(i,j-1)|
// (0 at the first and last column), DL = |P(i-1,j) - P(i,j-1)| (0 in row 0 and column 0),
// DR = |P(i-1,j) - P(i,j+1)| (0 in row 0 and the last column), each summed over the channels.
// pix(r, c) returns the word of pixel (r, c) (r, c inside the image).
template <typename Pix>
__device__ __forceinline__ void forward_at(Pix pix, int cols, int i, int j, uint32_t &cu, uint32_t &dl, uint32_t &dr) {
  const bool left = j >= 1, right = j + 1 < cols;
  const uint32_t pl = left ? pix(i, j - 1) : 0u, pr = right ? pix(i, j + 1) : 0u;
  cu = (left && right) ? sad4(pr, pl) : 0u;
  dl = dr = 0u;
  if (i >= 1) {
    const uint32_t up = pix(i - 1, j);
    if (left) dl = sad4(up, pl);
    if (right) dr = sad4(up, pr);
  }
}

// The forward-energy planes at the new columns s-1 and s of row i after removing `seam` (the
// other columns are shifted copies: the dirty set of the e1 refresh holds for all three planes),
// the image read through the pending-removal lists. out[plane] = value(s-1) | value(s) << 16.
__device__ __forceinline__ void patch_row_lazy_fwd(const uint32_t *img, int pitch, int H, int W, const int32_t *seam,
                                                   const int16_t *lists, int m, int i, uint32_t (&out)[3], bool *bad,
                                                   LazyRow *li) {
  const int Wn = W - 1;
  const int iu = i > 0 ? i - 1 : 0;
  const int s = seam[i], su = seam[iu];
  const LazyRow lc = lazy_row(lists + (int64_t)i * RPEND, m);
  const LazyRow lu = lazy_row(lists + (int64_t)iu * RPEND, m);
  *li = lc;
  out[0] = out[1] = out[2] = 0u;
  if (s < 0 || s >= W) {
    *bad = true;
    return;
  }
  // rows i (forward_at's row) and i - 1 (read only when i >= 1)
  auto pix = [&](int r, int j) -> uint32_t {
    const LazyRow &L = r == i ? lc : lu;
    const int x = j + (j >= (r == i ? s : su) ? 1 : 0);      // column in the width-W image
    return img[(int64_t)r * pitch + x + lazy_count(L, x)];
  };
  uint32_t cu, dl, dr;
  if (s >= 1) {
    forward_at(pix, Wn, i, s - 1, cu, dl, dr);
    out[0] = cu; out[1] = dl; out[2] = dr;
  }
  if (s <= Wn - 1) {
    forward_at(pix, Wn, i, s, cu, dl, dr);
    out[0] |= cu << 16; out[1] |= dl << 16; out[2] |= dr << 16;
  }
}

// refresh_row for the three forward-energy planes (plane p at E + p * pstride)
__device__ __forceinline__ bool refresh_row_fwd(const uint32_t *img, int pitch, uint16_t *E, int pe, int64_t pstride,
                                                int H, int W, const int32_t *seam, const int16_t *lists_in,
                                                int16_t *lists_out, int m, int i, int lane) {
  const int s = seam[i];
  if (s < 0 || s >= W) return false;
  uint32_t pr[3] = {0u, 0u, 0u};
  if (lane == 0) {
    bool bad = false;
    LazyRow li;
    patch_row_lazy_fwd(img, pitch, H, W, seam, lists_in, m, i, pr, &bad, &li);
    list_insert(li, lists_out + (int64_t)i * RPEND, s);
  }
#pragma unroll
  for (int pl = 0; pl < 3; ++pl) {
    const uint32_t v = __shfl_sync(0xffffffffu, pr[pl], 0);
    uint16_t *er = E + pl * pstride + (int64_t)i * pe;
    shift_row_u16(er, s, W, lane);
    if (lane == 0) {
      if (s >= 1) er[s - 1] = (uint16_t)(v & 0xFFFFu);
      if (s <= W - 2) er[s] = (uint16_t)(v >> 16);
    }
  }
  return true;
}

}  // namespace sc
