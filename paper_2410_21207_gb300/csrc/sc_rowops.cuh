// Per-pixel and per-row operations shared by the whole-image kernels (sc_kernels.cu) and the
// batched persistent kernel (sc_batch.cuh): the e1 energy of a pixel ("Energy Mapping", item e1),
// the two refreshed energies of a row after a removal, and the in-place row compaction ("Removal of
// Seams"). Pixels are uint32 words, channel c in byte c (unused bytes 0).
#pragma once
#include <cstdint>

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

// The two energies of row i that the removal of `seam` changes. After deleting seam s from a
// W-wide image, the energy of the (W-1)-wide image equals the old energy shifted left past s_i,
// except at the new columns s_i - 1 and s_i (their left/right neighbour changed, and, since
// |s_i - s_(i+-1)| <= 1, they are the only pixels whose upper/lower neighbour can change). They
// are computed from the old image seen through the removal: new pixel (r, j) = old (r, j + [j >= s_r]).
// Returns (e(s-1) | e(s) << 16); a value is 0 when its column does not exist. *bad is set when
// the seam column is out of range.
__device__ __forceinline__ uint32_t patch_row(const uint32_t *img, int pitch, int H, int W, const int32_t *seam,
                                              int i, bool *bad) {
  const int Wn = W - 1;
  const int s = seam[i];
  if (s < 0 || s >= W) {
    *bad = true;
    return 0u;
  }
  auto pix = [&](int r, int j) -> uint32_t {
    r = clampi(r, 0, H - 1);
    j = clampi(j, 0, Wn - 1);
    const int sr = seam[r];
    return img[(int64_t)r * pitch + j + (j >= sr ? 1 : 0)];
  };
  auto en = [&](int j) -> uint32_t { return sad4(pix(i, j + 1), pix(i, j - 1)) + sad4(pix(i + 1, j), pix(i - 1, j)); };
  const uint32_t p0 = (s >= 1) ? en(s - 1) : 0u;
  const uint32_t p1 = (s <= Wn - 1) ? en(s) : 0u;
  return p0 | (p1 << 16);
}

// In-place left shift by one of row[s+1 .. W-1] -> row[s .. W-2] by one warp: left to right in
// chunks of 32*R elements, every chunk read completely (by all lanes) before any lane writes it,
// so no element is overwritten before it has been read.
template <typename T>
__device__ __forceinline__ void shift_row(T *row, int s, int W, int lane) {
  constexpr int R = 8;
  for (int base = s; base < W - 1; base += 32 * R) {
    T x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int j = base + r * 32 + lane;
      x[r] = (j + 1 < W) ? row[j + 1] : T(0);
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int j = base + r * 32 + lane;
      if (j < W - 1) row[j] = x[r];
    }
    __syncwarp();
  }
}

// Compaction of row i of the image words and of the energy, then the two refreshed energies.
__device__ __forceinline__ void compact_row(uint32_t *img, int pitch, uint16_t *E, int pe, int W, int s,
                                            uint32_t patch, int i, int lane) {
  shift_row(img + (int64_t)i * pitch, s, W, lane);
  uint16_t *er = E + (int64_t)i * pe;
  shift_row(er, s, W, lane);
  if (lane == 0) {
    if (s >= 1) er[s - 1] = (uint16_t)(patch & 0xFFFFu);
    if (s <= W - 2) er[s] = (uint16_t)(patch >> 16);
  }
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
