// Internal declarations of libsc_gb300 (not part of the C ABI).
//
// Device data layout (one image being carved):
//   img   : uint32 per pixel (channel c in byte c, unused bytes 0), H rows x pitch_img words.
//           Kept in the current (carved) coordinates.
//   E     : uint16 energy, H rows x pitch_e elements; column j of row i lives at
//           E + i*pitch_e + E_PADL + j. The pads keep every window load of the seam search in
//           bounds; their contents are never used for a result.
//   Mrow  : uint32 cost-table rows saved at super-tile boundaries (see sc_dp.cu), same padding.
//   seam  : int32[H]; patch: uint32[H] (the two refreshed energies of a row, low/high half).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sc {

constexpr int E_PADL = 256;    // left pad (elements) of E and Mrow rows
constexpr int E_PADR = 1024;   // right pad (elements)

// Seam-search geometry (sc_search.cuh). A lane owns V consecutive columns; a warp's window is
// 32*V columns, of which 32*V - 2*KT are its own strip; windows exchange boundary rows every KT
// rows inside a CTA (shared memory) and every K2 rows between the CTAs of a cluster (DSMEM).
// Ancestors are tracked over super-tiles of KS rows; the single-map search of maps wider than a
// 4-warp cluster covers uses KS_WIDE (its ancestor chain reads other CTAs through DSMEM, one load per
// super-tile). Buffers of saved cost rows are sized for KS, the shorter. KT is a template
// parameter of each kernel.
constexpr int V = 4;
constexpr int KS = 32;
constexpr int KS_WIDE = 64;
constexpr int K2 = 64;
constexpr int MAX_CLUSTER = 16;

// Error bits recorded on the device.
constexpr int ERR_FILL_MISMATCH = 1;   // backtrack fill disagrees with the ancestor chain
constexpr int ERR_COST_MISMATCH = 2;   // recomputed cost disagrees with the argmin
constexpr int ERR_ENERGY_RANGE = 4;    // gate bit: seam sums may not fit the 24-bit cost field (not an error)
constexpr int ERR_TIMEOUT = 8;         // a bounded wait ran out
constexpr int ERR_BAD_SEAM = 16;       // a seam column out of range

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
inline int pitch_e_for(int W) { return E_PADL + round_up(W, 8) + E_PADR; }

struct DpShape {
  int nw;    // compute warps per CTA
  int kt;    // DP tile rows
  int cs;    // CTAs in the cluster
  int ow;    // CTA-own columns = nw*Q - 2*K2
};
DpShape dp_shape_for(int W);

struct DpArgs {
  const uint16_t *E;   // row 0, column 0 (already offset by E_PADL)
  int pitch_e;
  int H, W;
  uint32_t *Mrow;      // super-tile boundary rows, row s at Mrow + s*pitch_m (offset by E_PADL)
  int32_t *seam;       // out [H]
  int32_t *seam_log;   // nullable, out [H]
  int64_t *cost;       // nullable, out [1]
  int *err;            // device error word
  int *gate;           // nullable: with ERR_ENERGY_RANGE set the 24-bit search skips the map and the
                       // wide-cost search takes it (the multi-map search also sets it itself)
  int64_t pstride = 0; // forward energy: elements between the CU, DL, DR planes (0: the e1 map)
  int pitch_m = 0;     // row stride of Mrow (0: pitch_e)
};

// Launchers (enqueue on `st`; return cudaError_t of the launch).
cudaError_t launch_pack(const uint8_t *src, int H, int W, int C, uint32_t *img, int pitch_img, cudaStream_t st);
cudaError_t launch_unpack(const uint32_t *img, int pitch_img, int H, int W, int C, bool transposed, uint8_t *dst,
                          cudaStream_t st);
cudaError_t launch_transpose(const uint32_t *src, int pitch_src, int H, int W, uint32_t *dst, int pitch_dst,
                             cudaStream_t st);
cudaError_t launch_energy(const uint32_t *img, int pitch_img, int H, int W, uint16_t *E, int pitch_e, cudaStream_t st);
// caller map -> padded layout; sets *gate (ERR_ENERGY_RANGE) when a seam sum might not fit 24 bits
cudaError_t launch_copy_energy(const uint16_t *src, int H, int W, uint16_t *E, int pitch_e, int *gate, cudaStream_t st);
cudaError_t launch_unpad_energy(const uint16_t *E, int pitch_e, int H, int W, uint16_t *dst, cudaStream_t st);
// forward energy: the CU, DL, DR planes of a word image, or of a caller's planes (with the range
// gate and the unused border entries zeroed), plane p at E + p * pstride
cudaError_t launch_forward(const uint32_t *img, int pitch, int H, int W, uint16_t *E, int pitch_e, int64_t pstride,
                           cudaStream_t st);
cudaError_t launch_copy_planes(const uint16_t *cu, const uint16_t *dl, const uint16_t *dr, int H, int W, uint16_t *E,
                               int pitch_e, int64_t pstride, int *gate, cudaStream_t st);
cudaError_t launch_refresh_fwd(const uint32_t *img, int pitch, uint16_t *E, int pe, int64_t pstride, int H, int W,
                               const int32_t *seam, const int16_t *lists_in, int16_t *lists_out, int m, int *err,
                               cudaStream_t st);
cudaError_t launch_dp(const DpArgs &a, cudaStream_t st);   // forward energy when a.pstride > 0
// The wide-cost search (sc_dp_wide.cu): one CTA per map, exact 32-bit costs, for the maps whose
// gate is set (it returns at once for the others). Scratch per map: wide_dirs_words(H, W) uint32
// direction words and wide_anc_elems(H, W) uint16 ancestors. Forward energy when a.pstride > 0
// (W <= 4096); the multi-map form takes a device array of n DpArgs of one size (e1 only).
cudaError_t launch_dp_wide(const DpArgs &a, uint32_t *dirs, uint16_t *anc, cudaStream_t st);
struct MultiArgs;
cudaError_t launch_dp_wide_multi(const DpArgs *dargs_dev, const MultiArgs *inl, int n, int H, int W, uint32_t *dirs,
                                 uint16_t *anc, cudaStream_t st);
size_t wide_dirs_words(int H, int W);
size_t wide_anc_elems(int H, int W);
int dp_forward_max_width();                                 // widest map the forward search takes
// n searches of H x W maps in one launch (one cluster each); dargs_dev is a device array. The maps
// are read in place (E = row 0, column 0; pitch_e a multiple of 8; 16-byte aligned rows) and each
// map's 24-bit cost range is checked in the kernel: a map that fails sets its gate and is left to
// launch_dp_wide_multi
// Up to MULTI_INLINE maps' arguments travel in the launch itself (a __grid_constant__ parameter):
// no host-to-device copy per call. `inl` (host) is used when non-null, else `dargs_dev`.
constexpr int MULTI_INLINE = 64;
struct MultiArgs {
  DpArgs a[MULTI_INLINE];
};
cudaError_t launch_dp_multi(const DpArgs *dargs_dev, const MultiArgs *inl, int n, int H, int W, cudaStream_t st);
// how many H x W searches of launch_dp_multi are resident on the GPU at once
cudaError_t dp_multi_capacity(int H, int W, int *n_out);
// tile shape of launch_dp_multi: (compute warps per CTA, tile rows), (0, 0) = automatic;
// returns -1 for a shape that is not built
int dp_multi_set_shape(int nw, int kt);
// Algorithm 2's greedy seam of an unpadded H x W map (one warp)
cudaError_t launch_greedy(const uint16_t *e, int H, int W, int32_t *seam, int64_t *cost, cudaStream_t st);
// seam insertion (sc_enlarge.cu): seam log -> per-row bitmap of the input columns to widen at
// (cols, nullable, receives them seam by seam); then the widened image
cudaError_t launch_enlarge_map(const int32_t *log, int H, int W, int k, uint32_t *bits, int32_t *cols, int *err,
                               cudaStream_t st);
cudaError_t launch_insert(const uint8_t *img, int H, int W, int C, const uint32_t *bits, uint8_t *out, int tw,
                          cudaStream_t st);
// one bounded mbarrier wait that nothing completes (failure-detection self-test)
cudaError_t launch_wait_selftest(uint64_t limit_ns, int *err, cudaStream_t st);
// lazy image compaction (sc_rowops.cuh): refresh + list update per seam, bulk compaction
cudaError_t launch_compact_lazy(uint32_t *img, int pitch, int H, int w, const int16_t *lists, int m, cudaStream_t st);
// per seam: refreshed pair through the lazy map, list update and energy compaction (one warp per row)
cudaError_t launch_refresh(const uint32_t *img, int pitch, uint16_t *E, int pe, int H, int W, const int32_t *seam,
                           const int16_t *lists_in, int16_t *lists_out, int m, int *err, cudaStream_t st);

}  // namespace sc
