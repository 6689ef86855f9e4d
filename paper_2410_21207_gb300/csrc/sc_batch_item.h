// One image of a batched carve, as the persistent kernel reads it (device pointers).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sc {

struct BatchItem {
  const uint8_t *img;   // H x W x C uint8 (caller's)
  uint8_t *out;         // th x tw x C uint8 (caller's)
  int32_t *seam_log;    // nullable (caller's)
  int64_t *cost_log;    // nullable
  int H, W, C, tw, th;
  int pitch;            // words per row of img_w / img2_w (>= max(H, W))
  int pe;               // energy pitch (elements)
  int pad;
  uint32_t *img_w;      // max(H,W) x pitch words: the image being carved
  uint32_t *img2_w;     // max(H,W) x pitch words: its transpose for the horizontal pass
  uint16_t *E;          // rows x pe energies (column 0 at E + E_PADL)
  uint32_t *Mrow;       // (ceil(rows/KS) + 1) x pe saved cost rows (column 0 at Mrow + E_PADL)
  int32_t *seam;        // rows
  int16_t *lists;       // two generations of pending-removal lists, rows x RPEND each
  // nullable: set to 1 (or 2 if the device error word was non-zero) once `out` is complete and
  // visible to the host; `out` may then be host-mapped memory (the serving form)
  int *done;
};

// width a CTA of nw compute warps with tile height kt covers
inline int batch_width_limit(int nw, int kt) { return nw * (128 - 2 * kt); }

// pdl: launched as a programmatic dependent of the launch before it on st (which must trigger its
// dependents at its start); the kernel does not end before that launch does
cudaError_t launch_batch(int nw, int kt, const BatchItem *items, int n, int Smax, int grid, int *queue, int *err,
                         cudaStream_t st, bool pdl = false);
size_t batch_smem_bytes(int nw, int kt, int Smax);
int batch_blocks_per_sm(int nw, int kt, int Smax);   // after the kernel's smem attribute is set

}  // namespace sc
