// Host-side helpers shared by the C-ABI files (not part of the C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sc.h"
#include "sc_batch_item.h"

namespace sc {

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int check_carve_args(const void *img, int H, int W, int C, int tw, int th, const void *out);
// the cluster path of sc_carve on `st` (uses the stream's workspace)
int carve_impl(const uint8_t *img, int H, int W, int C, int tw, int th, uint8_t *out, int32_t *seam_log,
               int64_t *cost_log, cudaStream_t st);
int *device_error_word();

struct BatchCfg {
  int nw, kt;
};
struct BatchSetup {
  std::vector<BatchItem> items;   // batched images (device pointers filled in)
  std::vector<int> fallback;      // descriptor indices carved by the cluster path
  size_t pool_bytes = 0;
  int Smax = 1;
};
inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// widest searched width of an image (its width, or its height when it has horizontal seams)
int batch_need_width(const sc_image_desc &d);
void batch_layout(const sc_image_desc *descs, int n, const BatchCfg &c, unsigned char *pool, BatchSetup &b);

}  // namespace sc
