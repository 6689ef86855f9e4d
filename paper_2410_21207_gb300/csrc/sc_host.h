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
               int64_t *cost_log, cudaStream_t st, bool forward = false);
int *device_error_word();
// errors recorded by sc_find_seam_static calls on the current device and not yet reported (read and
// cleared; 0 when no static call ran on the device)
int static_pending_errors(int *bits);

struct BatchCfg {
  int nw, kt;
  // load balance: an image whose estimated carving time on one CTA exceeds thr_bal x the whole
  // batch's mean share per SM is carved by a cluster of the latency shape (CL_LAT, at least 2 CTAs)
  // instead of one CTA, so that it does not hold up the batch (0: off)
  float thr_bal = 0.f;
  // images wider than one CTA take the latency shape too (where 16 CTAs of it cover them): the
  // serving form, whose widest requests set its tail latency
  bool wide_lat = false;
  // images whose estimated carving time on one CTA exceeds lat_us microseconds take the latency
  // shape as well (0: off): the serving form's heaviest narrow requests
  float lat_us = 0.f;
  // SMs the balancing share is computed over (0: the current device's)
  int sms = 0;
};
// images carved by the cluster-per-image batched kernel: those wider than one CTA (CL_WIDE
// shape) and the heaviest ones of a balanced plan (CL_LAT); one group per shape and cluster size
struct ClusterGroup {
  int shape = 0;   // ClShape
  int cs = 1;
  int Smax = 1;
  std::vector<BatchItem> items;
  std::vector<int> index;         // descriptor index of each item
};
struct BatchSetup {
  std::vector<BatchItem> items;   // images carved by one CTA each (device pointers filled in)
  std::vector<ClusterGroup> cl;   // images carved by one cluster each
  std::vector<int> fallback;      // descriptor indices carved by the per-seam cluster path
  size_t pool_bytes = 0;
  int Smax = 1;
  int cluster_images() const {
    int n = 0;
    for (const ClusterGroup &g : cl) n += (int)g.items.size();
    return n;
  }
};
inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// widest searched width of an image (its width, or its height when it has horizontal seams)
int batch_need_width(const sc_image_desc &d);
void batch_layout(const sc_image_desc *descs, int n, const BatchCfg &c, unsigned char *pool, BatchSetup &b);
// CTAs in the cluster that carves an image wider than one CTA
int batch_cluster_size(const sc_image_desc &d);

}  // namespace sc
