/*
 * sc.h — C ABI of the GB300 (sm_103a) seam-carving library libsc_gb300.so.
 *
 * The operations follow arXiv 2410.21207 ("Analysis of Different Algorithmic Design Techniques
 * for Seam Carving"): the e1 energy (section "Energy Mapping"), the minimum vertical seam by the
 * dynamic-programming recurrence M(i,j) = e(i,j) + min(M(i-1,j-1), M(i-1,j), M(i-1,j+1))
 * (section "DP Seam Carving", Algorithm 3), removal of the seam by shifting each row left past it
 * (section "Removal of Seams"), and horizontal seams as vertical seams of the transposed image
 * (section "Design Techniques"). Integer arithmetic throughout:
 *   - images are uint8, H rows x W columns x C channels, row-major (HWC), C in {1, 3, 4};
 *   - e(i,j) = sum over channels of |I(i,j+1)-I(i,j-1)| + |I(i+1,j)-I(i-1,j)|, neighbour indices
 *     clamped to the image (edge replication); e <= 2*255*C fits uint16;
 *   - M is exact (int32 range); M(0,j) = e(0,j); neighbours outside the image are excluded;
 *   - ties: the leftmost of (j-1, j, j+1) wins, and the leftmost minimum of the last row wins;
 *   - a seam is int32 seam[H], seam[i] = its column in row i, in the coordinates of the image it
 *     was found in.
 * These fix one unique answer, so every seam and every output byte is reproducible bit for bit.
 *
 * Conventions for every entry point:
 *   - Pointers are DEVICE pointers owned by the caller unless the name ends in _host. The library
 *     never frees or keeps them after the call's work has finished on `stream`.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Work is
 *     enqueued asynchronously on it; argument errors are returned synchronously, before any work
 *     is enqueued.
 *   - The library owns internal scratch (a workspace per (device, stream), grown on demand with
 *     cudaMalloc and kept until sc_release_workspaces or exit). Calls on the same stream reuse it
 *     in order; calls on different streams use different workspaces.
 *   - Errors detected on the device (a failed internal consistency check, a bounded wait that
 *     ran out) are recorded in the workspace and reported by sc_check(stream), which waits for
 *     the stream.
 *   - Return value: SC_OK (0) or a negative sc_status. sc_last_error() describes the last failure
 *     of the calling thread.
 *   - Limits: 1 <= H, W; H <= SC_MAX_ROWS; W <= SC_MAX_COLS; H*W*C < 2^31. Seam costs are exact
 *     for every uint16 energy map of these sizes (they stay below 2^31).
 */
#ifndef SC_GB300_H
#define SC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SC_OK = 0,
  SC_EINVAL = -1,    /* bad argument (null pointer, size out of range, enlargement) */
  SC_ENOMEM = -2,    /* device or host allocation failed */
  SC_ECUDA = -3,     /* a CUDA runtime call failed (message in sc_last_error) */
  SC_ETIMEOUT = -4,  /* a bounded device-side wait ran out; the context is still usable */
  SC_EBUSY = -5,     /* a serving queue is full */
  SC_EINTERNAL = -6  /* a device-side consistency check failed */
} sc_status;

#define SC_MAX_ROWS 8192
#define SC_MAX_COLS 8192

/* Library version (major*10000 + minor*100 + patch). */
int sc_version(void);

/* Message for the last failing call on this thread (static storage, never NULL). */
const char *sc_last_error(void);

/* Wait for `stream` and report device-side errors recorded by earlier calls on it, by batched
 * launches on the current device, and by sc_find_seam_static calls on the current device whose work
 * has finished (and clear them). Returns SC_OK, SC_ETIMEOUT (a bounded wait ran out; takes
 * precedence), SC_EINTERNAL (a consistency check failed) or SC_ECUDA. */
int sc_check(void *stream);

/* Free every workspace the library holds for the current device (after synchronising it). */
int sc_release_workspaces(void);

/* ---- instrumentation (no counterpart in the paper) ----
 * sc_timing_enable(1) makes the library bracket every launch of the named kernels with CUDA
 * events on the launching stream and count every kernel launch it makes; sc_timing_read waits
 * for the recorded events and returns the summed device time (ms) and launch count of one kernel
 * ("dp", "patch", "shift", "energy", "transpose", "pack", "unpack", "carve_batch") or, for
 * kernel = "all", the total number of kernel launches (total_ms = 0). sc_timing_reset clears the
 * records. Off by default; meant for benchmarks, not for concurrent use from several threads. */
int sc_timing_enable(int on);
int sc_timing_reset(void);
int sc_timing_read(const char *kernel, double *total_ms, int64_t *launches);

/* Copy-bandwidth probe (instrumentation, no counterpart in the paper): allocates two device
 * buffers of `bytes` each, copies one into the other `reps` times within ONE kernel launch (so the
 * time is the copies' own, not the gaps between short launches), times that launch with CUDA events
 * on the legacy default stream after a warm-up launch, and returns read + write bytes per second
 * in GB/s. With both buffers inside L2 (2 x 32 MiB against a 126 MB L2) it measures the L2 copy
 * bandwidth; with buffers far larger than L2, the HBM copy bandwidth. Synchronous; frees what it
 * allocates. Errors: SC_EINVAL for bytes < 4096 or not a multiple of 16, reps outside 1..10000;
 * SC_ECUDA for a failed CUDA call. */
int sc_probe_copy_bandwidth(size_t bytes, int reps, double *gbs_out);

/* ---- e1 energy (section "Energy Mapping", item e1) ----
 * img:        device, H x W x C uint8, row-major.
 * energy_out: device, H x W uint16, row-major; written completely.
 * Errors: SC_EINVAL if a pointer is NULL, H < 1, W < 1, C not in {1,3,4} or H*W*C >= 2^31. */
int sc_energy(const uint8_t *img, int H, int W, int C, uint16_t *energy_out, void *stream);

/* ---- one minimum vertical seam (section "DP Seam Carving", Algorithm 3, with the readings in
 * the header comment) ----
 * energy:   device, H x W uint16, row-major; any values.
 * seam_out: device, int32[H]; seam_out[i] in [0, W), |seam_out[i] - seam_out[i-1]| <= 1.
 * cost_out: device, int64[1] or NULL: the seam's total energy (the minimum of M's last row).
 * The fast search packs each cost with its backtrack ancestor into 32 bits, which holds costs
 * below 2^24; while copying the map the library checks H * max(e) < 2^24 on the device, and a map
 * that fails it is searched instead by a slower kernel with exact 32-bit costs (one CTA, about
 * 0.1 ms per 1080 x 1920 map). Both give the same seam and cost; nothing is refused.
 * Errors: SC_EINVAL for NULL energy/seam_out, H < 1, W < 1, H > SC_MAX_ROWS, W > SC_MAX_COLS;
 *         device-side check failures via sc_check. */
int sc_find_seam(const uint16_t *energy, int H, int W, int32_t *seam_out, int64_t *cost_out, void *stream);

/* ---- forward energy (the paper cites it as an alternative to e1 without a formula) ----
 * Reading implemented: a seam costs the sum, over the pixel pairs its removal makes adjacent, of
 * their L1 colour difference. Per pixel (i, j): CU = |I(i,j+1) - I(i,j-1)| (0 at the first and
 * last column), DL = |I(i-1,j) - I(i,j-1)| (0 in row 0 / column 0), DR = |I(i-1,j) - I(i,j+1)|
 * (0 in row 0 / the last column), channels summed. Algorithm 3 with direction-dependent costs:
 * M(0,j) = CU(0,j); M(i,j) = CU(i,j) + min(M(i-1,j-1) + DL(i,j), M(i-1,j), M(i-1,j+1) + DR(i,j)),
 * leftmost ties, leftmost last-row minimum.
 * sc_forward_costs: the three uint16 H x W planes of a device image (C in {1,3,4}).
 * sc_find_seam_forward: the seam of caller planes (device uint16 H x W each; DL/DR entries with no
 *   predecessor are ignored); W <= 4096; any values (a map whose H * max(CU + max(DL, DR)) could
 *   reach 2^24 goes to the exact wide-cost search, as in sc_find_seam).
 * sc_carve_forward: sc_carve with forward energy (same arguments, seam and cost logs); every
 *   searched width (W, and H when target_h < H) must be <= 4096.
 * All asynchronous on `stream`. Errors: SC_EINVAL for null pointers or shapes out of range; device
 * errors via sc_check. */
int sc_forward_costs(const uint8_t *img, int H, int W, int C, uint16_t *cu, uint16_t *dl, uint16_t *dr, void *stream);
int sc_find_seam_forward(const uint16_t *cu, const uint16_t *dl, const uint16_t *dr, int H, int W, int32_t *seam_out,
                         int64_t *cost_out, void *stream);
int sc_carve_forward(const uint8_t *img, int H, int W, int C, int target_w, int target_h, uint8_t *out,
                     int32_t *seam_log, int64_t *cost_log, void *stream);

/* ---- failure-detection self-test (the paper has no counterpart) ----
 * Enqueues one kernel whose single wait, the same bounded mbarrier wait the seam search uses,
 * waits for an arrival that never comes; after limit_us (1 .. 1e6) it records a timeout in the
 * stream's device error word and returns normally. The next sc_check(stream) then returns
 * SC_ETIMEOUT, and the stream and context stay usable. Errors: SC_EINVAL for a limit out of range. */
int sc_selftest_wait_timeout(int limit_us, void *stream);

/* ---- seam insertion: widening by k = target_w - W seams (1 <= k <= W-1) ----
 * The paper names enlargement by seams ("Seam Carving" background) without giving its steps; the
 * reading implemented: take the first k seams that sc_carve(img, W - k, H) removes (Algorithm 3
 * on each shrinking image), map each back to the input column it deletes in every row, and after
 * every input pixel in one of those columns insert a pixel whose channels are the rounded-up mean
 * (a + b + 1) / 2 of it and its right neighbour (the pixel itself at the last column).
 * img: device H x W x C uint8 (C in {1,3,4}); out: device H x target_w x C; cols_out: device
 * int32[k*H] or NULL, receiving the mapped input column of seam t in row i at t*H + i.
 * Asynchronous on `stream`; uses the stream's workspace. Errors: SC_EINVAL for a null pointer, a
 * bad shape or channel count, or target_w outside (W, 2W); device errors via sc_check. */
int sc_enlarge(const uint8_t *img, int H, int W, int C, int target_w, uint8_t *out, int32_t *cols_out, void *stream);

/* ---- Algorithm 2 (section "Greedy Seam Carving"): the greedy seam ----
 * Starts at the leftmost minimum of the bottom row and climbs, row by row, to the leftmost minimum
 * of the in-range upper neighbours (j-1, j, j+1); cost = the sum of the energies on the seam.
 * Not optimal in general (the DP seam's cost is a lower bound); the paper compares it with the DP.
 * energy: device uint16 H x W row-major; seam_out: device int32[H]; cost_out: device int64 or
 * NULL. Asynchronous on `stream`. Errors: SC_EINVAL for a null pointer or a shape outside
 * 1..SC_MAX_ROWS x 1..SC_MAX_COLS. */
int sc_greedy_seam(const uint16_t *energy, int H, int W, int32_t *seam_out, int64_t *cost_out, void *stream);

/* ---- the same search for n independent maps of one size, in one launch ----
 * The Algorithm 3 seam (DP fill, last-row argmin, backtrack) of each map, independently.
 * energies: HOST array of n DEVICE pointers, each H x W uint16 row-major (as sc_find_seam).
 * seams_out: device int32[n*H] (map k's seam at seams_out + k*H); costs_out: device int64[n] or
 * NULL. One thread-block cluster per map; the clusters share the GPU, so with several maps in
 * flight the pass is bound by memory bandwidth rather than by one map's chain of dependent rows.
 * Results equal n calls of sc_find_seam (each map's energy range is checked on its own; maps that
 * fail it go to the wide-cost search). Errors: as sc_find_seam; n < 1 -> SC_EINVAL. */
int sc_find_seam_multi(const uint16_t *const *energies, int n, int H, int W, int32_t *seams_out, int64_t *costs_out,
                       void *stream);

/* How many H x W searches of sc_find_seam_multi are resident on the current device at once
 * (thread-block clusters that fit together); a batch of that many maps fills the GPU. */
int sc_find_seam_multi_capacity(int H, int W, int *n_out);

/* Tile shape of sc_find_seam_multi: compute warps per CTA (4 or 8) and DP tile rows (8 or 16);
 * (0, 0) restores the automatic choice. Process-wide. Any other pair -> SC_EINVAL. */
int sc_find_seam_multi_shape(int warps, int tile_rows);

/* ---- sc_find_seam without allocation (the paper has no counterpart: this is a deployment aid) ----
 * For programs that must not let a library allocate device memory: cudaMalloc/cudaFree can
 * synchronise the device and take unpredictable time inside a latency-critical loop, and hosts
 * that budget every device byte through their own allocator forbid allocations they do not
 * control. Same arguments and result as sc_find_seam (any uint16 map, exact seam and cost), but
 * every scratch byte (a padded copy of the energy map, the saved cost rows, the wide-cost search's
 * directions and ancestors, three status words) lives in one fixed array of 32 MiB inside the
 * library's device image, held by every GPU that loads the library until the process exits; the
 * call never calls cudaMalloc or cudaFree. Differences from sc_find_seam:
 *   - Size limit: the map must fit the array, roughly H * (W + 1280) * 2.3 bytes plus one row of
 *     4-byte costs per 32 rows (3840 x 2160 fits). A larger map returns SC_EINVAL (sc_last_error
 *     names the bytes needed) before any work is enqueued.
 *   - Device-side errors (a bounded wait that ran out, a failed self-check) are reported twice:
 *     through the outputs (every seam_out entry, and *cost_out when given, set to -1) and by the
 *     next sc_check on any stream of the device once the call's work has finished.
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress);
 *     make that first call before any stream capture.
 *   - All calls share the one array, which keeps the previous call's contents: calls whose work
 *     overlaps on the GPU (different streams, or different host threads) race and must be
 *     serialised by the caller. Each call clears its own status words first.
 * Argument errors: SC_EINVAL as sc_find_seam; a failed CUDA call returns SC_ECUDA. */
int sc_find_seam_static(const uint16_t *energy, int H, int W, int32_t *seam_out, int64_t *cost_out, void *stream);

/* Failure-detection self-test of sc_find_seam_static's error path (no counterpart in the paper).
 * Enqueues what a static call does when its device work fails, without a fault: it clears the
 * call's status words, runs the bounded mbarrier wait of the seam search on a barrier that nothing
 * completes (recording a timeout after limit_us, 1 .. 1e6), then the completion step of every
 * static call, which sets seam_out[0 .. H) and *cost_out (when given) to -1 and leaves the timeout
 * for the next sc_check (SC_ETIMEOUT). Errors: SC_EINVAL for a limit or H out of range or a null
 * seam_out. */
int sc_find_seam_static_selftest(int limit_us, int H, int32_t *seam_out, int64_t *cost_out, void *stream);

/* ---- carve: remove (W - target_w) vertical seams, then (H - target_h) horizontal seams (found
 * as vertical seams of the transposed image), recomputing the energy where the removal changed
 * it (sections "Removal of Seams" and "Design Techniques"). The result equals: for each seam,
 * recompute the full e1 energy, find the Algorithm 3 seam, delete it.
 * img:      device, H x W x C uint8 (not modified).
 * out:      device, target_h x target_w x C uint8.
 * seam_log: device int32 or NULL. When given it receives (W - target_w) vertical seams of H
 *           entries each (in the coordinates of the image each was found in), followed by
 *           (H - target_h) horizontal seams of target_w entries each (in the transposed frame:
 *           entry r is the row removed from column r).
 * cost_log: device int64 or NULL: one cost per removed seam, in the same order.
 * Errors: SC_EINVAL for NULL img/out, C not in {1,3,4}, target_w < 1, target_h < 1,
 *         target_w > W or target_h > H (no enlargement), H or W above the limits. */
int sc_carve(const uint8_t *img, int H, int W, int C, int target_w, int target_h, uint8_t *out,
             int32_t *seam_log, int64_t *cost_log, void *stream);

/* Same result as sc_carve, computed by the plain path: one image at a time with separate kernel
 * launches for every seam (find, refresh, compact), no persistent kernel and no graph. It is the
 * baseline the persistent/batched forms are measured against. Same arguments and errors. */
int sc_carve_plain(const uint8_t *img, int H, int W, int C, int target_w, int target_h, uint8_t *out,
                   int32_t *seam_log, int64_t *cost_log, void *stream);

/* sc_carve with HOST buffers: img (H*W*C bytes) and out (target_h*target_w*C bytes) are host
 * pointers (pinned memory is fastest); the call copies in, carves and copies out on `stream`, and
 * returns after the result is in `out` (it synchronises the stream). Device errors are returned
 * directly. Same limits as sc_carve. */
int sc_carve_host(const uint8_t *img_host, int H, int W, int C, int target_w, int target_h, uint8_t *out_host,
                  void *stream);

/* ---- batched form: many images of uneven sizes carved by one persistent launch ----
 * Each descriptor names one image; all pointers are device pointers. Images are processed
 * independently and each result equals sc_carve on that image alone. */
typedef struct {
  const uint8_t *img;   /* H x W x C uint8 */
  uint8_t *out;         /* target_h x target_w x C uint8 */
  int32_t *seam_log;    /* NULL or as in sc_carve */
  int H, W, C;
  int target_w, target_h;
  int reserved;
} sc_image_desc;

/* descs: HOST array of n descriptors (copied during the call). One persistent launch: each CTA
 * takes the next image from a queue and carves it completely (energy, every seam's search,
 * refresh and compaction, the transposed horizontal pass). Images whose searched width exceeds
 * what one CTA covers (1440 columns in the default configuration) are carved by the cluster path
 * of sc_carve on the same stream. The call waits for the previous batch on `stream` before reusing
 * its scratch. Errors: SC_EINVAL if n < 1, descs is NULL or any descriptor fails the sc_carve
 * checks (nothing is enqueued then); device-side errors via sc_check. */
int sc_carve_batch(const sc_image_desc *descs, int n, void *stream);

/* A batch plan: the scratch, the descriptor table and a CUDA graph of the persistent launches,
 * built once and replayed. Images that one CTA covers are carved by the one-CTA persistent
 * kernel; wider ones by the cluster-per-image persistent kernel, one launch per cluster size, each
 * chained ahead of the one-CTA launch (programmatic dependent launch) so that they have their
 * SMs first; the cluster counts minimise the estimated end of the batch.
 * autotune = 1 times every one-CTA configuration (8, 12 or 15 compute warps per CTA; DP tile
 * height 8, 16 or 32 rows) on the real batch, then load-balancing variants of the fastest (images
 * whose estimated carving time exceeds 0.8, 1.0, 1.2, 1.4, 1.7 or 2.0 x the batch's mean share
 * per SM carved by clusters of 32-row tiles, at least 2 CTAs, 384 columns per CTA), and keeps the
 * fastest; autotune = 2 takes the default configuration with that balancing at 1.4 x the mean share;
 * 0 takes the default configuration. The images' contents may
 * change between runs; their pointers and sizes may not. sc_batch_plan_run enqueues one replay on
 * `stream`; sc_batch_plan_info reports the chosen configuration (compute warps, tile height, CTAs
 * launched, images carved by one CTA / by one cluster each). */
/* The routing a batch plan applies, computed on the host with no device call (the paper has no
 * counterpart: this is the batched form's scheduler, exposed so that callers can see where their
 * images go). descs: HOST array of n descriptors (only H, W, C, target_w and target_h are read;
 * the pointers may be NULL); thr: the balancing threshold (images whose estimated one-CTA carve
 * exceeds thr x the batch's mean share per SM go to clusters of the 32-row-tile shape; 0: no
 * balancing; autotune = 2 uses 1.4); sms: the SM count the share is computed over (152 on a
 * GB300). Outputs, HOST arrays of n: cluster_size[k] 0 when one CTA carves image k, the cluster's
 * CTA count otherwise, -1 when no cluster covers it (the per-seam path carves it); shape[k] 0 for
 * clusters of 8-row tiles (images wider than one CTA), 1 for clusters of 32-row tiles; one_cta_us
 * (nullable): the carving-time model's estimate of image k's carve on one CTA, in microseconds.
 * Errors: SC_EINVAL for a NULL array, n < 1, thr < 0, sms < 1 or a descriptor that fails the
 * sc_carve size checks. */
int sc_batch_route(const sc_image_desc *descs, int n, float thr, int sms, int *cluster_size, int *shape,
                   double *one_cta_us);

typedef struct sc_batch_plan sc_batch_plan;
int sc_batch_plan_create(const sc_image_desc *descs, int n, int autotune, void *stream, sc_batch_plan **plan);
int sc_batch_plan_run(sc_batch_plan *plan, void *stream);
int sc_batch_plan_info(const sc_batch_plan *plan, int *nw, int *kt, int *grid, int *batched, int *fallback);
int sc_batch_plan_destroy(sc_batch_plan *plan);

/* ---- serving form: continuous batching with device-memory admission ----
 * A server owns one device arena of budget_bytes (the memory ledger) and `streams` CUDA streams.
 * A worker thread admits queued requests whenever the arena and a stream have room, as
 * micro-batches of up to max_batch requests of one kind, in arrival order within the kind:
 * requests that fit one CTA (searched width <= 1440) go to one persistent one-CTA-per-image
 * launch, wider ones, and those whose carve on one CTA would take over an estimated 50 ms, to one
 * persistent cluster-per-image launch per cluster size (clusters of 32-row tiles, 384 columns per
 * CTA: the heaviest requests set the tail latency). Micro-batches
 * on different streams run concurrently, so requests submitted while others are on the GPU start
 * as soon as memory and a stream free up. Every result equals sc_carve of that image alone.
 * sc_server_submit: img_host (H*W*C bytes) and out_host (target_h*target_w*C bytes) are host
 *   buffers that must stay valid until the request completes. The kernels write the carved image
 *   into out_host directly when it is page-locked (cudaHostAlloc / cudaHostRegister), otherwise
 *   into a page-locked staging block that the worker copies out; img_host should be page-locked
 *   too (its host->device copy is then asynchronous). A request completes as soon as its own
 *   image is done, whatever else its micro-batch holds. Images up to 4096 x 4096. Returns a
 *   ticket. Errors: SC_EINVAL (as sc_carve), SC_ENOMEM (larger than the whole budget).
 * sc_server_poll: 1 when done (latency_s = completion - submission, seconds), 0 while pending,
 *   a negative status if the request failed.
 * sc_server_drain: waits until nothing is queued or running (SC_ETIMEOUT after timeout_s).
 * sc_server_stats: counters and latency percentiles over the completed requests. */
typedef struct sc_server sc_server;
typedef struct {
  int64_t completed, queued, in_flight_groups, groups, batched, cluster_path;
  size_t bytes_in_use, peak_bytes, budget_bytes;
  int device_errors;
  double p50_s, p99_s, max_s;
} sc_server_stats_t;
int sc_server_create(size_t budget_bytes, int max_batch, int streams, sc_server **server);
int sc_server_submit(sc_server *server, const uint8_t *img_host, int H, int W, int C, int target_w, int target_h,
                     uint8_t *out_host, int64_t *ticket);
int sc_server_poll(sc_server *server, int64_t ticket, double *latency_s);
int sc_server_drain(sc_server *server, double timeout_s);
int sc_server_stats(sc_server *server, sc_server_stats_t *stats);
int sc_server_destroy(sc_server *server);

#ifdef __cplusplus
}
#endif
#endif /* SC_GB300_H */
