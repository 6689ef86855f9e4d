// Serving form: a request loop with continuous batching and device-memory admission.
//
// Callers submit carve requests (host buffers) at any time. A worker thread repeatedly
//   1. retires launch groups whose completion event has fired (frees their memory, time-stamps
//      their requests),
//   2. admits queued requests while the device-memory ledger (one arena of the configured budget,
//      first-fit) has room, as micro-batches of up to max_batch requests of one kind, in arrival
//      order within the kind: requests that fit one CTA go to the one-CTA persistent kernel
//      (k_batch), wider ones and those whose one-CTA carve would take over an estimated 50 ms to
//      the cluster-per-image persistent kernel in its latency shape (k_batch_cl), one micro-batch
//      per cluster size,
//   3. enqueues each micro-batch on a free stream: host->device copies of the inputs, the launch,
//      a completion event.
// The kernels write every carved image straight into host memory (the caller's page-locked output
// buffer, or a page-locked staging block for pageable ones) and then set that image's completion
// word in page-locked memory, so a request completes as soon as its own image is done, not when
// its whole micro-batch is; its device memory is returned to the ledger at that moment.
// Micro-batches on different streams run concurrently on the GPU, so requests that arrive while
// others are being carved start as soon as memory and a stream are free, and their work overlaps.
// Results do not depend on the grouping: every image is carved by the same integer arithmetic.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sc_batch_cl.h"
#include "sc_host.h"
#include "sc_internal.cuh"

namespace sc {

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// first-fit sub-allocator over one device region, or one page-locked host region mapped into the
// device's address space (256-byte granules)
struct Arena {
  unsigned char *base = nullptr;
  bool host = false;
  size_t size = 0, in_use = 0, peak = 0;
  std::map<size_t, size_t> free_;   // offset -> bytes
  bool init(size_t bytes) {
    size = a256(bytes);
    if (cudaMalloc(&base, size) != cudaSuccess) return false;
    free_[0] = size;
    return true;
  }
  bool init_host(size_t bytes) {
    size = a256(bytes);
    if (cudaHostAlloc((void **)&base, size, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      base = nullptr;
      return false;
    }
    host = true;
    free_[0] = size;
    return true;
  }
  void destroy() {
    if (base) host ? cudaFreeHost(base) : cudaFree(base);
    base = nullptr;
  }
  bool alloc(size_t n, size_t *off) {
    n = a256(n ? n : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n;
        const size_t o = it->first + n;
        free_.erase(it);
        if (rest) free_[o] = rest;
        in_use += n;
        peak = std::max(peak, in_use);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = a256(n ? n : 1);
    in_use -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct Request {
  const uint8_t *in = nullptr;
  uint8_t *out = nullptr;
  int H = 0, W = 0, C = 0, tw = 0, th = 0;
  double t_submit = 0, t_done = -1;
  int status = 0;                                   // 0 queued, 1 on the GPU, 2 done, < 0 error
  uint8_t *dout = nullptr;                          // where the kernel writes the result (host memory)
  bool staged = false;                              // out is pageable: the result goes through staging
  size_t hoff = 0, hbytes = 0;                      // staging block
  int flag = -1;                                    // index of the completion word
  int kind = 0;                                     // kind_of at submission (sizes and config fixed)
  std::vector<std::pair<size_t, size_t>> dallocs;   // device arena blocks (offset, bytes)
};

struct Group {
  int cs = 0;                                      // 0: one-CTA micro-batch; else the cluster size
  std::vector<int64_t> tickets;
  std::vector<std::pair<size_t, size_t>> allocs;   // device arena blocks of the launch itself
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int err_slot = -1;                               // completion word receiving the device error word
  int launch_failed = 0;
};

}  // namespace

}  // namespace sc

struct sc_server {
  size_t budget = 0;
  int max_batch = 64;
  int dev = 0;
  // wide requests, and those whose one-CTA carve would take over 50 ms, on latency-shaped clusters
  sc::BatchCfg cfg{15, 16, 0.f, true, 50000.f};
  int sms = 1, occ = 1;
  sc::Arena arena;
  sc::Arena staging;                   // page-locked results of pageable output buffers (lazy)
  int *flags = nullptr;                // page-locked completion words, one per request on the GPU
  std::vector<int> free_flags;
  std::vector<cudaEvent_t> free_events;
  std::vector<cudaEvent_t> all_events;
  std::vector<cudaStream_t> streams;   // free pool
  std::map<std::pair<int, int>, int> cl_capacity;   // (cluster size, super-tiles) -> clusters
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, sc::Request> reqs;
  std::vector<sc::Group> inflight;
  std::vector<double> latencies;
  int64_t next_ticket = 1;
  int64_t done_count = 0, batched_count = 0, big_count = 0, groups = 0;
  bool stop = false;
  int device_errors = 0;
  std::thread worker;
};

namespace sc {
namespace {

sc_image_desc desc_of(const Request &r) {
  sc_image_desc d{};
  d.H = r.H; d.W = r.W; d.C = r.C; d.target_w = r.tw; d.target_h = r.th;
  return d;
}

// 0 for a request one CTA carves, else the cluster that carves it: shape * 64 + cluster size (the
// layout of a one-request batch decides both)
int kind_of(const sc_server *s, const Request &r) {
  const sc_image_desc d = desc_of(r);
  BatchSetup b;
  batch_layout(&d, 1, s->cfg, nullptr, b);
  if (!b.items.empty()) return 0;
  if (b.cl.empty()) return batch_cluster_size(d);   // wider than any cluster: refused at submission
  return b.cl[0].shape * 64 + b.cl[0].cs;
}
int kind_cs(int kind) { return kind & 63; }
int kind_shape(int kind) { return kind >> 6; }

// scratch bytes and super-tiles of one request's carve
size_t item_bytes(const sc_server *s, const sc_image_desc &d, int *S) {
  BatchSetup b;
  batch_layout(&d, 1, s->cfg, nullptr, b);
  *S = b.items.empty() ? (b.cl.empty() ? 1 : b.cl[0].Smax) : b.Smax;
  return b.pool_bytes;
}

void release_request(sc_server *s, Request &r) {
  for (auto &a : r.dallocs) s->arena.release(a.first, a.second);
  r.dallocs.clear();
  if (r.staged && r.hbytes) s->staging.release(r.hoff, r.hbytes);
  r.hbytes = 0;
  if (r.flag >= 0) s->free_flags.push_back(r.flag);
  r.flag = -1;
}

void finish_request(sc_server *s, Request &r, bool ok, double t) {
  if (ok && r.staged) std::memcpy(r.out, r.dout, (size_t)r.th * r.tw * r.C);
  release_request(s, r);
  r.t_done = t;
  r.status = ok ? 2 : SC_EINTERNAL;
  s->latencies.push_back(t - r.t_submit);
  s->done_count++;
  if (!ok) s->device_errors++;
}

// Retire every request whose image is complete, and every launch whose stream has finished
// (caller holds the lock).
void retire(sc_server *s) {
  const double t = now_s();
  for (size_t g = 0; g < s->inflight.size();) {
    Group &G = s->inflight[g];
    for (int64_t tk : G.tickets) {
      Request &r = s->reqs[tk];
      if (r.status != 1) continue;
      const int v = *(volatile int *)&s->flags[r.flag];
      if (v == 0) continue;
      std::atomic_thread_fence(std::memory_order_acquire);   // the result bytes after the word
      finish_request(s, r, v == 1, t);
    }
    const cudaError_t q = cudaEventQuery(G.done);
    if (q == cudaErrorNotReady) { ++g; continue; }
    const bool ok = (q == cudaSuccess) && !G.launch_failed && (*(volatile int *)&s->flags[G.err_slot] == 0);
    for (int64_t tk : G.tickets) {
      Request &r = s->reqs[tk];
      if (r.status != 1) continue;
      const int v = *(volatile int *)&s->flags[r.flag];
      std::atomic_thread_fence(std::memory_order_acquire);
      finish_request(s, r, ok && v == 1, t);   // a launch that ended without completing it failed
    }
    for (auto &a : G.allocs) s->arena.release(a.first, a.second);
    s->free_events.push_back(G.done);   // page-locked allocations and frees would synchronise the
    s->free_flags.push_back(G.err_slot);  // device: events and words come from pools

    s->streams.push_back(G.stream);
    s->inflight.erase(s->inflight.begin() + g);
  }
  s->cv.notify_all();
}

// Start one micro-batch if possible (caller holds the lock). Returns true if something was launched.
bool admit(sc_server *s) {
  if (s->queue.empty() || s->streams.empty() || s->free_events.empty() || s->free_flags.size() < 2) return false;
  const int kind = s->reqs[s->queue.front()].kind;
  std::vector<int64_t> take;
  std::vector<sc_image_desc> descs;
  std::vector<std::pair<size_t, size_t>> allocs;
  int Smax = 1;
  for (int64_t tk : s->queue) {
    if ((int)take.size() >= s->max_batch) break;
    Request &r = s->reqs[tk];
    if (r.kind != kind) continue;   // another kind's micro-batch takes it
    sc_image_desc d = desc_of(r);
    int S = 1;
    const size_t scratch = item_bytes(s, d, &S);
    const int sm = std::max(Smax, S);
    const size_t smem = kind ? batch_cl_smem_bytes(sm, kind_shape(kind)) : batch_smem_bytes(s->cfg.nw, s->cfg.kt, sm);
    if (smem > 232448 - 1024) break;
    const size_t nin = (size_t)r.H * r.W * r.C, nout = (size_t)r.th * r.tw * r.C;
    if (s->free_flags.size() < 2) break;   // one word stays for the launch's error word
    if (r.staged && !s->staging.base && !s->staging.init_host(std::min(s->budget, (size_t)2 << 30))) break;
    size_t oin, osc, ohost = 0;
    if (!s->arena.alloc(nin, &oin)) break;
    if (!s->arena.alloc(scratch, &osc)) { s->arena.release(oin, nin); break; }
    if (r.staged && !s->staging.alloc(nout, &ohost)) { s->arena.release(oin, nin); s->arena.release(osc, scratch); break; }
    r.dallocs = {{oin, nin}, {osc, scratch}};
    allocs.push_back({oin, nin});
    allocs.push_back({osc, scratch});
    if (r.staged) {
      r.hoff = ohost;
      r.hbytes = nout;
      r.dout = s->staging.base + ohost;
    }
    r.flag = s->free_flags.back();
    s->free_flags.pop_back();
    s->flags[r.flag] = 0;
    d.img = s->arena.base + oin;
    d.out = r.dout;
    d.seam_log = nullptr;
    descs.push_back(d);
    take.push_back(tk);
    Smax = sm;
  }
  auto undo = [&]() {
    for (int64_t tk : take) release_request(s, s->reqs[tk]);
  };
  if (take.empty()) return false;
  const int n = (int)take.size();
  size_t otab, oq;
  const size_t tab_bytes = (size_t)n * sizeof(BatchItem);
  if (!s->arena.alloc(tab_bytes, &otab)) {
    undo();
    return false;
  }
  if (!s->arena.alloc(256, &oq)) {
    s->arena.release(otab, tab_bytes);
    undo();
    return false;
  }
  // per-image scratch layouts, each placed in its own arena block
  std::vector<BatchItem> items(n);
  for (int k = 0; k < n; ++k) {
    BatchSetup b;
    batch_layout(&descs[k], 1, s->cfg, s->arena.base + allocs[2 * k + 1].first, b);
    items[k] = kind ? b.cl[0].items[0] : b.items[0];
    items[k].done = s->flags + s->reqs[take[k]].flag;   // page-locked, mapped: the same address on the device
  }
  allocs.clear();
  allocs.push_back({otab, tab_bytes});
  allocs.push_back({oq, 256});
  // longest carves first in the launch's queue
  std::stable_sort(items.begin(), items.end(), [](const BatchItem &a, const BatchItem &c) {
    return (double)(a.W - a.tw) * a.H * a.W + (double)(a.H - a.th) * a.tw * a.H >
           (double)(c.W - c.tw) * c.H * c.W + (double)(c.H - c.th) * c.tw * c.H;
  });
  Group G;
  G.cs = kind;
  G.stream = s->streams.back();
  s->streams.pop_back();
  G.tickets = take;
  G.allocs = allocs;
  G.err_slot = s->free_flags.back();
  s->free_flags.pop_back();
  s->flags[G.err_slot] = 0;
  int *q = reinterpret_cast<int *>(s->arena.base + oq);
  int *derr = q + 1;
  BatchItem *dtab = reinterpret_cast<BatchItem *>(s->arena.base + otab);
  cudaMemcpyAsync(dtab, items.data(), tab_bytes, cudaMemcpyHostToDevice, G.stream);   // pageable: staged
  cudaMemsetAsync(q, 0, 2 * sizeof(int), G.stream);
  for (int k = 0; k < n; ++k) {
    Request &r = s->reqs[take[k]];
    cudaMemcpyAsync((void *)descs[k].img, r.in, (size_t)r.H * r.W * r.C, cudaMemcpyHostToDevice, G.stream);
    r.status = 1;
  }
  cudaError_t le;
  if (kind) {
    auto key = std::make_pair(kind, Smax);
    auto it = s->cl_capacity.find(key);
    if (it == s->cl_capacity.end()) {
      int cap = 0;
      if (batch_cl_capacity(kind_cs(kind), Smax, &cap, kind_shape(kind)) != cudaSuccess || cap < 1) cap = 1;
      it = s->cl_capacity.emplace(key, cap).first;
    }
    le = launch_batch_cl(dtab, n, kind_cs(kind), Smax, std::min(n, it->second), q, derr, G.stream, kind_shape(kind));
  } else {
    int grid = s->sms * s->occ;
    if (grid > n) grid = n;
    le = launch_batch(s->cfg.nw, s->cfg.kt, dtab, n, Smax, grid, q, derr, G.stream);
  }
  if (le != cudaSuccess) G.launch_failed = 1;
  cudaMemcpyAsync(&s->flags[G.err_slot], derr, sizeof(int), cudaMemcpyDeviceToHost, G.stream);
  G.done = s->free_events.back();
  s->free_events.pop_back();
  cudaEventRecord(G.done, G.stream);
  for (int64_t tk : take) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), tk));
  s->inflight.push_back(G);
  if (kind)
    s->big_count += n;
  else
    s->batched_count += n;
  s->groups++;
  return true;
}

void worker_loop(sc_server *s) {
  cudaSetDevice(s->dev);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    retire(s);
    bool launched = false;
    while (admit(s)) launched = true;
    if (s->stop && s->queue.empty() && s->inflight.empty()) break;
    if (!launched) {
      // nothing to start: wait briefly for a submission or a completion
      s->cv.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 500 : 20));
    }
  }
}

}  // namespace
}  // namespace sc

using namespace sc;

extern "C" {

int sc_server_create(size_t budget_bytes, int max_batch, int streams, sc_server **out) {
  if (!out) return fail(SC_EINVAL, "null server pointer");
  *out = nullptr;
  if (budget_bytes < ((size_t)64 << 20)) return fail(SC_EINVAL, "budget must be at least 64 MiB");
  if (max_batch < 1 || streams < 2) return fail(SC_EINVAL, "max_batch >= 1 and streams >= 2 required");
  sc_server *s = new sc_server();
  s->budget = budget_bytes;
  s->max_batch = max_batch;
  if (cudaGetDevice(&s->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->dev) != cudaSuccess) {
    delete s;
    return fail(SC_ECUDA, "no CUDA device");
  }
  if (!s->arena.init(budget_bytes)) {
    delete s;
    return fail(SC_ENOMEM, "cannot allocate the %zu-byte device arena", budget_bytes);
  }
  constexpr int kFlags = 1 << 16;   // requests on the GPU at once
  if (cudaHostAlloc((void **)&s->flags, kFlags * sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable) !=
      cudaSuccess) {
    s->flags = nullptr;
    s->arena.destroy();
    delete s;
    return fail(SC_ENOMEM, "cannot allocate the completion words");
  }
  for (int k = kFlags - 1; k >= 0; --k) s->free_flags.push_back(k);
  s->occ = batch_blocks_per_sm(s->cfg.nw, s->cfg.kt, 1);
  for (int k = 0; k < streams; ++k) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return fail(SC_ECUDA, "stream creation failed");
    }
    s->streams.push_back(st);
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      delete s;
      return fail(SC_ECUDA, "event creation failed");
    }
    s->free_events.push_back(ev);
    s->all_events.push_back(ev);
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return SC_OK;
}

int sc_server_submit(sc_server *s, const uint8_t *img_host, int H, int W, int C, int target_w, int target_h,
                     uint8_t *out_host, int64_t *ticket) {
  if (!s || !ticket) return fail(SC_EINVAL, "null server or ticket pointer");
  int rc = check_carve_args(img_host, H, W, C, target_w, target_h, out_host);
  if (rc) return rc;
  if (H > 4096 || W > 4096) return fail(SC_EINVAL, "served images are limited to 4096 x 4096");
  Request r;
  r.in = img_host;
  r.out = out_host;
  r.H = H; r.W = W; r.C = C; r.tw = target_w; r.th = target_h;
  // a page-locked output buffer is written by the kernels directly; a pageable one through staging
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, out_host) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer) {
    r.dout = static_cast<uint8_t *>(pa.devicePointer);
  } else {
    cudaGetLastError();
    r.staged = true;
  }
  r.t_submit = now_s();
  int S = 1;
  const size_t need = (size_t)H * W * C + (size_t)target_h * target_w * C + item_bytes(s, desc_of(r), &S) + 4096;
  if (need > s->arena.size) return fail(SC_ENOMEM, "a %d x %d request needs more than the whole budget", W, H);
  r.kind = kind_of(s, r);
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t t = s->next_ticket++;
  s->reqs[t] = r;
  s->queue.push_back(t);
  *ticket = t;
  s->cv.notify_all();
  return SC_OK;
}

int sc_server_poll(sc_server *s, int64_t ticket, double *latency_s) {
  if (!s) return fail(SC_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(SC_EINVAL, "unknown ticket");
  if (it->second.status == 2) {
    if (latency_s) *latency_s = it->second.t_done - it->second.t_submit;
    return 1;
  }
  if (it->second.status < 0) return it->second.status;
  return 0;
}

int sc_server_drain(sc_server *s, double timeout_s) {
  if (!s) return fail(SC_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  const double t_end = now_s() + timeout_s;
  while (!(s->queue.empty() && s->inflight.empty())) {
    if (now_s() > t_end) return fail(SC_ETIMEOUT, "requests still pending after %.1f s", timeout_s);
    s->cv.wait_for(lk, std::chrono::milliseconds(1));
  }
  return s->device_errors ? fail(SC_EINTERNAL, "%d launch groups reported device errors", s->device_errors) : SC_OK;
}

int sc_server_stats(sc_server *s, sc_server_stats_t *out) {
  if (!s || !out) return fail(SC_EINVAL, "null pointer");
  std::lock_guard<std::mutex> lk(s->mu);
  out->completed = s->done_count;
  out->queued = (int64_t)s->queue.size();
  out->in_flight_groups = (int64_t)s->inflight.size();
  out->groups = s->groups;
  out->batched = s->batched_count;
  out->cluster_path = s->big_count;
  out->bytes_in_use = s->arena.in_use;
  out->peak_bytes = s->arena.peak;
  out->budget_bytes = s->arena.size;
  out->device_errors = s->device_errors;
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) { return l.empty() ? 0.0 : l[(size_t)std::min<double>(l.size() - 1, p * (l.size() - 1) + 0.5)]; };
  out->p50_s = pct(0.50);
  out->p99_s = pct(0.99);
  out->max_s = l.empty() ? 0.0 : l.back();
  return SC_OK;
}

int sc_server_destroy(sc_server *s) {
  if (!s) return SC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : s->all_events) cudaEventDestroy(ev);
  s->arena.destroy();
  s->staging.destroy();
  if (s->flags) cudaFreeHost(s->flags);
  delete s;
  return SC_OK;
}

}  // extern "C"
