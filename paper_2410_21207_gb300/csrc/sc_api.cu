// C ABI of libsc_gb300 (declared in include/sc.h): argument checks, the per-(device, stream)
// workspace, and the host-side seam loops of the plain path.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sc.h"
#include "sc_internal.cuh"

namespace sc {

static thread_local std::string g_last_error = "no error";

static int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define SC_CUDA(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(SC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ---- optional per-kernel timing (CUDA events on the launching stream) ----
struct Timing {
  std::atomic<bool> on{false};
  std::mutex mu;
  struct Rec { cudaEvent_t a, b; };
  std::map<std::string, std::vector<Rec>> recs;
  std::map<std::string, int64_t> counts;
  int64_t total = 0;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
static Timing g_t;

template <typename F>
static cudaError_t timed(const char *name, cudaStream_t st, F &&launch) {
  if (!g_t.on.load(std::memory_order_relaxed)) return launch();
  std::lock_guard<std::mutex> lk(g_t.mu);
  Timing::Rec r{g_t.get(), g_t.get()};
  cudaEventRecord(r.a, st);
  cudaError_t e = launch();
  cudaEventRecord(r.b, st);
  g_t.recs[name].push_back(r);
  g_t.counts[name] += 1;
  g_t.total += 1;
  return e;
}

template <typename T>
struct DevBuf {
  T *p = nullptr;
  size_t cap = 0;   // elements
  cudaError_t ensure(size_t n) {
    if (n <= cap) return cudaSuccess;
    if (p) {
      cudaError_t e = cudaFree(p);   // synchronous: no earlier work can still use it
      p = nullptr;
      cap = 0;
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) { p = nullptr; return e; }
    cap = n;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

struct Workspace {
  std::mutex mu;
  DevBuf<uint32_t> img, img2, Mrow, patch;
  DevBuf<uint16_t> E;
  DevBuf<int32_t> seam;
  DevBuf<uint8_t> hin, hout;     // staging for the host-pointer entry point
  DevBuf<int> flags;             // [0] error word, [1] energy-range gate
  bool flags_zeroed = false;
  void release_all() {
    img.release(); img2.release(); Mrow.release(); patch.release();
    E.release(); seam.release(); hin.release(); hout.release(); flags.release();
    flags_zeroed = false;
  }
};

static std::mutex g_ws_mu;
static std::map<std::pair<int, void *>, Workspace *> g_ws;

static int get_ws(void *stream, Workspace **out) {
  int dev = 0;
  SC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_ws_mu);
  auto key = std::make_pair(dev, stream);
  auto it = g_ws.find(key);
  if (it == g_ws.end()) it = g_ws.emplace(key, new Workspace()).first;
  *out = it->second;
  return SC_OK;
}

static int ensure_flags(Workspace &ws, cudaStream_t st) {
  SC_CUDA(ws.flags.ensure(4));
  if (!ws.flags_zeroed) {
    SC_CUDA(cudaMemsetAsync(ws.flags.p, 0, 4 * sizeof(int), st));
    ws.flags_zeroed = true;
  }
  return SC_OK;
}

static bool valid_c(int C) { return C == 1 || C == 3 || C == 4; }

// Buffers for carving an H x W image (both passes).
static int ensure_carve_buffers(Workspace &ws, int H, int W) {
  const int R = H > W ? H : W;            // rows in either orientation
  const int P = round_up(R, 4);           // word pitch covering either orientation
  SC_CUDA(ws.img.ensure((size_t)R * P));
  SC_CUDA(ws.img2.ensure((size_t)R * P));
  const int pe = pitch_e_for(R);
  SC_CUDA(ws.E.ensure((size_t)R * pe));
  const int S = (R + KS - 1) / KS;
  SC_CUDA(ws.Mrow.ensure((size_t)(S + 1) * pe));
  SC_CUDA(ws.seam.ensure((size_t)R));
  SC_CUDA(ws.patch.ensure((size_t)R));
  return SC_OK;
}

static int launch_search(Workspace &ws, uint16_t *Ebase, int pe, int H, int W, int32_t *seam, int32_t *seam_log,
                         int64_t *cost, const int *gate, cudaStream_t st) {
  DpArgs a;
  a.E = Ebase + E_PADL;
  a.pitch_e = pe;
  a.H = H;
  a.W = W;
  a.Mrow = ws.Mrow.p + E_PADL;
  a.seam = seam;
  a.seam_log = seam_log;
  a.cost = cost;
  a.err = ws.flags.p;
  a.gate = gate;
  SC_CUDA(timed("dp", st, [&] { return launch_dp(a, st); }));
  return SC_OK;
}

// (count) vertical seams of an H x W word image in place; E holds its energy (pitch pe).
static int carve_pass_plain(Workspace &ws, uint32_t *img, int pitch, int H, int W, int count, int pe,
                            int32_t *seam_log, int64_t *cost_log, cudaStream_t st) {
  uint16_t *E = ws.E.p;
  for (int t = 0; t < count; ++t) {
    const int w = W - t;
    int rc = launch_search(ws, E, pe, H, w, ws.seam.p, seam_log ? seam_log + (size_t)t * H : nullptr,
                           cost_log ? cost_log + t : nullptr, nullptr, st);
    if (rc) return rc;
    SC_CUDA(timed("patch", st, [&] { return launch_patch(img, pitch, H, w, ws.seam.p, ws.patch.p, ws.flags.p, st); }));
    SC_CUDA(timed("shift", st, [&] { return launch_shift(img, pitch, E + E_PADL, pe, H, w, ws.seam.p, ws.patch.p, st); }));
  }
  return SC_OK;
}

static int check_carve_args(const void *img, int H, int W, int C, int tw, int th, const void *out) {
  if (!img || !out) return fail(SC_EINVAL, "null image or output pointer");
  if (H < 1 || W < 1) return fail(SC_EINVAL, "H and W must be >= 1 (got %d x %d)", H, W);
  if (!valid_c(C)) return fail(SC_EINVAL, "C must be 1, 3 or 4 (got %d)", C);
  if (tw < 1 || th < 1) return fail(SC_EINVAL, "targets must be >= 1 (got %d x %d)", tw, th);
  if (tw > W || th > H) return fail(SC_EINVAL, "enlargement is not supported (target %d x %d > %d x %d)", tw, th, W, H);
  if (H > SC_MAX_ROWS || W > SC_MAX_COLS)
    return fail(SC_EINVAL, "image %d x %d exceeds the %d x %d limit", W, H, SC_MAX_COLS, SC_MAX_ROWS);
  if ((int64_t)H * W * C >= ((int64_t)1 << 31)) return fail(SC_EINVAL, "H*W*C must be < 2^31");
  return SC_OK;
}

static int carve_impl(const uint8_t *img, int H, int W, int C, int tw, int th, uint8_t *out, int32_t *seam_log,
                      int64_t *cost_log, cudaStream_t st) {
  Workspace *wsp;
  int rc = get_ws((void *)st, &wsp);
  if (rc) return rc;
  Workspace &ws = *wsp;
  std::lock_guard<std::mutex> lk(ws.mu);
  if ((rc = ensure_flags(ws, st))) return rc;
  if ((rc = ensure_carve_buffers(ws, H, W))) return rc;
  const int R = H > W ? H : W;
  const int pitch = round_up(R, 4);
  const int pe = pitch_e_for(R);
  SC_CUDA(timed("pack", st, [&] { return launch_pack(img, H, W, C, ws.img.p, pitch, st); }));
  SC_CUDA(timed("energy", st, [&] { return launch_energy(ws.img.p, pitch, H, W, ws.E.p + E_PADL, pe, st); }));
  const int nv = W - tw, nh = H - th;
  rc = carve_pass_plain(ws, ws.img.p, pitch, H, W, nv, pe, seam_log, cost_log, st);
  if (rc) return rc;
  if (nh > 0) {
    SC_CUDA(timed("transpose", st, [&] { return launch_transpose(ws.img.p, pitch, H, tw, ws.img2.p, pitch, st); }));  // tw x H
    SC_CUDA(timed("energy", st, [&] { return launch_energy(ws.img2.p, pitch, tw, H, ws.E.p + E_PADL, pe, st); }));
    rc = carve_pass_plain(ws, ws.img2.p, pitch, tw, H, nh, pe, seam_log ? seam_log + (size_t)nv * H : nullptr,
                          cost_log ? cost_log + nv : nullptr, st);
    if (rc) return rc;
    SC_CUDA(timed("transpose", st, [&] { return launch_transpose(ws.img2.p, pitch, tw, th, ws.img.p, pitch, st); }));  // th x tw
  }
  SC_CUDA(timed("unpack", st, [&] { return launch_unpack(ws.img.p, pitch, th, tw, C, false, out, st); }));
  return SC_OK;
}

}  // namespace sc

using namespace sc;

extern "C" {

int sc_version(void) { return 100; }

const char *sc_last_error(void) { return g_last_error.c_str(); }

int sc_check(void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *wsp;
  int rc = get_ws(stream, &wsp);
  if (rc) return rc;
  Workspace &ws = *wsp;
  std::lock_guard<std::mutex> lk(ws.mu);
  SC_CUDA(cudaStreamSynchronize(st));
  if (!ws.flags.p) return SC_OK;
  int h[2] = {0, 0};
  SC_CUDA(cudaMemcpy(h, ws.flags.p, 2 * sizeof(int), cudaMemcpyDeviceToHost));
  SC_CUDA(cudaMemset(ws.flags.p, 0, 2 * sizeof(int)));
  const int e = h[0];
  if (e & ERR_TIMEOUT) return fail(SC_ETIMEOUT, "a bounded device wait ran out (error word 0x%x)", e);
  if (e & ERR_ENERGY_RANGE) return fail(SC_EINVAL, "energies too large: a seam sum could reach 2^24");
  if (e) return fail(SC_EINTERNAL, "device consistency check failed (error word 0x%x)", e);
  return SC_OK;
}

int sc_timing_enable(int on) {
  g_t.on.store(on != 0);
  return SC_OK;
}

int sc_timing_reset(void) {
  std::lock_guard<std::mutex> lk(g_t.mu);
  for (auto &kv : g_t.recs)
    for (auto &r : kv.second) { g_t.pool.push_back(r.a); g_t.pool.push_back(r.b); }
  g_t.recs.clear();
  g_t.counts.clear();
  g_t.total = 0;
  return SC_OK;
}

int sc_timing_read(const char *kernel, double *total_ms, int64_t *launches) {
  if (!kernel || !total_ms || !launches) return fail(SC_EINVAL, "null pointer");
  std::lock_guard<std::mutex> lk(g_t.mu);
  *total_ms = 0.0;
  *launches = 0;
  if (strcmp(kernel, "all") == 0) {
    *launches = g_t.total;
    return SC_OK;
  }
  auto it = g_t.recs.find(kernel);
  if (it == g_t.recs.end()) return SC_OK;
  double sum = 0.0;
  for (auto &r : it->second) {
    SC_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    SC_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    sum += ms;
  }
  *total_ms = sum;
  *launches = (int64_t)it->second.size();
  return SC_OK;
}

int sc_release_workspaces(void) {
  int dev = 0;
  SC_CUDA(cudaGetDevice(&dev));
  SC_CUDA(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(g_ws_mu);
  for (auto it = g_ws.begin(); it != g_ws.end();) {
    if (it->first.first == dev) {
      it->second->release_all();
      delete it->second;
      it = g_ws.erase(it);
    } else {
      ++it;
    }
  }
  return SC_OK;
}

int sc_energy(const uint8_t *img, int H, int W, int C, uint16_t *energy_out, void *stream) {
  if (!img || !energy_out) return fail(SC_EINVAL, "null pointer");
  if (H < 1 || W < 1 || !valid_c(C)) return fail(SC_EINVAL, "bad shape %d x %d x %d", H, W, C);
  if ((int64_t)H * W * C >= ((int64_t)1 << 31)) return fail(SC_EINVAL, "H*W*C must be < 2^31");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *wsp;
  int rc = get_ws(stream, &wsp);
  if (rc) return rc;
  Workspace &ws = *wsp;
  std::lock_guard<std::mutex> lk(ws.mu);
  const int pitch = round_up(W, 4);
  SC_CUDA(ws.img.ensure((size_t)H * pitch));
  SC_CUDA(launch_pack(img, H, W, C, ws.img.p, pitch, st));
  SC_CUDA(launch_energy(ws.img.p, pitch, H, W, energy_out, W, st));
  return SC_OK;
}

int sc_find_seam(const uint16_t *energy, int H, int W, int32_t *seam_out, int64_t *cost_out, void *stream) {
  if (!energy || !seam_out) return fail(SC_EINVAL, "null pointer");
  if (H < 1 || W < 1 || H > SC_MAX_ROWS || W > SC_MAX_COLS) return fail(SC_EINVAL, "bad shape %d x %d", H, W);
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *wsp;
  int rc = get_ws(stream, &wsp);
  if (rc) return rc;
  Workspace &ws = *wsp;
  std::lock_guard<std::mutex> lk(ws.mu);
  if ((rc = ensure_flags(ws, st))) return rc;
  const int pe = pitch_e_for(W);
  SC_CUDA(ws.E.ensure((size_t)H * pe));
  SC_CUDA(ws.Mrow.ensure((size_t)((H + KS - 1) / KS + 1) * pe));
  SC_CUDA(cudaMemsetAsync(ws.flags.p + 1, 0, sizeof(int), st));
  SC_CUDA(launch_copy_energy(energy, H, W, ws.E.p + E_PADL, pe, ws.flags.p, ws.flags.p + 1, st));
  return launch_search(ws, ws.E.p, pe, H, W, seam_out, nullptr, cost_out, ws.flags.p + 1, st);
}

int sc_carve_plain(const uint8_t *img, int H, int W, int C, int target_w, int target_h, uint8_t *out,
                   int32_t *seam_log, int64_t *cost_log, void *stream) {
  int rc = check_carve_args(img, H, W, C, target_w, target_h, out);
  if (rc) return rc;
  return carve_impl(img, H, W, C, target_w, target_h, out, seam_log, cost_log, (cudaStream_t)stream);
}

int sc_carve(const uint8_t *img, int H, int W, int C, int target_w, int target_h, uint8_t *out, int32_t *seam_log,
             int64_t *cost_log, void *stream) {
  int rc = check_carve_args(img, H, W, C, target_w, target_h, out);
  if (rc) return rc;
  return carve_impl(img, H, W, C, target_w, target_h, out, seam_log, cost_log, (cudaStream_t)stream);
}

int sc_carve_host(const uint8_t *img_host, int H, int W, int C, int target_w, int target_h, uint8_t *out_host,
                  void *stream) {
  int rc = check_carve_args(img_host, H, W, C, target_w, target_h, out_host);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *wsp;
  rc = get_ws(stream, &wsp);
  if (rc) return rc;
  const size_t nin = (size_t)H * W * C, nout = (size_t)target_h * target_w * C;
  {
    std::lock_guard<std::mutex> lk(wsp->mu);
    SC_CUDA(wsp->hin.ensure(nin));
    SC_CUDA(wsp->hout.ensure(nout));
  }
  uint8_t *din = wsp->hin.p, *dout = wsp->hout.p;
  SC_CUDA(cudaMemcpyAsync(din, img_host, nin, cudaMemcpyHostToDevice, st));
  rc = carve_impl(din, H, W, C, target_w, target_h, dout, nullptr, nullptr, st);
  if (rc) return rc;
  SC_CUDA(cudaMemcpyAsync(out_host, dout, nout, cudaMemcpyDeviceToHost, st));
  return sc_check(stream);
}

int sc_carve_batch(const sc_image_desc *descs, int n, void *stream) {
  if (!descs || n < 1) return fail(SC_EINVAL, "empty batch");
  for (int k = 0; k < n; ++k) {
    const sc_image_desc &d = descs[k];
    int rc = check_carve_args(d.img, d.H, d.W, d.C, d.target_w, d.target_h, d.out);
    if (rc) return fail(rc, "descriptor %d: %s", k, g_last_error.c_str());
  }
  for (int k = 0; k < n; ++k) {
    const sc_image_desc &d = descs[k];
    int rc = carve_impl(d.img, d.H, d.W, d.C, d.target_w, d.target_h, d.out, d.seam_log, nullptr,
                        (cudaStream_t)stream);
    if (rc) return rc;
  }
  return SC_OK;
}

}  // extern "C"
