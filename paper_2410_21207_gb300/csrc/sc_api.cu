// C ABI of libsc_gb300 (declared in include/sc.h): argument checks, the per-(device, stream)
// workspace, and the host-side seam loops of the plain path.
#include <algorithm>
#include <queue>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sc.h"
#include "sc_batch_item.h"
#include "sc_batch_cl.h"
#include "sc_host.h"
#include "sc_internal.cuh"
#include "sc_rowops.cuh"

namespace sc {

static thread_local std::string g_last_error = "no error";

int fail(int code, const char *fmt, ...) {
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
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
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
  DevBuf<uint32_t> img, img2, Mrow;
  DevBuf<uint16_t> E;
  DevBuf<int32_t> seam;
  DevBuf<int16_t> lists;          // two generations of pending-removal lists
  DevBuf<uint8_t> hin, hout;     // staging for the host-pointer entry point
  DevBuf<int> flags;             // [0] error word, [1] energy-range gate
  DevBuf<int> gates;             // one energy-range gate per map of sc_find_seam_multi
  DevBuf<uint32_t> wdirs;        // wide-cost search: directions and ancestors (per map)
  DevBuf<uint16_t> wanc;
  DevBuf<uint16_t> Emulti;       // padded maps of sc_find_seam_multi
  DevBuf<int32_t> enl_log;       // sc_enlarge: the k seams, the carved copy, the widening bitmap
  DevBuf<uint8_t> enl_tmp;
  DevBuf<uint32_t> enl_bits;
  DevBuf<uint32_t> Mmulti;
  DevBuf<DpArgs> dargs;
  bool flags_zeroed = false;
  void release_all() {
    img.release(); img2.release(); Mrow.release();
    E.release(); seam.release(); lists.release(); hin.release(); hout.release(); flags.release();
    Emulti.release(); Mmulti.release(); dargs.release(); gates.release(); wdirs.release(); wanc.release();
    enl_log.release(); enl_tmp.release(); enl_bits.release();
    flags_zeroed = false;
  }
};

static std::mutex g_ws_mu;
static std::map<std::pair<int, void *>, Workspace *> g_ws;

// One error word per device for batched launches (plans may run on any stream); sc_check reads it.
static std::mutex g_gerr_mu;
static std::map<int, int *> g_gerr;
int *device_error_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_gerr_mu);
  auto it = g_gerr.find(dev);
  if (it != g_gerr.end()) return it->second;
  int *p = nullptr;
  if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
  if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
  g_gerr[dev] = p;
  return p;
}

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
  SC_CUDA(ws.lists.ensure((size_t)2 * R * RPEND));
  return SC_OK;
}

// Grow a stream's workspace for images up to H x W in both orientations (no allocation later).
int workspace_reserve(cudaStream_t st, int H, int W) {
  Workspace *wsp;
  int rc = get_ws((void *)st, &wsp);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(wsp->mu);
  if ((rc = ensure_flags(*wsp, st))) return rc;
  return ensure_carve_buffers(*wsp, H, W);
}

static int launch_search(Workspace &ws, uint16_t *Ebase, int pe, int H, int W, int32_t *seam, int32_t *seam_log,
                         int64_t *cost, int *gate, cudaStream_t st, int64_t pstride = 0) {
  DpArgs a;
  a.pstride = pstride;
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
  // a map whose seam sums may not fit the 24-bit search was skipped by it (gate set): the wide-cost
  // search takes it; for every other map this launch returns at once
  SC_CUDA(timed("dp_wide", st, [&] { return launch_dp_wide(a, ws.wdirs.p, ws.wanc.p, st); }));
  return SC_OK;
}

static int ensure_wide(Workspace &ws, int H, int W, int n) {
  SC_CUDA(ws.wdirs.ensure(wide_dirs_words(H, W) * n));
  SC_CUDA(ws.wanc.ensure(wide_anc_elems(H, W) * n));
  return SC_OK;
}

// (count) vertical seams of an H x W word image; ws.E holds its energy (pitch pe). Per seam: the
// search, then one warp per row computes the refreshed energy pair through the pending-removal
// lists, adds the removal to the row's list and compacts the energy row. The image words are
// compacted every RPEND seams and at the end of the pass.
static int carve_pass_plain(Workspace &ws, uint32_t *img, int pitch, int H, int W, int count, int pe,
                            int32_t *seam_log, int64_t *cost_log, cudaStream_t st, int64_t pstride = 0) {
  int16_t *lb[2] = {ws.lists.p, ws.lists.p + (size_t)H * RPEND};
  int cur = 0, m = 0;
  for (int t = 0; t < count; ++t) {
    const int w = W - t;
    DpArgs a;
    a.E = ws.E.p + E_PADL;
    a.pitch_e = pe;
    a.H = H;
    a.W = w;
    a.Mrow = ws.Mrow.p + E_PADL;
    a.seam = ws.seam.p;
    a.seam_log = seam_log ? seam_log + (size_t)t * H : nullptr;
    a.cost = cost_log ? cost_log + t : nullptr;
    a.err = ws.flags.p;
    a.gate = nullptr;
    a.pstride = pstride;
    SC_CUDA(timed("dp", st, [&] { return launch_dp(a, st); }));
    SC_CUDA(timed("refresh", st, [&] {
      return pstride ? launch_refresh_fwd(img, pitch, ws.E.p + E_PADL, pe, pstride, H, w, ws.seam.p, lb[cur],
                                          lb[cur ^ 1], m, ws.flags.p, st)
                     : launch_refresh(img, pitch, ws.E.p + E_PADL, pe, H, w, ws.seam.p, lb[cur], lb[cur ^ 1], m,
                                      ws.flags.p, st);
    }));
    cur ^= 1;
    if (++m == RPEND) {
      SC_CUDA(timed("compact", st, [&] { return launch_compact_lazy(img, pitch, H, w - 1, lb[cur], m, st); }));
      m = 0;
    }
  }
  if (m > 0) SC_CUDA(timed("compact", st, [&] { return launch_compact_lazy(img, pitch, H, W - count, lb[cur], m, st); }));
  return SC_OK;
}

int check_carve_args(const void *img, int H, int W, int C, int tw, int th, const void *out) {
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

int carve_impl(const uint8_t *img, int H, int W, int C, int tw, int th, uint8_t *out, int32_t *seam_log,
               int64_t *cost_log, cudaStream_t st, bool forward) {
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
  // forward energy keeps three cost planes, R rows apart
  const int64_t pstride = forward ? (int64_t)R * pe : 0;
  if (forward) SC_CUDA(ws.E.ensure((size_t)3 * R * pe));
  auto energy = [&](const uint32_t *words, int rows, int cols) {
    return forward ? launch_forward(words, pitch, rows, cols, ws.E.p + E_PADL, pe, pstride, st)
                   : launch_energy(words, pitch, rows, cols, ws.E.p + E_PADL, pe, st);
  };
  SC_CUDA(timed("pack", st, [&] { return launch_pack(img, H, W, C, ws.img.p, pitch, st); }));
  SC_CUDA(timed("energy", st, [&] { return energy(ws.img.p, H, W); }));
  const int nv = W - tw, nh = H - th;
  rc = carve_pass_plain(ws, ws.img.p, pitch, H, W, nv, pe, seam_log, cost_log, st, pstride);
  if (rc) return rc;
  if (nh > 0) {
    SC_CUDA(timed("transpose", st, [&] { return launch_transpose(ws.img.p, pitch, H, tw, ws.img2.p, pitch, st); }));  // tw x H
    SC_CUDA(timed("energy", st, [&] { return energy(ws.img2.p, tw, H); }));
    rc = carve_pass_plain(ws, ws.img2.p, pitch, tw, H, nh, pe, seam_log ? seam_log + (size_t)nv * H : nullptr,
                          cost_log ? cost_log + nv : nullptr, st, pstride);
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
  // a stream with no earlier work has fresh (uninitialised) flag words: they start at zero
  if ((rc = ensure_flags(ws, st))) return rc;
  SC_CUDA(cudaStreamSynchronize(st));
  int h[2] = {0, 0};
  SC_CUDA(cudaMemcpy(h, ws.flags.p, 2 * sizeof(int), cudaMemcpyDeviceToHost));
  SC_CUDA(cudaMemset(ws.flags.p, 0, 2 * sizeof(int)));
  int e = h[0];
  if (int *ge = device_error_word()) {
    int g = 0;
    SC_CUDA(cudaMemcpy(&g, ge, sizeof(int), cudaMemcpyDeviceToHost));
    if (g) SC_CUDA(cudaMemset(ge, 0, sizeof(int)));
    e |= g;
  }
  int sbits = 0;
  if ((rc = static_pending_errors(&sbits))) return rc;
  e |= sbits;
  if (e & ERR_TIMEOUT) return fail(SC_ETIMEOUT, "a bounded device wait ran out (error word 0x%x)", e);
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
  if ((rc = ensure_wide(ws, H, W, 1))) return rc;
  SC_CUDA(cudaMemsetAsync(ws.flags.p + 1, 0, sizeof(int), st));
  SC_CUDA(launch_copy_energy(energy, H, W, ws.E.p + E_PADL, pe, ws.flags.p + 1, st));
  return launch_search(ws, ws.E.p, pe, H, W, seam_out, nullptr, cost_out, ws.flags.p + 1, st);
}

int sc_find_seam_multi(const uint16_t *const *energies, int n, int H, int W, int32_t *seams_out, int64_t *costs_out,
                       void *stream) {
  if (!energies || !seams_out || n < 1) return fail(SC_EINVAL, "null pointer or empty batch");
  if (H < 1 || W < 1 || H > SC_MAX_ROWS || W > SC_MAX_COLS) return fail(SC_EINVAL, "bad shape %d x %d", H, W);
  for (int k = 0; k < n; ++k)
    if (!energies[k]) return fail(SC_EINVAL, "null energy map %d", k);
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *wsp;
  int rc = get_ws(stream, &wsp);
  if (rc) return rc;
  Workspace &ws = *wsp;
  std::lock_guard<std::mutex> lk(ws.mu);
  if ((rc = ensure_flags(ws, st))) return rc;
  const int pe = pitch_e_for(W);
  const int S = (H + KS - 1) / KS;
  const size_t e_per = (size_t)H * pe, m_per = (size_t)(S + 1) * pe;
  // a map is read in place when its rows are 16-byte aligned (W a multiple of 8, aligned base);
  // any other map is first copied into a padded workspace
  auto in_place = [&](int k) { return (W % 8) == 0 && ((uintptr_t)energies[k] & 15u) == 0; };
  int ncopy = 0;
  for (int k = 0; k < n; ++k) ncopy += !in_place(k);
  if (ncopy) SC_CUDA(ws.Emulti.ensure(e_per * ncopy));
  SC_CUDA(ws.Mmulti.ensure(m_per * n));
  SC_CUDA(ws.dargs.ensure((size_t)n));
  SC_CUDA(ws.gates.ensure((size_t)n));
  if ((rc = ensure_wide(ws, H, W, n))) return rc;
  SC_CUDA(cudaMemsetAsync(ws.gates.p, 0, (size_t)n * sizeof(int), st));
  std::vector<DpArgs> h(n);
  int c = 0;
  for (int k = 0; k < n; ++k) {
    DpArgs &a = h[k];
    if (in_place(k)) {
      a.E = energies[k];
      a.pitch_e = W;
    } else {
      uint16_t *Ek = ws.Emulti.p + e_per * c++;
      SC_CUDA(launch_copy_energy(energies[k], H, W, Ek + E_PADL, pe, ws.gates.p + k, st));
      a.E = Ek + E_PADL;
      a.pitch_e = pe;
    }
    a.H = H;
    a.W = W;
    a.Mrow = ws.Mmulti.p + m_per * k + E_PADL;
    a.pitch_m = pe;
    a.seam = seams_out + (size_t)k * H;
    a.seam_log = nullptr;
    a.cost = costs_out ? costs_out + k : nullptr;
    a.err = ws.flags.p;
    a.gate = ws.gates.p + k;
  }
  // up to MULTI_INLINE maps' arguments travel in the launches themselves; more go through a copy
  std::unique_ptr<MultiArgs> inl;
  if (n <= MULTI_INLINE) {
    inl.reset(new MultiArgs());
    for (int k = 0; k < n; ++k) inl->a[k] = h[k];
  } else {
    SC_CUDA(cudaMemcpyAsync(ws.dargs.p, h.data(), n * sizeof(DpArgs), cudaMemcpyHostToDevice, st));
  }
  SC_CUDA(timed("dp_multi", st, [&] { return launch_dp_multi(ws.dargs.p, inl.get(), n, H, W, st); }));
  // maps whose seam sums may not fit 24 bits (gates set by the search or the copy) were left over
  SC_CUDA(timed("dp_wide", st, [&] {
    return launch_dp_wide_multi(ws.dargs.p, inl.get(), n, H, W, ws.wdirs.p, ws.wanc.p, st);
  }));
  return SC_OK;
}

int sc_carve_forward(const uint8_t *img, int H, int W, int C, int target_w, int target_h, uint8_t *out,
                     int32_t *seam_log, int64_t *cost_log, void *stream) {
  int rc = check_carve_args(img, H, W, C, target_w, target_h, out);
  if (rc) return rc;
  const int need = target_h < H ? (W > H ? W : H) : W;
  if (need > dp_forward_max_width())
    return fail(SC_EINVAL, "forward energy searches at most %d columns (this carve needs %d)", dp_forward_max_width(),
                need);
  return carve_impl(img, H, W, C, target_w, target_h, out, seam_log, cost_log, (cudaStream_t)stream, true);
}

int sc_forward_costs(const uint8_t *img, int H, int W, int C, uint16_t *cu, uint16_t *dl, uint16_t *dr,
                     void *stream) {
  if (!img || !cu || !dl || !dr) return fail(SC_EINVAL, "null pointer");
  if (H < 1 || W < 1 || H > SC_MAX_ROWS || W > SC_MAX_COLS || !valid_c(C))
    return fail(SC_EINVAL, "bad shape %d x %d x %d", H, W, C);
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *wsp;
  int rc = get_ws(stream, &wsp);
  if (rc) return rc;
  Workspace &ws = *wsp;
  std::lock_guard<std::mutex> lk(ws.mu);
  const int pitch = round_up(W, 4);
  const int pe = pitch_e_for(W);
  const int64_t pstride = (int64_t)H * pe;
  SC_CUDA(ws.img.ensure((size_t)H * pitch));
  SC_CUDA(ws.E.ensure((size_t)3 * H * pe));
  SC_CUDA(launch_pack(img, H, W, C, ws.img.p, pitch, st));
  SC_CUDA(launch_forward(ws.img.p, pitch, H, W, ws.E.p + E_PADL, pe, pstride, st));
  SC_CUDA(launch_unpad_energy(ws.E.p + E_PADL, pe, H, W, cu, st));
  SC_CUDA(launch_unpad_energy(ws.E.p + E_PADL + pstride, pe, H, W, dl, st));
  SC_CUDA(launch_unpad_energy(ws.E.p + E_PADL + 2 * pstride, pe, H, W, dr, st));
  return SC_OK;
}

int sc_find_seam_forward(const uint16_t *cu, const uint16_t *dl, const uint16_t *dr, int H, int W, int32_t *seam_out,
                         int64_t *cost_out, void *stream) {
  if (!cu || !dl || !dr || !seam_out) return fail(SC_EINVAL, "null pointer");
  if (H < 1 || W < 1 || H > SC_MAX_ROWS || W > dp_forward_max_width())
    return fail(SC_EINVAL, "bad shape %d x %d (forward energy takes at most %d columns)", H, W, dp_forward_max_width());
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *wsp;
  int rc = get_ws(stream, &wsp);
  if (rc) return rc;
  Workspace &ws = *wsp;
  std::lock_guard<std::mutex> lk(ws.mu);
  if ((rc = ensure_flags(ws, st))) return rc;
  const int pe = pitch_e_for(W);
  const int64_t pstride = (int64_t)H * pe;
  SC_CUDA(ws.E.ensure((size_t)3 * H * pe));
  SC_CUDA(ws.Mrow.ensure((size_t)((H + KS - 1) / KS + 1) * pe));
  if ((rc = ensure_wide(ws, H, W, 1))) return rc;
  SC_CUDA(cudaMemsetAsync(ws.flags.p + 1, 0, sizeof(int), st));
  SC_CUDA(launch_copy_planes(cu, dl, dr, H, W, ws.E.p + E_PADL, pe, pstride, ws.flags.p + 1, st));
  return launch_search(ws, ws.E.p, pe, H, W, seam_out, nullptr, cost_out, ws.flags.p + 1, st, pstride);
}

int sc_enlarge(const uint8_t *img, int H, int W, int C, int target_w, uint8_t *out, int32_t *cols_out, void *stream) {
  const int k = target_w - W;
  if (!img || !out) return fail(SC_EINVAL, "null pointer");
  if (k < 1 || k > W - 1) return fail(SC_EINVAL, "target_w %d outside (W, 2W) for W = %d", target_w, W);
  int rc = check_carve_args(img, H, W, C, W - k, H, out);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *wsp;
  if ((rc = get_ws(stream, &wsp))) return rc;
  Workspace &ws = *wsp;
  const int nwords = (W + 31) / 32;
  {
    std::lock_guard<std::mutex> lk(ws.mu);
    if ((rc = ensure_flags(ws, st))) return rc;
    SC_CUDA(ws.enl_log.ensure((size_t)k * H));
    SC_CUDA(ws.enl_tmp.ensure((size_t)H * (W - k) * C));
    SC_CUDA(ws.enl_bits.ensure((size_t)H * nwords));
  }
  // the k seams the carve would remove, each in its own shrinking image's columns
  if ((rc = carve_impl(img, H, W, C, W - k, H, ws.enl_tmp.p, ws.enl_log.p, nullptr, st))) return rc;
  std::lock_guard<std::mutex> lk(ws.mu);
  SC_CUDA(timed("enlarge_map", st, [&] {
    return launch_enlarge_map(ws.enl_log.p, H, W, k, ws.enl_bits.p, cols_out, ws.flags.p, st);
  }));
  SC_CUDA(timed("insert", st, [&] { return launch_insert(img, H, W, C, ws.enl_bits.p, out, target_w, st); }));
  return SC_OK;
}

int sc_selftest_wait_timeout(int limit_us, void *stream) {
  if (limit_us < 1 || limit_us > 1000000) return fail(SC_EINVAL, "limit must be 1 us .. 1 s");
  cudaStream_t st = (cudaStream_t)stream;
  Workspace *wsp;
  int rc = get_ws(stream, &wsp);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(wsp->mu);
  if ((rc = ensure_flags(*wsp, st))) return rc;
  SC_CUDA(launch_wait_selftest((uint64_t)limit_us * 1000u, wsp->flags.p, st));
  return SC_OK;
}

int sc_greedy_seam(const uint16_t *energy, int H, int W, int32_t *seam_out, int64_t *cost_out, void *stream) {
  if (!energy || !seam_out) return fail(SC_EINVAL, "null pointer");
  if (H < 1 || W < 1 || H > SC_MAX_ROWS || W > SC_MAX_COLS) return fail(SC_EINVAL, "bad shape %d x %d", H, W);
  SC_CUDA(timed("greedy", (cudaStream_t)stream,
                [&] { return launch_greedy(energy, H, W, seam_out, cost_out, (cudaStream_t)stream); }));
  return SC_OK;
}

int sc_find_seam_multi_capacity(int H, int W, int *n_out) {
  if (!n_out) return fail(SC_EINVAL, "null pointer");
  if (H < 1 || W < 1 || H > SC_MAX_ROWS || W > SC_MAX_COLS) return fail(SC_EINVAL, "bad shape %d x %d", H, W);
  SC_CUDA(dp_multi_capacity(H, W, n_out));
  return SC_OK;
}

int sc_find_seam_multi_shape(int warps, int tile_rows) {
  if (dp_multi_set_shape(warps, tile_rows) != 0)
    return fail(SC_EINVAL, "no multi-search shape with %d warps and %d-row tiles", warps, tile_rows);
  return SC_OK;
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

}  // extern "C"

namespace sc {

// ---- batched carve (one persistent launch; images wider than a CTA go to the cluster path) ----
static const BatchCfg kBatchCfgs[] = {{15, 16}, {15, 8}, {12, 8}, {12, 16}, {8, 16}, {8, 8}, {8, 32}};
// load-balancing thresholds the autotuner times on top of its fastest configuration: images whose
// work exceeds thr x the mean share per SM go to latency-shaped clusters; autotune = 2 takes
// kBalanceDefault without timing
static const float kBalanceThr[] = {0.8f, 1.0f, 1.2f, 1.4f, 1.7f, 2.0f};
constexpr float kBalanceDefault = 1.4f;

int batch_need_width(const sc_image_desc &d) {
  const int nh = d.H - d.target_h;
  return nh > 0 ? (d.W > d.H ? d.W : d.H) : d.W;
}


// Scratch of one image in the pool at `off` (pool may be null to size it). `limit` is the widest
// column range the search stages: the CTA's width, or the cluster's owned columns.
static BatchItem layout_item(const sc_image_desc &d, int limit, unsigned char *pool, size_t &off, int *S_out) {
  const int nh = d.H - d.target_h;
  const int R = d.H > d.W ? d.H : d.W;
  const int rows_max = (nh > 0 && d.target_w > d.H) ? d.target_w : d.H;
  const int cols_max = nh > 0 ? R : d.W;
  BatchItem it;
  it.img = d.img;
  it.out = d.out;
  it.seam_log = d.seam_log;
  it.cost_log = nullptr;
  it.H = d.H; it.W = d.W; it.C = d.C; it.tw = d.target_w; it.th = d.target_h;
  it.pitch = round_up(R, 4);
  // the search stages columns [-KT - 64, limit + 64) whatever the image width
  it.pe = pitch_e_for(cols_max > limit + 64 ? cols_max : limit + 64);
  it.pad = 0;
  it.done = nullptr;
  const int S = (rows_max + KS - 1) / KS;
  *S_out = S;
  auto take = [&](size_t bytes) { unsigned char *p = pool ? pool + off : nullptr; off += a256(bytes); return p; };
  it.img_w = (uint32_t *)take((size_t)d.H * it.pitch * 4);
  it.img2_w = nh > 0 ? (uint32_t *)take((size_t)d.target_w * it.pitch * 4) : nullptr;
  it.E = (uint16_t *)take((size_t)rows_max * it.pe * 2);
  it.Mrow = (uint32_t *)take((size_t)(S + 1) * it.pe * 4);
  it.seam = (int32_t *)take((size_t)rows_max * 4);
  it.lists = (int16_t *)take((size_t)2 * rows_max * RPEND * 2);
  return it;
}

int batch_cluster_size(const sc_image_desc &d) {
  const int own = batch_cl_own_cols();
  return (batch_need_width(d) + own - 1) / own;
}

// Estimated carving time, for load balancing: per seam of an h-row, w-column map, c + h (a + b w)
// microseconds, fitted to measured per-seam times of single images (one GB300, 240..1280 columns,
// 180..944 rows): the per-row term is the chain of dependent rows, the per-column term the row's
// work. One CTA of the one-CTA kernel: c 8.3, a 0.0874, b 9.34e-5 (a row costs as much as 936
// columns: small images cost far more per pixel than large ones). A cluster of cs CTAs of the
// latency shape: c 11.5, a 0.065, b 1.5e-4 / cs. The 8-row-tile cluster shape is counted as one
// CTA on a map cs / 2 times narrower.
struct SeamCost {
  double c, a, b;
};
static SeamCost cost_one_cta() { return {8.3, 0.0874, 9.34e-5}; }
static SeamCost cost_cluster(int shape, int cs) {
  return shape == CL_LAT ? SeamCost{11.5, 0.065, 1.5e-4 / cs} : SeamCost{8.3, 0.0874, 9.34e-5 * 2.0 / cs};
}
// n seams of an h-row map whose width starts at w and drops by one per seam
static double pass_us(const SeamCost &k, double h, double w, double n) {
  return n * (k.c + h * k.a) + h * k.b * (n * w - n * (n - 1) / 2.0);
}
static double carve_us(int H, int W, int tw, int th, const SeamCost &k) {
  return pass_us(k, H, W, W - tw) + pass_us(k, tw, H, H - th);
}
static double item_us(const sc_image_desc &d, const SeamCost &k) {
  return carve_us(d.H, d.W, d.target_w, d.target_h, k);
}

static int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

// Lays out every batched image's scratch in one pool (offsets; `pool` may be null to size it):
// images that one CTA of configuration c covers first, then the wider ones by cluster size.
void batch_layout(const sc_image_desc *descs, int n, const BatchCfg &c, unsigned char *pool, BatchSetup &b) {
  b.items.clear();
  b.cl.clear();
  b.fallback.clear();
  b.Smax = 1;
  size_t off = 0;
  const int limit = batch_width_limit(c.nw, c.kt);
  std::vector<int> wide;
  // the images that would hold up the batch on one CTA each: carving work above thr_bal x the mean
  // share per SM goes to a latency-shaped cluster (the batch then ends when the average SM does,
  // not when the largest image does)
  std::vector<char> bal(n, 0);
  if (c.thr_bal > 0.f) {
    const int sms = c.sms > 0 ? c.sms : device_sms();
    double total = 0.0;
    for (int k = 0; k < n; ++k) total += item_us(descs[k], cost_one_cta());
    const double share = sms > 0 ? total / sms : 0.0;
    for (int k = 0; k < n && share > 0.0; ++k) bal[k] = item_us(descs[k], cost_one_cta()) > share * c.thr_bal ? 1 : 0;
  }
  if (c.lat_us > 0.f)
    for (int k = 0; k < n; ++k)
      if (item_us(descs[k], cost_one_cta()) > c.lat_us) bal[k] = 1;
  for (int k = 0; k < n; ++k) {
    const sc_image_desc &d = descs[k];
    const int nh0 = d.H - d.target_h;
    const int rows0 = (nh0 > 0 && d.target_w > d.H) ? d.target_w : d.H;
    // the refreshed pairs of a pass live in the CTA's staging ring between searches
    const size_t ring_bytes = (size_t)3 * c.kt * (c.nw * (128 - 2 * c.kt) + 2 * c.kt) * 2;
    if (batch_need_width(d) > limit || (size_t)rows0 * 4 > ring_bytes || bal[k]) {
      wide.push_back(k);
      continue;
    }
    int S;
    b.items.push_back(layout_item(d, limit, pool, off, &S));
    if (S > b.Smax) b.Smax = S;
  }
  for (int k : wide) {
    const sc_image_desc &d = descs[k];
    int shape = CL_WIDE, cs = batch_cluster_size(d);
    if (bal[k] || c.wide_lat) {
      const int own = batch_cl_own_cols(CL_LAT);
      const int cl = std::max(2, (batch_need_width(d) + own - 1) / own);
      if (cl <= MAX_CLUSTER) {
        shape = CL_LAT;
        cs = cl;
      }
    }
    if (cs > MAX_CLUSTER) {
      b.fallback.push_back(k);
      continue;
    }
    ClusterGroup *g = nullptr;
    for (ClusterGroup &x : b.cl)
      if (x.cs == cs && x.shape == shape) g = &x;
    if (!g) {
      b.cl.emplace_back();
      g = &b.cl.back();
      g->cs = cs;
      g->shape = shape;
    }
    int S;
    g->items.push_back(layout_item(d, cs * batch_cl_own_cols(shape), pool, off, &S));
    g->index.push_back(k);
    if (S > g->Smax) g->Smax = S;
  }
  b.pool_bytes = off;
  // the queues hand out the longest carves first (longest-processing-time order), so that no
  // CTA starts a long image after the others have run dry
  auto by_time = [](const SeamCost &k) {
    return [k](const BatchItem &a, const BatchItem &c) {
      return carve_us(a.H, a.W, a.tw, a.th, k) > carve_us(c.H, c.W, c.tw, c.th, k);
    };
  };
  std::stable_sort(b.items.begin(), b.items.end(), by_time(cost_one_cta()));
  for (ClusterGroup &g : b.cl) {
    const auto longer = by_time(cost_cluster(g.shape, g.cs));
    std::vector<int> order(g.items.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return longer(g.items[x], g.items[y]); });
    std::vector<BatchItem> items;
    std::vector<int> index;
    for (int q : order) {
      items.push_back(g.items[q]);
      index.push_back(g.index[q]);
    }
    g.items.swap(items);
    g.index.swap(index);
  }
}

static int check_batch_descs(const sc_image_desc *descs, int n) {
  if (!descs || n < 1) return fail(SC_EINVAL, "empty batch");
  for (int k = 0; k < n; ++k) {
    const sc_image_desc &d = descs[k];
    int rc = check_carve_args(d.img, d.H, d.W, d.C, d.target_w, d.target_h, d.out);
    if (rc) return fail(rc, "descriptor %d: %s", k, g_last_error.c_str());
  }
  return SC_OK;
}

// the widest configuration whose shared memory fits this batch and that covers the most images
static BatchCfg default_batch_cfg(const sc_image_desc *descs, int n) {
  BatchCfg best = kBatchCfgs[0];
  int best_cover = -1;
  for (const BatchCfg &c : kBatchCfgs) {
    BatchSetup b;
    batch_layout(descs, n, c, nullptr, b);
    if (batch_smem_bytes(c.nw, c.kt, b.Smax) > 232448 - 1024) continue;
    const int cover = (int)b.items.size();
    if (cover > best_cover) { best_cover = cover; best = c; }
  }
  return best;
}

struct BatchRun {
  DevBuf<unsigned char> pool;
  DevBuf<BatchItem> items;      // one-CTA images, then every cluster group's images
  DevBuf<int> queue;            // one counter for the one-CTA launch and one per cluster group
  BatchSetup setup;
  BatchCfg cfg{15, 16};
  int grid = 1;
  std::vector<int> cl_clusters;   // clusters launched per group
  BatchRun() = default;
  BatchRun(const BatchRun &) = delete;
  BatchRun &operator=(const BatchRun &) = delete;
};

static double batch_item_us(const BatchItem &it, const SeamCost &k) { return carve_us(it.H, it.W, it.tw, it.th, k); }

// Longest-processing-time makespan of the times t (longest first) on `slots` identical workers: how
// a persistent launch whose queue hands out the longest carves first ends.
static double lpt_makespan(const std::vector<double> &t, int slots) {
  if (t.empty()) return 0.0;
  if (slots < 1) return 1e300;
  std::priority_queue<double, std::vector<double>, std::greater<double>> q;
  for (int k = 0; k < slots && k < (int)t.size(); ++k) q.push(0.0);
  double end = 0.0;
  for (double x : t) {
    const double f = q.top() + x;
    q.pop();
    q.push(f);
    end = std::max(end, f);
  }
  return end;
}

// Allocates and uploads everything one batched launch needs (synchronous upload).
static int batch_prepare(BatchRun &r, const sc_image_desc *descs, int n, const BatchCfg &c) {
  r.cfg = c;
  batch_layout(descs, n, c, nullptr, r.setup);
  SC_CUDA(r.pool.ensure(r.setup.pool_bytes ? r.setup.pool_bytes : 256));
  batch_layout(descs, n, c, r.pool.p, r.setup);
  const int nb = (int)r.setup.items.size();
  const int ng = (int)r.setup.cl.size();
  std::vector<BatchItem> all = r.setup.items;
  for (const ClusterGroup &g : r.setup.cl) all.insert(all.end(), g.items.begin(), g.items.end());
  SC_CUDA(r.items.ensure(all.empty() ? 1 : all.size()));
  SC_CUDA(r.queue.ensure((size_t)1 + ng));
  if (!all.empty())
    SC_CUDA(cudaMemcpy(r.items.p, all.data(), all.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
  int dev = 0, sms = 1;
  SC_CUDA(cudaGetDevice(&dev));
  SC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = batch_blocks_per_sm(c.nw, c.kt, r.setup.Smax);
  // Clusters per group: the counts that minimise the estimated end of the batch. Each part ends as
  // its longest-first schedule does: one-CTA images on the SMs the clusters leave (estimated time,
  // x per_sm when CTAs share an SM), a group's images on its clusters (estimated time on a cluster
  // of its shape and size). For every end time T a group can reach, each group takes the fewest
  // clusters that end by T and the one-CTA images the SMs left over; the T whose batch ends first
  // wins. At least one cluster per group, never more than resident at once (on an otherwise idle
  // GPU) or than the group has images; the one-CTA launch keeps at least one SM.
  r.cl_clusters.assign(ng, 1);
  std::vector<double> t1;
  for (const BatchItem &it : r.setup.items) t1.push_back(batch_item_us(it, cost_one_cta()) * per_sm);
  std::vector<std::vector<double>> mk(ng);   // mk[g][c - 1]: group g's end on c clusters
  for (int g = 0; g < ng; ++g) {
    const ClusterGroup &G = r.setup.cl[g];
    std::vector<double> tg;
    for (const BatchItem &it : G.items) tg.push_back(batch_item_us(it, cost_cluster(G.shape, G.cs)));
    int cap = 0;
    SC_CUDA(batch_cl_capacity(G.cs, G.Smax, &cap, G.shape));
    const int lim = std::max(1, std::min(cap, (int)G.items.size()));
    for (int q = 1; q <= lim; ++q) mk[g].push_back(lpt_makespan(tg, q));   // (items longest first)
  }
  if (nb == 0) {
    for (int g = 0; g < ng; ++g) r.cl_clusters[g] = (int)mk[g].size();   // the GPU is the clusters'
  } else if (ng > 0) {
    double best = 1e300;
    std::vector<int> cnt(ng);
    for (int g0 = 0; g0 < ng; ++g0) {
      for (double T : mk[g0]) {
        int used = 0;
        double e = 0.0;
        for (int g = 0; g < ng; ++g) {
          int q = 1;
          while (q < (int)mk[g].size() && mk[g][q - 1] > T) ++q;
          cnt[g] = q;
          used += q * r.setup.cl[g].cs;
          e = std::max(e, mk[g][q - 1]);
        }
        if (used > sms - 1) continue;
        e = std::max(e, lpt_makespan(t1, (sms - used) * per_sm));
        if (e < best) {
          best = e;
          r.cl_clusters = cnt;
        }
      }
    }
    // when no candidate leaves the one-CTA launch an SM, every group keeps one cluster and the
    // launches share the GPU's SMs as they free up
  }
  int cl_sms = 0;
  for (int g = 0; g < ng; ++g) cl_sms += r.cl_clusters[g] * r.setup.cl[g].cs;
  // the one-CTA launch leaves the clusters' SMs to them: they run side by side
  r.grid = (sms - (nb > 0 ? std::min(cl_sms, sms - 1) : 0)) * per_sm;
  if (r.grid > nb) r.grid = nb;
  if (r.grid < 1) r.grid = 1;
  return SC_OK;
}

// the launches of one batched carve (what a plan captures)
static cudaError_t batch_launches(BatchRun &r, cudaStream_t st, int *err) {
  const int nb = (int)r.setup.items.size();
  const int ng = (int)r.setup.cl.size();
  cudaError_t e = cudaMemsetAsync(r.queue.p, 0, (size_t)(1 + ng) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  // The launches form one chain on st: every cluster group, then the one-CTA launch, each a
  // programmatic dependent of the one before. A cluster launch triggers its dependents as soon as
  // every one of its CTAs is resident, so the next launch starts beside it at once and the clusters
  // have their SMs (grouped by GPC) before the one-CTA launch spreads over the rest; each launch
  // waits for its predecessor before it ends, so work after the chain follows all of them.
  size_t base = nb;
  for (int g = 0; g < ng; ++g) {
    const ClusterGroup &G = r.setup.cl[g];
    e = launch_batch_cl(r.items.p + base, (int)G.items.size(), G.cs, G.Smax, r.cl_clusters[g], r.queue.p + 1 + g,
                        err, st, G.shape, g > 0);
    if (e != cudaSuccess) return e;
    base += G.items.size();
  }
  if (nb) {
    e = launch_batch(r.cfg.nw, r.cfg.kt, r.items.p, nb, r.setup.Smax, r.grid, r.queue.p, err, st, ng > 0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static int batch_enqueue(BatchRun &r, const sc_image_desc *descs, cudaStream_t st, int *err) {
  if (!r.setup.items.empty() || !r.setup.cl.empty())
    SC_CUDA(timed("carve_batch", st, [&] { return batch_launches(r, st, err); }));
  for (int k : r.setup.fallback) {
    const sc_image_desc &d = descs[k];
    int rc = carve_impl(d.img, d.H, d.W, d.C, d.target_w, d.target_h, d.out, d.seam_log, nullptr, st);
    if (rc) return rc;
  }
  return SC_OK;
}

}  // namespace sc

struct sc_batch_plan {
  sc::BatchRun run;
  std::vector<sc_image_desc> descs;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int *err = nullptr;
};

extern "C" {

int sc_carve_batch(const sc_image_desc *descs, int n, void *stream) {
  int rc = check_batch_descs(descs, n);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int *err = device_error_word();
  if (!err) return fail(SC_ECUDA, "cannot allocate the device error word");
  static std::mutex mu;
  static std::map<std::pair<int, void *>, BatchRun *> runs;   // scratch reused per (device, stream)
  int dev = 0;
  SC_CUDA(cudaGetDevice(&dev));
  BatchRun *r;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, stream);
    auto it = runs.find(key);
    if (it == runs.end()) it = runs.emplace(key, new BatchRun()).first;
    r = it->second;
  }
  SC_CUDA(cudaStreamSynchronize(st));   // the previous batch on this stream may still use the scratch
  if ((rc = batch_prepare(*r, descs, n, default_batch_cfg(descs, n)))) return rc;
  return batch_enqueue(*r, descs, st, err);
}

int sc_batch_plan_create(const sc_image_desc *descs, int n, int autotune, void *stream, sc_batch_plan **out) {
  if (!out) return fail(SC_EINVAL, "null plan pointer");
  *out = nullptr;
  int rc = check_batch_descs(descs, n);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  sc_batch_plan *p = new sc_batch_plan();
  p->descs.assign(descs, descs + n);
  p->err = device_error_word();
  if (!p->err) { delete p; return fail(SC_ECUDA, "cannot allocate the device error word"); }
  if (autotune < 0 || autotune > 2) { delete p; return fail(SC_EINVAL, "autotune must be 0, 1 or 2"); }
  BatchCfg best = default_batch_cfg(descs, n);
  if (autotune == 2) best.thr_bal = kBalanceDefault;   // the default configuration, balanced
  if (autotune == 1) {
    // time every configuration that batches as many images as the default, on the real batch;
    // then, for the fastest, the load-balancing variants (the heaviest images on clusters)
    BatchSetup b0;
    batch_layout(descs, n, best, nullptr, b0);
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    SC_CUDA(cudaEventCreate(&e0));
    SC_CUDA(cudaEventCreate(&e1));
    auto trial_ms = [&](const BatchCfg &c, float *ms) -> int {
      BatchRun trial;
      int rc2 = batch_prepare(trial, descs, n, c);
      if (!rc2) rc2 = batch_enqueue(trial, descs, st, p->err);
      if (rc2) return rc2;
      SC_CUDA(cudaEventRecord(e0, st));
      if ((rc2 = batch_enqueue(trial, descs, st, p->err))) return rc2;
      SC_CUDA(cudaEventRecord(e1, st));
      SC_CUDA(cudaEventSynchronize(e1));
      SC_CUDA(cudaEventElapsedTime(ms, e0, e1));
      return SC_OK;
    };
    for (const BatchCfg &c : kBatchCfgs) {
      BatchSetup b;
      batch_layout(descs, n, c, nullptr, b);
      if (b.items.size() < b0.items.size()) continue;
      if (batch_smem_bytes(c.nw, c.kt, b.Smax) > 232448 - 1024) continue;
      float ms = 0.f;
      if ((rc = trial_ms(c, &ms))) { delete p; return rc; }
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
    const BatchCfg base = best;
    for (float thr : kBalanceThr) {
      BatchCfg c = base;
      c.thr_bal = thr;
      BatchSetup b;
      batch_layout(descs, n, c, nullptr, b);
      if (!b.fallback.empty() || b.cluster_images() == b0.cluster_images()) continue;   // nothing moves
      float ms = 0.f;
      if ((rc = trial_ms(c, &ms))) { delete p; return rc; }
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if ((rc = batch_prepare(p->run, descs, n, best))) { delete p; return rc; }
  // capture the batched launches (queue reset + persistent kernels) in a CUDA graph
  if (!p->run.setup.items.empty() || !p->run.setup.cl.empty()) {
    cudaStream_t cap;
    SC_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    SC_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaSuccess;
    cudaError_t e2 = batch_launches(p->run, cap, p->err);
    cudaError_t e3 = cudaStreamEndCapture(cap, &p->graph);
    cudaStreamDestroy(cap);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
      delete p;
      return fail(SC_ECUDA, "graph capture failed: %s / %s / %s", cudaGetErrorString(e1), cudaGetErrorString(e2),
                  cudaGetErrorString(e3));
    }
    SC_CUDA(cudaGraphInstantiate(&p->exec, p->graph, 0));
  }
  *out = p;
  return SC_OK;
}

int sc_batch_plan_run(sc_batch_plan *plan, void *stream) {
  if (!plan) return fail(SC_EINVAL, "null plan");
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->exec) SC_CUDA(timed("carve_batch", st, [&] { return cudaGraphLaunch(plan->exec, st); }));
  for (int k : plan->run.setup.fallback) {
    const sc_image_desc &d = plan->descs[k];
    int rc = carve_impl(d.img, d.H, d.W, d.C, d.target_w, d.target_h, d.out, d.seam_log, nullptr, st);
    if (rc) return rc;
  }
  return SC_OK;
}

int sc_batch_route(const sc_image_desc *descs, int n, float thr, int sms, int *cluster_size, int *shape,
                   double *one_cta_us) {
  if (!descs || n < 1 || !cluster_size || !shape) return fail(SC_EINVAL, "empty batch or null output");
  if (!(thr >= 0.f) || sms < 1) return fail(SC_EINVAL, "need thr >= 0 and sms >= 1");
  for (int k = 0; k < n; ++k) {
    const sc_image_desc &d = descs[k];
    // only the sizes matter here: the descriptor's own address stands in for the image pointers
    const int rc = check_carve_args(&d, d.H, d.W, d.C, d.target_w, d.target_h, &d);
    if (rc) return fail(rc, "descriptor %d: %s", k, g_last_error.c_str());
  }
  BatchCfg c = default_batch_cfg(descs, n);
  c.thr_bal = thr;
  c.sms = sms;
  BatchSetup b;
  batch_layout(descs, n, c, nullptr, b);
  for (int k = 0; k < n; ++k) {
    cluster_size[k] = 0;
    shape[k] = CL_WIDE;
    if (one_cta_us) one_cta_us[k] = item_us(descs[k], cost_one_cta());
  }
  for (const ClusterGroup &g : b.cl)
    for (int k : g.index) {
      cluster_size[k] = g.cs;
      shape[k] = g.shape;
    }
  for (int k : b.fallback) cluster_size[k] = -1;
  return SC_OK;
}

int sc_batch_plan_info(const sc_batch_plan *plan, int *nw, int *kt, int *grid, int *batched, int *fallback) {
  if (!plan) return fail(SC_EINVAL, "null plan");
  if (nw) *nw = plan->run.cfg.nw;
  if (kt) *kt = plan->run.cfg.kt;
  if (grid) *grid = plan->run.grid;
  if (batched) *batched = (int)plan->run.setup.items.size();
  if (fallback) *fallback = plan->run.setup.cluster_images() + (int)plan->run.setup.fallback.size();
  return SC_OK;
}

int sc_batch_plan_destroy(sc_batch_plan *plan) {
  if (!plan) return SC_OK;
  cudaDeviceSynchronize();
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  plan->run.pool.release();
  plan->run.items.release();
  plan->run.queue.release();
  delete plan;
  return SC_OK;
}

}  // extern "C"
