"""Thin Python binding of libsc_gb300 (include/sc.h): argument marshalling only.

Every step of the seam-carving path runs in the library's CUDA kernels; PyTorch only provides
device memory and the current stream. There is no CPU fallback: if the library is missing or no
GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

_lib = None
_lock = threading.Lock()

SC_OK, SC_EINVAL, SC_ENOMEM, SC_ECUDA, SC_ETIMEOUT, SC_EBUSY, SC_EINTERNAL = 0, -1, -2, -3, -4, -5, -6
MAX_ROWS = 8192
MAX_COLS = 8192


class ScError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sc status {code}: {msg}")
        self.code = code


class ImageDesc(ctypes.Structure):
    _fields_ = [
        ("img", ctypes.c_void_p), ("out", ctypes.c_void_p), ("seam_log", ctypes.c_void_p),
        ("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int),
        ("target_w", ctypes.c_int), ("target_h", ctypes.c_int), ("reserved", ctypes.c_int),
    ]


def header_functions() -> List[str]:
    """Names of the functions include/sc.h declares."""
    with open(os.path.join(_build.INCLUDE, "sc.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sc_\w+)\s*\(", text, flags=re.M)))


def load(path: Optional[str] = None):
    """Load the shared library (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or _build.build()
            lib = ctypes.CDLL(p)
            P, I = ctypes.c_void_p, ctypes.c_int
            sig = {
                "sc_version": ([], I),
                "sc_last_error": ([], ctypes.c_char_p),
                "sc_check": ([P], I),
                "sc_release_workspaces": ([], I),
                "sc_energy": ([P, I, I, I, P, P], I),
                "sc_find_seam": ([P, I, I, P, P, P], I),
                "sc_find_seam_static": ([P, I, I, P, P, P], I),
                "sc_find_seam_static_selftest": ([I, I, P, P, P], I),
                "sc_find_seam_multi": ([P, I, I, I, P, P, P], I),
                "sc_batch_route": ([P, I, ctypes.c_float, I, P, P, P], I),
                "sc_greedy_seam": ([P, I, I, P, P, P], I),
                "sc_enlarge": ([P, I, I, I, I, P, P, P], I),
                "sc_selftest_wait_timeout": ([I, P], I),
                "sc_forward_costs": ([P, I, I, I, P, P, P, P], I),
                "sc_find_seam_forward": ([P, P, P, I, I, P, P, P], I),
                "sc_carve_forward": ([P, I, I, I, I, I, P, P, P, P], I),
                "sc_find_seam_multi_capacity": ([I, I, P], I),
                "sc_find_seam_multi_shape": ([I, I], I),
                "sc_carve": ([P, I, I, I, I, I, P, P, P, P], I),
                "sc_carve_plain": ([P, I, I, I, I, I, P, P, P, P], I),
                "sc_carve_host": ([P, I, I, I, I, I, P, P], I),
                "sc_carve_batch": ([P, I, P], I),
                "sc_batch_plan_create": ([P, I, I, P, P], I),
                "sc_batch_plan_run": ([P, P], I),
                "sc_batch_plan_info": ([P, P, P, P, P, P], I),
                "sc_batch_plan_destroy": ([P], I),
                "sc_timing_enable": ([I], I),
                "sc_timing_reset": ([], I),
                "sc_timing_read": ([ctypes.c_char_p, P, P], I),
                "sc_probe_copy_bandwidth": ([ctypes.c_size_t, I, P], I),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _raise(code: int):
    if code != SC_OK:
        raise ScError(code, load().sc_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libsc_gb300 needs a CUDA GPU; none is available")
    return torch


def _stream(torch, device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _img_shape(img) -> Tuple[int, int, int]:
    if img.dim() == 2:
        return img.shape[0], img.shape[1], 1
    if img.dim() != 3:
        raise ValueError("image must be H x W or H x W x C")
    return img.shape[0], img.shape[1], img.shape[2]


def _check_device_u8(img):
    if img.device.type != "cuda" or str(img.dtype) != "torch.uint8" or not img.is_contiguous():
        raise ValueError("image must be a contiguous uint8 CUDA tensor")


def version() -> int:
    return load().sc_version()


def check(device=None) -> None:
    """Wait for the current stream and raise if a device-side check failed."""
    torch = _torch()
    _raise(load().sc_check(_stream(torch, device)))


def energy(img):
    """e1 energy of an H x W x C uint8 CUDA image -> H x W uint16 CUDA tensor."""
    torch = _torch()
    _check_device_u8(img)
    H, W, C = _img_shape(img)
    out = torch.empty((H, W), dtype=torch.uint16, device=img.device)
    _raise(load().sc_energy(_ptr(img), H, W, C, _ptr(out), _stream(torch, img.device)))
    return out


def find_seam(e):
    """Algorithm 3 seam of an H x W uint16 CUDA energy map -> (int32[H] seam, int64[1] cost)."""
    torch = _torch()
    if e.device.type != "cuda" or e.dtype != torch.uint16 or e.dim() != 2 or not e.is_contiguous():
        raise ValueError("energy must be a contiguous H x W uint16 CUDA tensor")
    H, W = e.shape
    seam = torch.empty(H, dtype=torch.int32, device=e.device)
    cost = torch.empty(1, dtype=torch.int64, device=e.device)
    _raise(load().sc_find_seam(_ptr(e), H, W, _ptr(seam), _ptr(cost), _stream(torch, e.device)))
    return seam, cost


def enlarge(img, target_w: int, with_cols: bool = False):
    """Seam insertion: widen a CUDA uint8 image (H x W x C or H x W) to target_w = W + k,
    1 <= k <= W - 1. Returns the widened image, or (image, cols[k, H]) with ``with_cols``."""
    torch = _torch()
    _check_device_u8(img)
    H, W, C = _img_shape(img)
    k = int(target_w) - W
    shape = (H, int(target_w)) if img.dim() == 2 else (H, int(target_w), C)
    out = torch.empty(shape, dtype=torch.uint8, device=img.device)
    cols = torch.empty((max(k, 1), H), dtype=torch.int32, device=img.device) if with_cols else None
    _raise(load().sc_enlarge(_ptr(img), H, W, C, int(target_w), _ptr(out), _ptr(cols) if with_cols else None,
                             _stream(torch, img.device)))
    return (out, cols) if with_cols else out


def selftest_wait_timeout(limit_us: int = 1000) -> None:
    """Enqueue the bounded-wait self-test on the current stream (sc_check then raises SC_ETIMEOUT)."""
    torch = _torch()
    _raise(load().sc_selftest_wait_timeout(int(limit_us), _stream(torch, torch.device("cuda", torch.cuda.current_device()))))


def forward_costs(img):
    """Forward-energy planes (CU, DL, DR) of a CUDA uint8 image: three H x W uint16 CUDA tensors."""
    torch = _torch()
    _check_device_u8(img)
    H, W, C = _img_shape(img)
    planes = [torch.empty((H, W), dtype=torch.uint16, device=img.device) for _ in range(3)]
    _raise(load().sc_forward_costs(_ptr(img), H, W, C, *[_ptr(t) for t in planes], _stream(torch, img.device)))
    return tuple(planes)


def find_seam_forward(cu, dl, dr):
    """Algorithm 3 with forward costs on three H x W uint16 CUDA planes -> (int32[H] seam, int64[1] cost)."""
    torch = _torch()
    for t in (cu, dl, dr):
        if t.device.type != "cuda" or t.dtype != torch.uint16 or t.dim() != 2 or not t.is_contiguous() or t.shape != cu.shape:
            raise ValueError("planes must be contiguous H x W uint16 CUDA tensors of one shape")
    H, W = cu.shape
    seam = torch.empty(H, dtype=torch.int32, device=cu.device)
    cost = torch.empty(1, dtype=torch.int64, device=cu.device)
    _raise(load().sc_find_seam_forward(_ptr(cu), _ptr(dl), _ptr(dr), H, W, _ptr(seam), _ptr(cost),
                                       _stream(torch, cu.device)))
    return seam, cost


def carve_forward(img, target_w: int, target_h: int, with_log: bool = False):
    """sc_carve with forward energy; returns the carved image (and the seam and cost logs)."""
    torch = _torch()
    _check_device_u8(img)
    H, W, C = _img_shape(img)
    shape = (target_h, target_w) if img.dim() == 2 else (target_h, target_w, C)
    out = torch.empty(shape, dtype=torch.uint8, device=img.device)
    log = cost = None
    if with_log:
        n = (W - target_w) * H + (H - target_h) * target_w
        log = torch.empty(max(n, 1), dtype=torch.int32, device=img.device)
        cost = torch.empty(max(W - target_w + H - target_h, 1), dtype=torch.int64, device=img.device)
    _raise(load().sc_carve_forward(_ptr(img), H, W, C, int(target_w), int(target_h), _ptr(out), _ptr(log), _ptr(cost),
                                   _stream(torch, img.device)))
    if with_log:
        nv, nh = W - target_w, H - target_h
        return out, log[: nv * H + nh * target_w], cost[: nv + nh]
    return out


def greedy_seam(e):
    """Algorithm 2's greedy seam of an H x W uint16 CUDA energy map -> (int32[H] seam, int64[1] cost)."""
    torch = _torch()
    if e.device.type != "cuda" or e.dtype != torch.uint16 or e.dim() != 2 or not e.is_contiguous():
        raise ValueError("energy must be a contiguous H x W uint16 CUDA tensor")
    H, W = e.shape
    seam = torch.empty(H, dtype=torch.int32, device=e.device)
    cost = torch.empty(1, dtype=torch.int64, device=e.device)
    _raise(load().sc_greedy_seam(_ptr(e), H, W, _ptr(seam), _ptr(cost), _stream(torch, e.device)))
    return seam, cost


def find_seam_multi(energies):
    """The Algorithm 3 search of n same-size H x W uint16 CUDA maps in one launch (one cluster per
    map) -> (int32[n, H] seams, int64[n] costs); equal to n calls of find_seam."""
    torch = _torch()
    es = list(energies)
    if not es:
        raise ValueError("need at least one energy map")
    e0 = es[0]
    if e0.device.type != "cuda" or e0.dim() != 2:
        raise ValueError("energies must be contiguous H x W uint16 CUDA tensors of one shape and device")
    H, W = e0.shape
    shape0, dev0, u16 = e0.shape, e0.get_device(), torch.uint16
    ptrs = []
    for e in es:   # one pass, cheap checks: this runs on every call
        if e.dtype is not u16 or e.shape != shape0 or not e.is_contiguous() or e.get_device() != dev0:
            raise ValueError("energies must be contiguous H x W uint16 CUDA tensors of one shape and device")
        ptrs.append(e.data_ptr())
    n = len(es)
    seams = torch.empty((n, H), dtype=torch.int32, device=e0.device)
    costs = torch.empty(n, dtype=torch.int64, device=e0.device)
    ptrs = (ctypes.c_void_p * n)(*ptrs)
    _raise(load().sc_find_seam_multi(ptrs, n, H, W, _ptr(seams), _ptr(costs), _stream(torch, es[0].device)))
    return seams, costs


def find_seam_multi_capacity(H: int, W: int) -> int:
    """How many H x W maps find_seam_multi keeps resident at once on the current device."""
    _torch()
    n = ctypes.c_int(0)
    _raise(load().sc_find_seam_multi_capacity(H, W, ctypes.byref(n)))
    return n.value


def find_seam_multi_shape(warps: int = 0, tile_rows: int = 0) -> None:
    """Fix find_seam_multi's tile shape (compute warps per CTA, DP tile rows); (0, 0) = automatic."""
    _raise(load().sc_find_seam_multi_shape(warps, tile_rows))


def find_seam_static(e):
    """sc_find_seam_static: the same search as find_seam, with the library's fixed scratch array
    instead of allocated scratch (for callers that must not allocate device memory)."""
    torch = _torch()
    if e.device.type != "cuda" or e.dtype != torch.uint16 or e.dim() != 2 or not e.is_contiguous():
        raise ValueError("energy must be a contiguous H x W uint16 CUDA tensor")
    H, W = e.shape
    seam = torch.empty(H, dtype=torch.int32, device=e.device)
    cost = torch.empty(1, dtype=torch.int64, device=e.device)
    _raise(load().sc_find_seam_static(_ptr(e), H, W, _ptr(seam), _ptr(cost), _stream(torch, e.device)))
    return seam, cost


def find_seam_static_selftest(H: int, limit_us: int = 1000, device=None):
    """sc_find_seam_static_selftest: the static search's device-error path without a fault (a
    bounded wait that runs out). Returns the (int32[H] seam, int64[1] cost) outputs it wrote."""
    torch = _torch()
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    seam = torch.zeros(H, dtype=torch.int32, device=dev)
    cost = torch.zeros(1, dtype=torch.int64, device=dev)
    _raise(load().sc_find_seam_static_selftest(int(limit_us), int(H), _ptr(seam), _ptr(cost), _stream(torch, dev)))
    return seam, cost


def carve(img, target_w: int, target_h: int, with_log: bool = False, plain: bool = False):
    """Remove (W - target_w) vertical then (H - target_h) horizontal seams on the GPU.

    Returns the target_h x target_w x C uint8 CUDA tensor, or (out, seam_log, cost_log) with
    ``with_log``. ``plain`` selects the per-seam-launch baseline path (same result)."""
    torch = _torch()
    _check_device_u8(img)
    H, W, C = _img_shape(img)
    shape = (target_h, target_w) if img.dim() == 2 else (target_h, target_w, C)
    out = torch.empty(shape, dtype=torch.uint8, device=img.device)
    log = cost = None
    if with_log:
        n = (W - target_w) * H + (H - target_h) * target_w
        log = torch.empty(max(n, 1), dtype=torch.int32, device=img.device)
        cost = torch.empty(max(W - target_w + H - target_h, 1), dtype=torch.int64, device=img.device)
    fn = load().sc_carve_plain if plain else load().sc_carve
    _raise(fn(_ptr(img), H, W, C, int(target_w), int(target_h), _ptr(out), _ptr(log), _ptr(cost),
              _stream(torch, img.device)))
    if with_log:
        nv, nh = W - target_w, H - target_h
        return out, log[: nv * H + nh * target_w], cost[: nv + nh]
    return out


def carve_host(img: np.ndarray, target_w: int, target_h: int, stream=None) -> np.ndarray:
    """sc_carve_host: host image in, host image out (copies inside the call)."""
    torch = _torch()
    a = np.ascontiguousarray(img, dtype=np.uint8)
    if a.ndim == 2:
        a = a[:, :, None]
    H, W, C = a.shape
    out = np.empty((target_h, target_w, C), dtype=np.uint8)
    st = ctypes.c_void_p(stream) if stream is not None else _stream(torch, None)
    _raise(load().sc_carve_host(ctypes.c_void_p(a.ctypes.data), H, W, C, int(target_w), int(target_h),
                                ctypes.c_void_p(out.ctypes.data), st))
    return out if img.ndim == 3 else out[:, :, 0]


def _batch_descs(imgs, targets, with_log):
    torch = _torch()
    descs = (ImageDesc * len(imgs))()
    outs, logs = [], []
    for k, (img, (tw, th)) in enumerate(zip(imgs, targets)):
        _check_device_u8(img)
        H, W, C = _img_shape(img)
        shape = (th, tw) if img.dim() == 2 else (th, tw, C)
        out = torch.empty(shape, dtype=torch.uint8, device=img.device)
        outs.append(out)
        log = None
        if with_log:
            log = torch.empty(max((W - tw) * H + (H - th) * tw, 1), dtype=torch.int32, device=img.device)
        logs.append(log)
        descs[k] = ImageDesc(img.data_ptr(), out.data_ptr(), log.data_ptr() if log is not None else 0,
                             H, W, C, int(tw), int(th), 0)
    return descs, outs, logs


def carve_batch(imgs: Sequence, targets: Sequence[Tuple[int, int]], with_log: bool = False):
    """sc_carve_batch over CUDA images (one persistent launch); returns the outputs (and seam logs)."""
    torch = _torch()
    descs, outs, logs = _batch_descs(imgs, targets, with_log)
    dev = imgs[0].device if len(imgs) else None
    _raise(load().sc_carve_batch(ctypes.cast(descs, ctypes.c_void_p), len(imgs), _stream(torch, dev)))
    return (outs, logs) if with_log else outs


class BatchPlan:
    """sc_batch_plan: scratch, descriptor table and a CUDA graph of the persistent launch, built once
    (optionally autotuned) and replayed by run(). The input tensors must stay alive and keep their
    storage; their contents may change between runs."""

    def __init__(self, imgs: Sequence, targets: Sequence[Tuple[int, int]], autotune=False,
                 with_log: bool = False):
        """autotune: False/0 default configuration, True/1 time the configurations and balancing
        variants, 2 default configuration with the heaviest images on 32-row-tile clusters."""
        torch = _torch()
        self.imgs = list(imgs)
        self.descs, self.outs, self.logs = _batch_descs(self.imgs, targets, with_log)
        self.device = self.imgs[0].device
        h = ctypes.c_void_p(0)
        _raise(load().sc_batch_plan_create(ctypes.cast(self.descs, ctypes.c_void_p), len(self.imgs),
                                           int(autotune), _stream(torch, self.device), ctypes.byref(h)))
        self._h = h

    def run(self):
        torch = _torch()
        _raise(load().sc_batch_plan_run(self._h, _stream(torch, self.device)))
        return self.outs

    def info(self) -> dict:
        v = [ctypes.c_int(0) for _ in range(5)]
        _raise(load().sc_batch_plan_info(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("compute_warps", "tile_rows", "ctas", "batched", "cluster_path"), (x.value for x in v)))

    def close(self):
        if getattr(self, "_h", None):
            load().sc_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_route(sizes, thr: float = 1.4, sms: int = 152):
    """sc_batch_route: where a batch plan carves each image, computed on the host (no device call).
    sizes: (H, W, C, target_w, target_h) per image -> (cluster_size, shape, one_cta_us) lists:
    cluster_size 0 for one CTA, the cluster's CTA count, or -1 for the per-seam path; shape 0 for
    8-row-tile clusters, 1 for 32-row-tile clusters; one_cta_us the model's one-CTA carve time."""
    n = len(sizes)
    descs = (ImageDesc * max(n, 1))()
    for k, (H, W, C, tw, th) in enumerate(sizes):
        descs[k].H, descs[k].W, descs[k].C, descs[k].target_w, descs[k].target_h = H, W, C, tw, th
    cs = (ctypes.c_int * max(n, 1))()
    sh = (ctypes.c_int * max(n, 1))()
    us = (ctypes.c_double * max(n, 1))()
    _raise(load().sc_batch_route(ctypes.cast(descs, ctypes.c_void_p), n, ctypes.c_float(thr), int(sms), cs, sh, us))
    return list(cs)[:n], list(sh)[:n], list(us)[:n]


def probe_copy_bandwidth(nbytes: int, reps: int) -> float:
    """sc_probe_copy_bandwidth: GB/s (read + write) of `reps` copies of an nbytes buffer in one launch."""
    _torch()
    g = ctypes.c_double(0.0)
    _raise(load().sc_probe_copy_bandwidth(ctypes.c_size_t(nbytes), int(reps), ctypes.byref(g)))
    return g.value


def timing_enable(on: bool = True) -> None:
    _raise(load().sc_timing_enable(1 if on else 0))


def timing_reset() -> None:
    _raise(load().sc_timing_reset())


def timing_read(kernel: str) -> Tuple[float, int]:
    """(summed device ms, launches) of one kernel since the last reset; ("all") -> (0, launches)."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _raise(load().sc_timing_read(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("queued", ctypes.c_int64), ("in_flight_groups", ctypes.c_int64),
                ("groups", ctypes.c_int64), ("batched", ctypes.c_int64), ("cluster_path", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("device_errors", ctypes.c_int), ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double),
                ("max_s", ctypes.c_double)]


def _server_sigs(lib):
    P, I = ctypes.c_void_p, ctypes.c_int
    for name, args, res in (
            ("sc_server_create", [ctypes.c_size_t, I, I, P], I),
            ("sc_server_submit", [P, P, I, I, I, I, I, P, P], I),
            ("sc_server_poll", [P, ctypes.c_int64, P], I),
            ("sc_server_drain", [P, ctypes.c_double], I),
            ("sc_server_stats", [P, P], I),
            ("sc_server_destroy", [P], I)):
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res


class Server:
    """sc_server: continuous-batching request loop with a device-memory budget.

    submit() takes a host image (numpy uint8 H x W x C) and returns a ticket; the result lands in a
    pinned host array owned by this object (result(ticket)). Inputs are copied into pinned memory
    here so the server's device copies are asynchronous."""

    def __init__(self, budget_bytes: int = 40 << 30, max_batch: int = 64, streams: int = 16):
        self.torch = _torch()
        lib = load()
        _server_sigs(lib)
        h = ctypes.c_void_p(0)
        _raise(lib.sc_server_create(ctypes.c_size_t(budget_bytes), max_batch, streams, ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, img: np.ndarray, target_w: int, target_h: int, pinned: bool = True) -> int:
        """Queue a carve; with pinned=False the buffers stay pageable (the server stages them)."""
        torch = self.torch
        a = np.ascontiguousarray(img, dtype=np.uint8)
        if a.ndim == 2:
            a = a[:, :, None]
        H, W, C = a.shape
        src = torch.from_numpy(a)
        dst = torch.empty((target_h, target_w, C), dtype=torch.uint8)
        if pinned:
            src, dst = src.pin_memory(), dst.pin_memory()
        t = ctypes.c_int64(0)
        _raise(load().sc_server_submit(self._h, ctypes.c_void_p(src.data_ptr()), H, W, C, int(target_w),
                                       int(target_h), ctypes.c_void_p(dst.data_ptr()), ctypes.byref(t)))
        self._keep[t.value] = (src, dst)
        return t.value

    def poll(self, ticket: int):
        lat = ctypes.c_double(0.0)
        rc = load().sc_server_poll(self._h, ticket, ctypes.byref(lat))
        if rc < 0:
            _raise(rc)
        return rc == 1, lat.value

    def result(self, ticket: int) -> np.ndarray:
        return self._keep[ticket][1].numpy()

    def release(self, ticket: int):
        self._keep.pop(ticket, None)

    def drain(self, timeout_s: float = 600.0):
        _raise(load().sc_server_drain(self._h, ctypes.c_double(timeout_s)))

    def stats(self) -> dict:
        st = ServerStats()
        _raise(load().sc_server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().sc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
