"""Seam-carving oracle (test infrastructure only).

A plain, slow, single-threaded C implementation (``sc_oracle.c``) of what the seam-carving hot
path computes, written from arXiv 2410.21207: the e1 energy ("Energy Mapping"), Algorithm 1
(brute force), Algorithm 2 (greedy), Algorithm 3 (dynamic programming), seam removal ("Removal
of Seams") and the repeated loop with horizontal seams by transposition ("Design Techniques").
The readings taken where the paper is silent or garbled are listed at the top of
``sc_oracle.c``.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import this package.
It shares no code with the CUDA library, and nothing here reads a value the CUDA library
produced. This wrapper only marshals numpy arrays into the C functions; it holds no arithmetic
of the method. ``build()`` compiles the C file with gcc into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile sc_oracle.c into a shared library (gcc -O2); returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if force or not fresh:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i = ctypes.c_int
            lib.orc_energy.argtypes = [P, i, i, i, P]
            lib.orc_energy.restype = None
            lib.orc_dp_seam.argtypes = [P, i, i, P]
            lib.orc_dp_seam.restype = ctypes.c_int64
            lib.orc_dp_last_row.argtypes = [P, i, i, P]
            lib.orc_dp_last_row.restype = None
            lib.orc_greedy_seam.argtypes = [P, i, i, P]
            lib.orc_greedy_seam.restype = ctypes.c_int64
            lib.orc_brute_seam.argtypes = [P, i, i, P, P]
            lib.orc_brute_seam.restype = ctypes.c_int64
            lib.orc_remove_seam.argtypes = [P, i, i, i, P, P]
            lib.orc_remove_seam.restype = None
            lib.orc_transpose.argtypes = [P, i, i, i, P]
            lib.orc_transpose.restype = None
            lib.orc_carve.argtypes = [P, i, i, i, i, i, P, P, P]
            lib.orc_carve.restype = ctypes.c_int
            lib.orc_enlarge.argtypes = [P, i, i, i, i, P, P]
            lib.orc_enlarge.restype = ctypes.c_int
            lib.orc_forward_costs.argtypes = [P, i, i, i, P, P, P]
            lib.orc_forward_costs.restype = None
            lib.orc_dp_seam_forward.argtypes = [P, P, P, i, i, P]
            lib.orc_dp_seam_forward.restype = ctypes.c_int64
            lib.orc_carve_forward.argtypes = [P, i, i, i, i, i, P, P, P]
            lib.orc_carve_forward.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _img(img) -> tuple[np.ndarray, int, int, int]:
    a = np.ascontiguousarray(img, dtype=np.uint8)
    if a.ndim == 2:
        a = a[:, :, None]
    if a.ndim != 3:
        raise ValueError("image must be H x W or H x W x C")
    H, W, C = a.shape
    return a, H, W, C


def energy(img) -> np.ndarray:
    """e1 energy of an H x W x C uint8 image -> H x W uint16."""
    a, H, W, C = _img(img)
    e = np.empty((H, W), dtype=np.uint16)
    _load().orc_energy(_ptr(a), H, W, C, _ptr(e))
    return e


def _e(e) -> tuple[np.ndarray, int, int]:
    a = np.ascontiguousarray(e, dtype=np.uint16)
    if a.ndim != 2 or a.shape[0] < 1 or a.shape[1] < 1:
        raise ValueError("energy must be a non-empty H x W array")
    return a, a.shape[0], a.shape[1]


def dp_seam(e) -> tuple[np.ndarray, int]:
    """Algorithm 3: (seam[H] int32, cost)."""
    a, H, W = _e(e)
    s = np.empty(H, dtype=np.int32)
    cost = _load().orc_dp_seam(_ptr(a), H, W, _ptr(s))
    return s, int(cost)


def dp_last_row(e) -> np.ndarray:
    """The last row of Algorithm 3's cumulative cost table M, int64[W]."""
    a, H, W = _e(e)
    out = np.empty(W, dtype=np.int64)
    _load().orc_dp_last_row(_ptr(a), H, W, _ptr(out))
    return out


def greedy_seam(e) -> tuple[np.ndarray, int]:
    """Algorithm 2: (seam[H] int32, cost = sum of e along it)."""
    a, H, W = _e(e)
    s = np.empty(H, dtype=np.int32)
    cost = _load().orc_greedy_seam(_ptr(a), H, W, _ptr(s))
    return s, int(cost)


def brute_seam(e) -> tuple[np.ndarray, int, int]:
    """Algorithm 1: (seam[H] int32, cost, number of paths enumerated)."""
    a, H, W = _e(e)
    s = np.empty(H, dtype=np.int32)
    leaves = np.zeros(1, dtype=np.int64)
    cost = _load().orc_brute_seam(_ptr(a), H, W, _ptr(s), _ptr(leaves))
    return s, int(cost), int(leaves[0])


def remove_seam(img, seam) -> np.ndarray:
    a, H, W, C = _img(img)
    s = np.ascontiguousarray(seam, dtype=np.int32)
    if s.shape != (H,) or W < 2 or s.min() < 0 or s.max() >= W:
        raise ValueError("bad seam")
    out = np.empty((H, W - 1, C), dtype=np.uint8)
    _load().orc_remove_seam(_ptr(a), H, W, C, _ptr(s), _ptr(out))
    return out


def transpose(img) -> np.ndarray:
    a, H, W, C = _img(img)
    out = np.empty((W, H, C), dtype=np.uint8)
    _load().orc_transpose(_ptr(a), H, W, C, _ptr(out))
    return out


def carve(img, target_w: int, target_h: int, with_log: bool = False):
    """The full loop: (W - tw) vertical seams, then (H - th) horizontal seams by transposition.

    Returns the th x tw x C image, or (image, seam_log, cost_log) with ``with_log``. The seam log
    holds (W-tw) vertical seams of H entries, then (H-th) horizontal seams of tw entries (in the
    transposed frame)."""
    a, H, W, C = _img(img)
    if not (1 <= target_w <= W and 1 <= target_h <= H):
        raise ValueError("targets must satisfy 1 <= target <= size")
    out = np.empty((target_h, target_w, C), dtype=np.uint8)
    nv, nh = W - target_w, H - target_h
    log = np.empty(max(1, nv * H + nh * target_w), dtype=np.int32)
    costs = np.empty(max(1, nv + nh), dtype=np.int64)
    rc = _load().orc_carve(_ptr(a), H, W, C, int(target_w), int(target_h), _ptr(out), _ptr(log), _ptr(costs))
    if rc != 0:
        raise ValueError("orc_carve rejected its arguments")
    if with_log:
        return out, log[: nv * H + nh * target_w], costs[: nv + nh]
    return out


def enlarge(img, target_w: int, with_cols: bool = False):
    """Seam insertion (reading R9): widen to target_w = W + k, 1 <= k <= W - 1, by inserting a
    rounded-up mean pixel right of every input pixel on one of the first k seams the carve would
    remove. Returns the H x target_w x C image, or (image, cols) with ``with_cols`` (cols[t, i] =
    the input column seam t deletes in row i)."""
    a, H, W, C = _img(img)
    k = int(target_w) - W
    if not (1 <= k <= W - 1):
        raise ValueError("target_w must satisfy W < target_w < 2 W")
    out = np.empty((H, int(target_w), C), dtype=np.uint8)
    cols = np.empty((k, H), dtype=np.int32)
    rc = _load().orc_enlarge(_ptr(a), H, W, C, int(target_w), _ptr(out), _ptr(cols))
    if rc != 0:
        raise ValueError("orc_enlarge rejected its arguments")
    return (out, cols) if with_cols else out


def forward_costs(img) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Forward energy (reading R10): the CU, DL, DR planes (uint16 H x W) of an image."""
    a, H, W, C = _img(img)
    cu = np.empty((H, W), dtype=np.uint16)
    dl = np.empty((H, W), dtype=np.uint16)
    dr = np.empty((H, W), dtype=np.uint16)
    _load().orc_forward_costs(_ptr(a), H, W, C, _ptr(cu), _ptr(dl), _ptr(dr))
    return cu, dl, dr


def dp_seam_forward(cu, dl, dr) -> tuple[np.ndarray, int]:
    """Algorithm 3 with forward costs: (seam[H] int32, cost)."""
    cu = np.ascontiguousarray(cu, dtype=np.uint16)
    dl = np.ascontiguousarray(dl, dtype=np.uint16)
    dr = np.ascontiguousarray(dr, dtype=np.uint16)
    H, W = cu.shape
    s = np.empty(H, dtype=np.int32)
    cost = _load().orc_dp_seam_forward(_ptr(cu), _ptr(dl), _ptr(dr), H, W, _ptr(s))
    return s, int(cost)


def carve_forward(img, target_w: int, target_h: int, with_log: bool = False):
    """The full loop with forward energy (as carve, the forward costs recomputed per seam)."""
    a, H, W, C = _img(img)
    if not (1 <= target_w <= W and 1 <= target_h <= H):
        raise ValueError("targets must satisfy 1 <= target <= size")
    out = np.empty((target_h, target_w, C), dtype=np.uint8)
    nv, nh = W - target_w, H - target_h
    log = np.empty(max(1, nv * H + nh * target_w), dtype=np.int32)
    costs = np.empty(max(1, nv + nh), dtype=np.int64)
    rc = _load().orc_carve_forward(_ptr(a), H, W, C, int(target_w), int(target_h), _ptr(out), _ptr(log),
                                   _ptr(costs))
    if rc != 0:
        raise ValueError("orc_carve_forward rejected its arguments")
    if with_log:
        return out, log[: nv * H + nh * target_w], costs[: nv + nh]
    return out
