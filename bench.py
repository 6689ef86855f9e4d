#!/usr/bin/env python3
"""Seam-carving benchmark: seams/s of the GB300 path on the 1920x1080 -> 1440 workload.

A step is one whole carve of the workload image: e1 energy once, then per seam the DP search
(fill, argmin, backtrack), local energy refresh and row compaction, all on the GPU through the C
ABI. Inputs are resident in HBM when timing starts; L2 is flushed (256 MB write) between steps,
outside the per-step CUDA-event brackets. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Multi-GPU: every rank carves its own copy (replicas, weak scaling); value = all ranks' seams /
the slowest rank's time. ``--impl reference`` times the oracle (plain C, host cores) on a bounded
sample of the same workload.

Besides the headline, rank 0 measures the other workloads (4K carve, 58 concurrent 4K searches,
the 256-image batch, the serving trace: its first 300 requests against the plain path and all
10,000 at their arrival times), an L2 copy peak for the L2 roofline fractions, and the oracle on
the host cores for every configuration; a compact ``summary`` object is the line's last key.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import random
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--plain", action="store_true", help="time the per-seam-launch plain path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched (256-image) measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving (Poisson trace) measurement")
    ap.add_argument("--no-4k", action="store_true", help="skip the 3840x2160 measurement")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper's n x n workload points")
    ap.add_argument("--serving-requests", type=int, default=300)
    ap.add_argument("--trace-requests", type=int, default=10000,
                    help="requests of the full serving-trace replay (0 skips it)")
    ap.add_argument("--profile-batch", metavar="N", type=int, default=None,
                    help="only run the first N images of the batched workload through a batch plan twice "
                         "(for ncu captures of k_batch)")
    ap.add_argument("--balanced", action="store_true",
                    help="with --profile-batch: a balanced plan (autotune = 2: the heaviest images on "
                         "latency-shaped clusters, for ncu captures of k_batch_cl)")
    ap.add_argument("--profile-search", metavar="HxW[xB]", default=None,
                    help="only call sc_find_seam a few times on a seeded HxW energy map, or sc_find_seam_multi "
                         "on B maps (for ncu captures)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_throughput(local_s: float, units: int, ws: int, device):
    """Whole-job throughput of ws independent replicas (one per rank, each doing `units` units in
    `local_s` seconds): the units of all ranks over the slowest rank's time (a MAX all-reduce over
    the process group when ws > 1). Returns (units per second, max seconds)."""
    total_s = local_s
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([local_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    return units * ws / total_s, total_s


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic_from_profile(name="k_dp_1920x1080.txt"):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary, if any."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            for ln in f:
                if ln.startswith("dram_bytes_per_launch:"):
                    return float(ln.split(":")[1])
    except OSError:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for ln in f:
                    parts = [p.strip() for p in ln.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            if self.path:
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_info():
    """Host cores and CPU model, printed beside every oracle timing."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"host_cores": os.cpu_count(), "cpu_model": model or platform.machine()}


def l2_peak(sc):
    """The L2 copy bandwidth, the denominator of the L2 roofline fractions: two 32 MiB buffers
    (inside the 126 MB L2) copied 40 times within one launch of the library's probe, read + write
    bytes over the CUDA-event time of that launch; best of 3."""
    return max(sc.probe_copy_bandwidth(32 << 20, 40) for _ in range(3))


def _workload():
    from paper_2410_21207_gb300 import synth
    return synth.config2()


def cpu_baseline(job, img, budget_s: float = 15.0):
    """The oracle (plain single-threaded C) on a bounded prefix of the workload's seams."""
    import oracle
    W, H = job.W, job.H
    t0 = time.perf_counter()
    oracle.carve(img, W - 2, H)
    per = (time.perf_counter() - t0) / 2
    n = max(2, min(W - job.target_w, int(budget_s / max(per, 1e-6))))
    t0 = time.perf_counter()
    oracle.carve(img, W - n, H)
    dt = time.perf_counter() - t0
    mpix = sum(H * (W - t) for t in range(n)) / 1e6
    return {"value": n / dt, "unit": "seams/s", "mpix_seam_per_s": mpix / dt, "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {W - job.target_w} seams of the {W}x{H} workload, single-threaded C, "
                      f"full energy recompute per seam", **cpu_info()}


def _oracle_carve_all(imgs, targets, threads):
    """oracle.carve of every image, spread over `threads` host threads (the C calls release the
    GIL), longest first; returns the wall time."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    order = sorted(range(len(imgs)), key=lambda k: -imgs[k].shape[0] * imgs[k].shape[1] *
                   (imgs[k].shape[1] - targets[k][0] + imgs[k].shape[0] - targets[k][1]))
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda k: oracle.carve(imgs[k], *targets[k]), order))
    return time.perf_counter() - t0


def cpu_oracle_configs(sample5):
    """The oracle on the host cores for configurations 3, 4 and 5: config 3's 4K carve on one
    thread over its first seams (bounded), the whole 256-image batch spread over all cores, and a
    seeded 200-request sample of the serving trace spread over all cores."""
    import oracle
    from paper_2410_21207_gb300 import synth
    info = cpu_info()
    cores = info["host_cores"] or 1
    out = dict(info)
    job = synth.config3()
    img = job.make()
    t0 = time.perf_counter()
    oracle.carve(img, job.W - 2, job.H)
    per = (time.perf_counter() - t0) / 2
    n = max(2, min(job.W - job.target_w, int(15.0 / max(per, 1e-6))))
    t0 = time.perf_counter()
    oracle.carve(img, job.W - n, job.H)
    dt = time.perf_counter() - t0
    mpix = sum(job.H * (job.W - t) for t in range(n)) / 1e6
    out["config3"] = {"seams_per_s": n / dt, "mpix_seam_per_s": mpix / dt, "threads": 1,
                      "sample": f"first {n} of 960 vertical seams of the 3840x2160 image"}
    jobs = synth.config4()
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=cores) as ex:
        imgs = list(ex.map(lambda j: j.make(), jobs))
    dt = _oracle_carve_all(imgs, [(j.target_w, j.target_h) for j in jobs], cores)
    out["config4"] = {"seams_per_s": sum(j.seams for j in jobs) / dt,
                      "mpix_seam_per_s": sum(j.mpix_seams() for j in jobs) / dt, "threads": cores,
                      "sample": "all 256 images", "s": dt}
    if sample5:
        reqs = synth.config5()
        idx = sorted(sample5)
        dt = _oracle_carve_all([sample5[k] for k in idx], [(reqs[k].target_w, reqs[k].target_h) for k in idx], cores)
        out["config5"] = {"req_per_s": len(idx) / dt, "seams_per_s": sum(reqs[k].seams for k in idx) / dt,
                          "mpix_seam_per_s": sum(reqs[k].mpix_seams() for k in idx) / dt, "threads": cores,
                          "sample": f"{len(idx)} requests drawn from the 10,000 (random.Random(5).sample)", "s": dt}
    return out


def batched_measurement(sc, torch, dev, flush, steps, peak, l2):
    """Config 4 (256 images, W 240..1280, H 180..960, width -10..40 %) as one autotuned batch plan
    (persistent kernels in a CUDA graph) against the plain path (one image at a time, per-seam
    launches) on the same 256 images. Roofline of the batch graph (k_batch, plus k_batch_cl for
    the images wider than one CTA): algorithmic bytes = 2.25 B per pixel of every searched map."""
    from paper_2410_21207_gb300 import synth
    jobs = synth.config4()
    imgs = [torch.from_numpy(j.make()).to(dev) for j in jobs]
    targets = [(j.target_w, j.target_h) for j in jobs]
    seams = sum(j.seams for j in jobs)
    mpix = sum(j.mpix_seams() for j in jobs)
    plan = sc.BatchPlan(imgs, targets, autotune=True)
    for _ in range(3):
        plan.run()
    sc.check()
    ms = []
    for _ in range(max(5, steps)):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record()
        plan.run()
        s1.record()
        torch.cuda.synchronize(dev)
        ms.append(s0.elapsed_time(s1))
    sc.check()
    info = plan.info()
    plan.close()
    bms = statistics.median(ms)
    for k in range(2):
        sc.carve(imgs[k], *targets[k], plain=True)
    torch.cuda.synchronize(dev)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record()
    for k in range(len(jobs)):
        sc.carve(imgs[k], *targets[k], plain=True)
    p1.record()
    torch.cuda.synchronize(dev)
    sc.check()
    plain_sps = seams / (p0.elapsed_time(p1) / 1000.0)
    batched_sps = seams / (bms / 1000.0)
    alg = 2.25 * mpix * 1e6
    achieved = alg / (bms / 1000.0) / 1e9
    return {"workload": "256 images, W 240..1280, H 180..960, width -10..40 % (seed 4)",
            "seams_per_batch": seams, "ms_per_batch": bms, "seams_per_s": batched_sps,
            "mpix_seam_per_s": mpix / (bms / 1000.0), "plan": info,
            "plain_seams_per_s": plain_sps, "plain_sample": "all 256 images, one image per launch sequence",
            "batched_over_plain": batched_sps / plain_sps,
            "roofline": {"kernel": "k_batch graph (k_batch + k_batch_cl)", "bound": "hbm", "achieved": achieved,
                         "unit": "GB/s", "peak": peak, "frac": achieved / peak, "l2_peak": l2,
                         "l2_frac": achieved / l2 if l2 else None, "algorithmic_bytes_per_batch": alg,
                         "traffic": _traffic_from_profile("k_batch_config4.txt"),
                         "note": "the whole carve runs inside the graph; algorithmic bytes count the "
                                 "energy+DP pass only (2.25 B per pixel per searched map)"}}


_TRACE = {}
TRACE_CANVASES = 8


def _trace(n):
    """The serving trace (cached per process: building all 10,000 requests takes a second or two)."""
    from paper_2410_21207_gb300 import synth
    if n not in _TRACE:
        _TRACE[n] = synth.config5(n=n)
    return _TRACE[n]


def _gen_request(args):
    """Worker (spawned process): pixels of request k of the serving trace."""
    import sys as _sys
    _sys.path.insert(0, ROOT)
    k, n = args
    return k, _trace(n)[k].make()


def _gen_canvas(k):
    """Worker (spawned process): a 4096x2160 canvas of generator G (rectangles scaled by area, as
    for every request) from which the full-trace replay crops its requests' pixels."""
    import sys as _sys
    _sys.path.insert(0, ROOT)
    from paper_2410_21207_gb300 import synth
    R, smin, smax = synth.scaled_rects(4096, 2160)
    return synth.gen_image(4096, 2160, R, smin, smax, 50000 + k)


def cpu_sample_indices():
    """The seeded 200-request sample of the trace that the oracle is timed on."""
    return sorted(random.Random(5).sample(range(10000), 200))


def pregenerate(n_serving, canvases, sample):
    """Pixels made by a spawned process pool before any GPU work in this process: the first
    n_serving requests of the trace, the replay's canvases, and the oracle's request sample."""
    from multiprocessing import get_context
    procs = max(1, min(14, (os.cpu_count() or 2) - 2))
    with get_context("spawn").Pool(procs) as pool:
        serving = dict(pool.map(_gen_request, [(k, n_serving) for k in range(n_serving)], chunksize=4)) \
            if n_serving else {}
        canv = pool.map(_gen_canvas, range(TRACE_CANVASES)) if canvases else []
        samp = dict(pool.map(_gen_request, [(k, 10000) for k in sample], chunksize=2)) if sample else {}
    return serving, canv, samp


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * (len(xs) - 1) + 0.5))] if xs else None


def serving_measurement(sc, torch, dev, imgs, n):
    """Config 5's first n requests (Poisson arrivals at 200/s, sizes log-uniform 128..4096 x
    128..2160) replayed in real time into sc_server (40 GB budget), against the plain path: the same
    arrivals served first-come first-served, one request at a time, by sc_carve_plain (device image
    in, device image out; the served path also copies host->device->host)."""
    from paper_2410_21207_gb300 import synth
    reqs = synth.config5(n=n)
    seams = sum(r.seams for r in reqs)
    srv = sc.Server(budget_bytes=40 << 30, max_batch=64, streams=16)
    warm = [srv.submit(imgs[k], reqs[k].target_w, reqs[k].target_h) for k in range(min(n, 8))]
    srv.drain()
    for t in warm:
        srv.release(t)
    st0 = srv.stats()
    # (1) the trace's arrival times, replayed in real time: latency under the offered load
    tickets = []
    t0 = time.perf_counter()
    for k, r in enumerate(reqs):
        delay = r.arrival_s - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(imgs[k], r.target_w, r.target_h))
    srv.drain(900)
    wall = time.perf_counter() - t0
    lats = [srv.poll(t)[1] for t in tickets]
    st = srv.stats()
    for t in tickets:
        srv.release(t)
    # (2) every request submitted at once: the server's capacity (throughput when never idle)
    t0 = time.perf_counter()
    tickets = [srv.submit(imgs[k], r.target_w, r.target_h) for k, r in enumerate(reqs)]
    srv.drain(900)
    cap_wall = time.perf_counter() - t0
    for t in tickets:
        srv.release(t)
    srv.close()
    # plain path: FIFO, one request at a time, per-seam launches
    dimgs = [torch.from_numpy(imgs[k]).to(dev) for k in range(n)]
    sc.carve(dimgs[0], reqs[0].target_w, reqs[0].target_h, plain=True)
    torch.cuda.synchronize(dev)
    plain_lat, clock = [], 0.0
    tp0 = time.perf_counter()
    for k, r in enumerate(reqs):
        start = max(clock, r.arrival_s)
        t1 = time.perf_counter()
        sc.carve(dimgs[k], r.target_w, r.target_h, plain=True)
        torch.cuda.synchronize(dev)
        clock = start + (time.perf_counter() - t1)
        plain_lat.append(clock - r.arrival_s)
    plain_busy = time.perf_counter() - tp0
    sc.check()
    return {"workload": f"first {n} requests of the 10,000-request trace (seed 5): Poisson 200 req/s, "
                        "W, H log-uniform 128..4096 x 128..2160, target 50..90 % x 80..100 %",
            "served": {"req_per_s": n / wall, "seams_per_s": seams / wall, "p50_ms": 1e3 * _pct(lats, 0.5),
                       "p99_ms": 1e3 * _pct(lats, 0.99), "launch_groups": st["groups"] - st0["groups"],
                       "one_cta_images": st["batched"] - st0["batched"],
                       "cluster_images": st["cluster_path"] - st0["cluster_path"],
                       "peak_device_bytes": st["peak_bytes"], "budget_bytes": st["budget_bytes"],
                       "note": "arrivals replayed in real time; throughput is bounded by the offered load"},
            "served_capacity": {"req_per_s": n / cap_wall, "seams_per_s": seams / cap_wall,
                                "note": "the same requests submitted at once (host->device->host copies included)"},
            "plain": {"req_per_s": n / plain_busy, "seams_per_s": seams / plain_busy,
                      "p50_ms": 1e3 * _pct(plain_lat, 0.5), "p99_ms": 1e3 * _pct(plain_lat, 0.99),
                      "note": "same arrivals, first-come first-served, one request at a time"},
            "served_over_plain_throughput": plain_busy / cap_wall}


def trace_replay_measurement(sc, torch, dev, canvases, n):
    """All n requests of the serving trace (Poisson arrivals at 200 req/s, sizes log-uniform
    128..4096 x 128..2160, targets 50..90 % x 80..100 %) submitted to sc_server (40 GB budget) at
    their arrival times. Each request's size, targets and arrival come from the trace; its pixels
    are a crop of one of the pre-generated canvases of generator G (making 10,000 images one by one
    would take longer than the replay). Latency = completion - scheduled arrival; finished
    requests are released as the replay goes, so host memory stays bounded."""
    import numpy as np
    reqs = _trace(10000)[:n]
    seams = sum(r.seams for r in reqs)
    mpix = sum(r.mpix_seams() for r in reqs)

    def pixels(k, r):
        c = canvases[k % len(canvases)]
        x0 = (k * 7919) % (4096 - r.W + 1)
        y0 = (k * 104729) % (2160 - r.H + 1)
        return np.ascontiguousarray(c[y0:y0 + r.H, x0:x0 + r.W])

    srv = sc.Server(budget_bytes=40 << 30, max_batch=64, streams=16)
    for k in range(8):
        srv.submit(pixels(k, reqs[k]), reqs[k].target_w, reqs[k].target_h)
    srv.drain()
    st0 = srv.stats()
    outstanding = {}
    lats = []

    def collect():
        for t in list(outstanding):
            done, lat = srv.poll(t)
            if done:
                sub, arr = outstanding.pop(t)
                lats.append(sub - arr + lat)
                srv.release(t)

    t0 = time.perf_counter()
    late = 0
    for k, r in enumerate(reqs):
        delay = r.arrival_s - (time.perf_counter() - t0)
        if delay > 0.002:
            collect()
            delay = r.arrival_s - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        else:
            late += 1
        sub = time.perf_counter() - t0
        outstanding[srv.submit(pixels(k, r), r.target_w, r.target_h)] = (sub, r.arrival_s)
    srv.drain(1800)
    wall = time.perf_counter() - t0
    collect()
    st = srv.stats()
    srv.close()
    sc.check()
    return {"workload": f"all {n} requests of the trace (seed 5) at their arrival times; pixels cropped from "
                        f"{len(canvases)} generator-G canvases of 4096x2160",
            "requests": len(lats), "wall_s": wall, "req_per_s": len(lats) / wall, "seams_per_s": seams / wall,
            "mpix_seam_per_s": mpix / wall, "p50_ms": 1e3 * _pct(lats, 0.5), "p99_ms": 1e3 * _pct(lats, 0.99),
            "max_ms": 1e3 * max(lats), "submitted_late": late,
            "launch_groups": st["groups"] - st0["groups"], "peak_device_bytes": st["peak_bytes"],
            "device_errors": st["device_errors"]}


def fourk_measurement(sc, torch, dev, flush, steps):
    """Config 3: 3840x2160 -> 2880x1620 (960 vertical + 540 horizontal seams via transposition)."""
    from paper_2410_21207_gb300 import synth
    job = synth.config3()
    img = torch.from_numpy(job.make()).to(dev)
    sc.carve(img, job.target_w, job.target_h)
    torch.cuda.synchronize(dev)
    ms = []
    for _ in range(5):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sc.carve(img, job.target_w, job.target_h)
        e1.record()
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    sc.check()
    t = statistics.median(ms) / 1000.0
    return {"workload": job.name, "seams_per_s": job.seams / t, "mpix_seam_per_s": job.mpix_seams() / t,
            "ms_per_carve": 1e3 * t, "runs": len(ms)}


def uhd_search_measurement(sc, torch, dev, steps, peak, l2):
    """The energy+DP pass at 3840x2160 with B independent maps in flight (one cluster each, B = how
    many fit on the GPU at once): the bandwidth view of the search, next to the single-map latency
    chain. Algorithmic bytes = H*W*2.25 per map (energy read + one direction record). The maps are
    the e1 energy of config 3's image (sc_energy) and column rotations of it."""
    from paper_2410_21207_gb300 import synth
    H, W = 2160, 3840
    B = max(1, sc.find_seam_multi_capacity(H, W))
    e = sc.energy(torch.from_numpy(synth.config3().make()).to(dev))
    maps = [torch.roll(e.view(torch.int16), 37 * k, dims=1).view(torch.uint16).contiguous() for k in range(B)]
    sc.check()
    for _ in range(3):
        sc.find_seam_multi(maps)
    torch.cuda.synchronize(dev)
    ms = []
    for _ in range(max(5, steps)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sc.find_seam_multi(maps)
        e1.record()
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    # the same calls back to back (no wait in between): the host's preparation of a call overlaps
    # the previous call's kernels, as in a pipeline
    reps = max(10, steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        sc.find_seam_multi(maps)
    e1.record()
    torch.cuda.synchronize(dev)
    t_pipe = e0.elapsed_time(e1) / 1000.0 / reps
    sc.timing_reset()
    sc.timing_enable(True)
    for _ in range(max(5, steps)):
        sc.find_seam_multi(maps)
    torch.cuda.synchronize(dev)
    sc.timing_enable(False)
    k_ms, k_n = sc.timing_read("dp_multi")
    sc.check()
    t = statistics.median(ms) / 1000.0
    tk = k_ms / 1000.0 / max(k_n, 1)
    alg = 2.25 * H * W * B
    return {"workload": f"energy+DP pass (seam search) on {B} concurrent 3840x2160 maps", "maps": B,
            "us_per_call": 1e6 * t, "seams_per_s": B / t, "mpix_seam_per_s": B * H * W / 1e6 / t,
            "kernel": "k_dp_multi", "kernel_us_per_launch": 1e6 * tk,
            "algorithmic_bytes_per_launch": alg, "achieved_gbs": alg / tk / 1e9,
            "peak_gbs": peak, "frac": alg / tk / 1e9 / peak if peak else None,
            "l2_peak_gbs": l2, "l2_frac": alg / tk / 1e9 / l2 if l2 else None,
            "call_gbs": alg / t / 1e9, "call_frac": alg / t / 1e9 / peak if peak else None,
            "us_per_call_pipelined": 1e6 * t_pipe, "call_frac_pipelined": alg / t_pipe / 1e9 / peak if peak else None,
            "traffic": _traffic_from_profile("k_dp_multi_3840x2160x58.txt") if B == 58 else None,
            "note": "working set B x 16.6 MB exceeds L2, so no flush; us_per_call is one call waited for "
                    "(host preparation included while the GPU idles), us_per_call_pipelined the same calls "
                    "back to back; the kernel figure is k_dp_multi alone"}


def forward_measurement(sc, torch, dev, img, tw, th, seams):
    """The headline carve with forward energy instead of e1 (three cost planes per pixel)."""
    sc.carve_forward(img, tw, th)
    torch.cuda.synchronize(dev)
    ms = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sc.carve_forward(img, tw, th)
        e1.record()
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    sc.check()
    t = statistics.median(ms) / 1000.0
    return {"workload": "1920x1080 -> 1440x1080, forward energy", "ms_per_carve": 1e3 * t, "seams_per_s": seams / t}


def enlarge_measurement(sc, torch, dev, img):
    """Seam insertion: the 1920x1080 image widened to 2400 (480 seams found by the carve, mapped
    back to the input and inserted)."""
    out = sc.enlarge(img, 2400)
    torch.cuda.synchronize(dev)
    ms = []
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sc.enlarge(img, 2400)
        e1.record()
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    sc.check()
    t = statistics.median(ms) / 1000.0
    return {"workload": "1920x1080 -> 2400x1080 (480 inserted seams)", "ms": 1e3 * t, "seams_per_s": 480 / t,
            "out_shape": list(out.shape)}


def paper_workload_measurement(sc, torch, dev, cpu: bool):
    """The paper's own workload ("Runtime For different sized images"): n x n images at n = 180,
    360, 480, 720, 1080 with s = 0.5, i.e. n/2 vertical seams. On the GPU: one DP seam search
    T(n, n) (sc_find_seam), one greedy seam (sc_greedy_seam, Algorithm 2) and the full DP carve
    C(n, n, 0.5) (sc_carve); on one host core, the oracle's DP seam, greedy seam and full carve, and
    brute force (Algorithm 1) at n = 2, 5, 7, 10, 12 (the paper's brute-force sizes)."""
    import numpy as np
    from paper_2410_21207_gb300 import synth
    import oracle

    def ev_ms(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    def cpu_s(fn, budget_s=1.0):
        t0 = time.perf_counter()
        fn()
        t = time.perf_counter() - t0
        reps = max(1, min(20, int(budget_s / max(t, 1e-6))))
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        return (time.perf_counter() - t0) / reps

    rows = []
    for n in (180, 360, 480, 720, 1080):
        R, smin, smax = synth.scaled_rects(n, n)
        img = synth.gen_image(n, n, R, smin, smax, 7000 + n)
        dimg = torch.from_numpy(img).to(dev)
        e = sc.energy(dimg)
        row = {"n": n, "seams": n // 2,
               "gpu_dp_seam_ms": ev_ms(lambda: sc.find_seam(e), 20),
               "gpu_greedy_seam_ms": ev_ms(lambda: sc.greedy_seam(e), 20),
               "gpu_dp_carve_ms": ev_ms(lambda: sc.carve(dimg, n - n // 2, n), 3)}
        if cpu:
            e_host = oracle.energy(img)
            row["cpu_dp_seam_ms"] = 1e3 * cpu_s(lambda: oracle.dp_seam(e_host))
            row["cpu_greedy_seam_ms"] = 1e3 * cpu_s(lambda: oracle.greedy_seam(e_host))
            row["cpu_dp_carve_ms"] = 1e3 * cpu_s(lambda: oracle.carve(img, n - n // 2, n), 0.0)
        rows.append(row)
    sc.check()
    out = {"workload": "n x n synthetic images (generator G), s = 0.5: n/2 vertical seams", "points": rows}
    if cpu:
        rng = np.random.default_rng(425)
        out["cpu_brute_force_seam_ms"] = {
            str(n): 1e3 * cpu_s(lambda e=rng.integers(0, 1531, size=(n, n)).astype(np.uint16): oracle.brute_seam(e), 0.2)
            for n in (2, 5, 7, 10, 12)}
        out["cpu_cores"] = 1
    return out


def profile_search(spec: str):
    """sc_find_seam four times on a seeded H x W uint16 energy map (the kernel to capture is k_dp);
    with HxWxB, sc_find_seam_multi on B shifted copies (the kernel is k_dp_multi)."""
    import numpy as np
    import torch
    from paper_2410_21207_gb300 import binding as sc
    dims = [int(x) for x in spec.lower().split("x")]
    H, W = dims[0], dims[1]
    B = dims[2] if len(dims) > 2 else 0
    e = np.random.default_rng(0).integers(0, 1531, size=(H, W)).astype(np.uint16)
    t = torch.from_numpy(e).to("cuda:0")
    maps = [torch.from_numpy(np.ascontiguousarray(np.roll(e, 37 * k, axis=1))).to("cuda:0") for k in range(B)]
    for _ in range(4):
        if B:
            sc.find_seam_multi(maps)
        else:
            sc.find_seam(t)
    torch.cuda.synchronize()
    sc.check()
    print(json.dumps({"profile_search": spec, "ok": True}))
    return 0


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    job = _workload()
    img = job.make()
    import oracle
    W, H = job.W, job.H
    t0 = time.perf_counter()
    oracle.carve(img, W - 2, H)
    per = (time.perf_counter() - t0) / 2
    n = max(2, min(W - job.target_w, int(20.0 / max(a.steps, 1) / max(per, 1e-6))))
    for _ in range(a.warmup):
        oracle.carve(img, W - 1, H)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.carve(img, W - n, H)
        times.append(time.perf_counter() - t0)
    dt = sum(times)
    value = n * a.steps / dt
    line = {
        "impl": "reference", "metric": "seams/s", "value": value, "unit": "seams/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * dt / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{job.name}; each step = the first {n} seams (bounded sample)",
                   "parallelism": "single-threaded CPU oracle"},
        "cpu_baseline": {"value": value, "unit": "seams/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {n} of {W - job.target_w} seams per step", **cpu_info()},
        "e2e": {"value": value, "unit": "seams/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_native(a):
    import numpy as np
    import torch

    from paper_2410_21207_gb300 import binding as sc

    ws, rank, local = _dist()
    serving_imgs, canvases, sample5 = None, [], {}
    if rank == 0:
        # pixels made before any GPU work (a spawned pool)
        serving_imgs, canvases, sample5 = pregenerate(
            0 if a.no_serving else a.serving_requests,
            not a.no_serving and a.trace_requests > 0,
            cpu_sample_indices() if (not a.no_cpu_baseline and ws == 1) else [])
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    job = _workload()
    img_np = job.make()
    H, W, tw, th = job.H, job.W, job.target_w, job.target_h
    seams = (W - tw) + (H - th)
    mpix = job.mpix_seams()
    img = torch.from_numpy(img_np).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        return sc.carve(img, tw, th, plain=a.plain)

    for _ in range(max(a.warmup, 3)):
        step()
    sc.check()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed_steps(instrumented: bool):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
        if instrumented:
            sc.timing_reset()
            sc.timing_enable(True)
        barrier()
        for k in range(a.steps):
            flush.zero_()
            starts[k].record()
            step()
            ends[k].record()
        barrier()
        if instrumented:
            sc.timing_enable(False)
        sc.check()
        return [st.elapsed_time(en) for st, en in zip(starts, ends)]

    # headline: uninstrumented
    with ClockSampler(local if ws > 1 else 0) as clk:
        step_ms = timed_steps(False)
    # the same steps again with the library bracketing every k_dp launch with CUDA events
    timed_steps(True)
    dp_ms, dp_n = sc.timing_read("dp")
    _, launches = sc.timing_read("all")
    launches //= max(1, a.steps)
    value, total_s = replica_throughput(sum(step_ms) / 1000.0, seams * a.steps, ws, dev)

    # roofline of the dominant kernel (the DP seam search): algorithmic bytes = H*W_cur*2.25 per launch
    dp_bytes = 2.25 * sum(H * (W - t) for t in range(W - tw)) + 2.25 * sum(tw * (H - t) for t in range(H - th))
    dp_bytes_per_launch = dp_bytes / max(seams, 1)
    achieved = (dp_bytes * a.steps) / (dp_ms / 1000.0) / 1e9 if dp_ms > 0 else None
    peak, peak_src = _peaks()
    l2 = l2_peak(sc)
    traffic = _traffic_from_profile()

    line = {
        "metric": "seams/s", "value": value, "unit": "seams/s", "n_gpus": ws, "steps": a.steps,
        "warmup": max(a.warmup, 3), "ms_per_step": 1000.0 * total_s / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": job.name + (" [plain path]" if a.plain else ""), "seams_per_step": seams,
                   "mpix_seam_per_step": round(mpix, 1), "image": f"{W}x{H} RGB uint8 (synthetic generator G, seed 2)",
                   "l2": "flushed between steps (256 MB write), outside the timed brackets",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "mpix_seam_per_s": mpix * a.steps * ws / total_s,
        "gpu_launches": int(launches) * a.steps,
        "roofline": {"kernel": "k_dp (seam search)", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "peak_source": peak_src, "l2_peak": l2, "l2_frac": (achieved / l2) if achieved else None,
                     "dp_ms_per_launch": dp_ms / max(dp_n, 1), "algorithmic_bytes_per_launch": dp_bytes_per_launch},
        "clocks": clk.summary(),
    }

    if rank == 0 and not a.no_e2e:
        pinned = torch.from_numpy(img_np).pin_memory()
        host_in = pinned.numpy()
        t_e2e = []
        for k in range(max(2, a.steps)):
            t0 = time.perf_counter()
            sc.carve_host(host_in, tw, th)
            t_e2e.append(time.perf_counter() - t0)
        e2e_s = statistics.median(t_e2e[1:]) if len(t_e2e) > 1 else t_e2e[0]
        line["e2e"] = {"value": seams / e2e_s, "unit": "seams/s", "h2d_bytes_per_step": H * W * 3,
                       "d2h_bytes_per_step": th * tw * 3}
    if rank == 0 and not a.no_batched:
        line["batched"] = batched_measurement(sc, torch, dev, flush, a.steps, peak, l2)
    if rank == 0 and not a.no_4k:
        line["uhd_3840x2160"] = fourk_measurement(sc, torch, dev, flush, a.steps)
        line["uhd_search_concurrent"] = uhd_search_measurement(sc, torch, dev, a.steps, peak, l2)
    if rank == 0 and not a.no_paper:
        line["enlarge_1920x1080"] = enlarge_measurement(sc, torch, dev, img)
        line["forward_energy_1920x1080"] = forward_measurement(sc, torch, dev, img, tw, th, seams)
        line["paper_nxn"] = paper_workload_measurement(sc, torch, dev, cpu=not a.no_cpu_baseline and ws == 1)
    if rank == 0 and serving_imgs:
        line["serving"] = serving_measurement(sc, torch, dev, serving_imgs, a.serving_requests)
    if rank == 0 and canvases:
        line["serving_trace"] = trace_replay_measurement(sc, torch, dev, canvases, a.trace_requests)
    if rank == 0 and not a.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(job, img_np)
        line["cpu_oracle"] = cpu_oracle_configs(sample5)
    if rank == 0:
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def summary(line):
    """The headline figures of every workload in a few hundred bytes (the line's last key, so
    that a reader who keeps only the end of the output still has them)."""
    def r(x, nd=3):
        return None if x is None else round(float(x), nd)
    out = {"c2_seams_s": r(line["value"], 0), "k_dp_us": r(1e3 * line["roofline"]["dp_ms_per_launch"], 1),
           "k_dp_hbm_frac": r(line["roofline"]["frac"], 4), "k_dp_l2_frac": r(line["roofline"]["l2_frac"], 4),
           "l2_peak_gbs": r(line["roofline"]["l2_peak"], 0)}
    if "e2e" in line:
        out["c2_e2e_seams_s"] = r(line["e2e"]["value"], 0)
    if "uhd_3840x2160" in line:
        out["c3_seams_s"] = r(line["uhd_3840x2160"]["seams_per_s"], 0)
    if "uhd_search_concurrent" in line:
        u = line["uhd_search_concurrent"]
        out["uhd_maps"] = u["maps"]
        out["uhd_kernel_us"] = r(u["kernel_us_per_launch"], 1)
        out["uhd_call_us"] = r(u["us_per_call"], 1)
        out["uhd_call_pipe_us"] = r(u["us_per_call_pipelined"], 1)
        out["uhd_hbm_frac"] = r(u["frac"])
        out["uhd_l2_frac"] = r(u["l2_frac"])
        out["uhd_call_hbm_frac"] = r(u["call_frac"])
    if "batched" in line:
        b = line["batched"]
        out["c4_seams_s"] = r(b["seams_per_s"], 0)
        out["c4_over_plain"] = r(b["batched_over_plain"], 2)
        out["k_batch_hbm_frac"] = r(b["roofline"]["frac"])
        out["k_batch_l2_frac"] = r(b["roofline"]["l2_frac"])
    if "serving" in line:
        sv = line["serving"]
        out["c5_300_p50_ms"] = r(sv["served"]["p50_ms"], 1)
        out["c5_300_p99_ms"] = r(sv["served"]["p99_ms"], 1)
        out["c5_capacity_over_plain"] = r(sv["served_over_plain_throughput"], 2)
    if "serving_trace" in line:
        t = line["serving_trace"]
        out["c5_full_requests"] = t["requests"]
        out["c5_full_p50_ms"] = r(t["p50_ms"], 1)
        out["c5_full_p99_ms"] = r(t["p99_ms"], 1)
        out["c5_full_req_s"] = r(t["req_per_s"], 1)
    if "forward_energy_1920x1080" in line:
        out["fwd_c2_seams_s"] = r(line["forward_energy_1920x1080"]["seams_per_s"], 0)
    if "cpu_oracle" in line:
        c = line["cpu_oracle"]
        out["cpu"] = {"cores": c["host_cores"], "model": c["cpu_model"],
                      "c2_seams_s": r(line["cpu_baseline"]["value"], 1),
                      "c3_seams_s": r(c["config3"]["seams_per_s"], 1),
                      "c4_seams_s": r(c["config4"]["seams_per_s"], 1)}
        if "config5" in c:
            out["cpu"]["c5_req_s"] = r(c["config5"]["req_per_s"], 2)
    return out


def profile_batch(n: int, balanced: bool = False):
    """The first n images of the batched workload through a batch plan (no autotuning, or the
    default balancing), run twice (the kernels to capture are k_batch and k_batch_cl)."""
    import torch
    from paper_2410_21207_gb300 import binding as sc
    from paper_2410_21207_gb300 import synth
    jobs = synth.config4()[:n]
    imgs = [torch.from_numpy(j.make()).to("cuda:0") for j in jobs]
    plan = sc.BatchPlan(imgs, [(j.target_w, j.target_h) for j in jobs], autotune=2 if balanced else 0)
    for _ in range(2):
        plan.run()
    torch.cuda.synchronize()
    sc.check()
    info = plan.info()
    plan.close()
    print(json.dumps({"profile_batch": n, "plan": info, "ok": True}))
    return 0


def main():
    a = _args()
    if a.profile_search:
        return profile_search(a.profile_search)
    if a.profile_batch:
        return profile_batch(a.profile_batch, a.balanced)
    if a.impl == "reference":
        return run_reference(a)
    return run_native(a)


if __name__ == "__main__":
    sys.exit(main())
