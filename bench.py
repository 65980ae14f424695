#!/usr/bin/env python
"""Benchmark of the MeshSplats hot path on GB300.

One step = one pass of the hot path over the 1,000,000-Gaussian clustered scene at
1920x1080 (SH degree 3 in bfloat16, K = 8): fan conversion with SH colour, render
(projection, tile binning, radix sort, exact-order composite), L1 loss against a
jittered-scene target, adjoint, and the two-learning-rate Adam update of the fans.

Prints one JSON line (rank 0).  `value` is rendered megapixels per second of the
forward+backward step summed over ranks (every rank runs its own replica); `e2e`
is the same step through the public API with the Gaussians copied from pinned host
memory and the loss read back inside the timed region, the next step's copy overlapping
the current step on a second stream (the serial figure is reported beside it).  `--impl reference` times
the plain CPU oracle on a bounded window of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# multiply-adds x 2 of one row of the initializer: 16x128 + 128x128 + 128x32 (padded outputs)
MLP_FLOPS_PER_ROW = 2 * (16 * 128 + 128 * 128 + 128 * 32)
# Gaussian counts of the clustered-surface scenes whose fine-tunes give the initializer's
# 4 x 125k = 500k training pairs: densities from below to the evaluated scene's
PAIR_SCENES = (250_000, 500_000, 1_000_000, 3_000_000)
METRIC = "rendered Mpix/s fwd and fwd+bwd (1080p, 1M fans) vs plain, at 1e-4 image err"
STAGES = ["mesh_build", "bin", "sort", "raster", "raster_bwd", "loss", "adam", "mlp"]
NSTAGE = len(STAGES)
# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of a stage's
# kernels on the 1M-fan 1080p workload stored in spatial order, with the digest of the kernel
# sources it was taken on; reported only while the digest still matches.  Measured on that
# workload itself (one pass per launch): work items 0.2 MB, count 193, tile prefix 24, pixel
# scan 8, pixel order 8, fill 648, resolve 491.
TRAFFIC = {"raster": {"bytes": 1.37e9, "digest": "94721382e11f362b"}}


def kernel_digest():
    """Digest of the sources of the rasterisation stage's kernels."""
    import hashlib
    h = hashlib.sha256()
    for f in ("raster.cu", "resolve.cu", "raster_common.cuh", "fan_geom.cuh"):
        h.update(f.encode())
        h.update(open(os.path.join(ROOT, "paper_2502_07754_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=700)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", type=int, default=3)
    p.add_argument("--gaussians", type=int, default=0, help="override the Gaussian count (profiling cases)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--input-order", action="store_true",
                   help="keep the Gaussians in the generator's order (no spatial storage order)")
    p.add_argument("--no-next-rows", action="store_true",
                   help="skip the rows beyond the hot path (full-loss fine-tune, three-fan, mesh prior, ray tracing)")
    p.add_argument("--no-other-workloads", action="store_true",
                   help="skip the compact measurements of the other configurations")
    p.add_argument("--tile", type=int, default=16, help="screen tile edge (single-view workloads; batch workloads with --no-autotune)")
    p.add_argument("--kbuf", type=int, default=8, help="per-pixel pending buffer (single-view workloads; batch workloads with --no-autotune)")
    p.add_argument("--pairs-per-scene", type=int, default=125_000, help="training pairs kept per pair scene")
    p.add_argument("--finetune-steps", type=int, default=150)
    p.add_argument("--mlp-steps", type=int, default=400)
    p.add_argument("--initializer-only", action="store_true",
                   help="time the initializer's inference alone and fused into the conversion (profiling case)")
    return p.parse_args()


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    """The slowest rank's value (every rank gets it); NCCL on GPUs, gloo on the host."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """SM clock and throttle reasons sampled during the timed region: every ~2 ms through
    NVML (read-only queries of libnvidia-ml, loaded with ctypes), else every 200 ms from
    nvidia-smi.  Nothing here changes a GPU setting."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_index, period_s=0.002):
        self.local = local_index
        self.period = period_s
        self.proc = None
        self.thread = None
        self.samples = []       # (sm_mhz, max_mhz, reasons set)
        self.source = None

    def _nvml_handle(self):
        nv = C.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            return None, None
        h = C.c_void_p()
        try:
            import torch
            uid = str(torch.cuda.get_device_properties(self.local).uuid)
            for cand in (uid, "GPU-" + uid):
                if nv.nvmlDeviceGetHandleByUUID(cand.encode(), C.byref(h)) == 0:
                    return nv, h
        except Exception:
            pass
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        idx = self.local
        if vis:
            parts = [x.strip() for x in vis.split(",")]
            if self.local < len(parts) and parts[self.local].isdigit():
                idx = int(parts[self.local])
        if nv.nvmlDeviceGetHandleByIndex_v2(C.c_uint(idx), C.byref(h)) == 0:
            return nv, h
        return None, None

    def _poll(self, nv, h):
        clk, mx, rs = C.c_uint(), C.c_uint(), C.c_ulonglong()
        getr = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        nv.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx))
        while not self.stop:
            if nv.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0 and getr(h, C.byref(rs)) == 0:
                self.samples.append((float(clk.value), float(mx.value),
                                     {n for b, n in self.REASONS.items() if rs.value & b}))
            time.sleep(self.period)

    def __enter__(self):
        self.stop = False
        try:
            nv, h = self._nvml_handle()
        except OSError:
            nv, h = None, None
        if nv is not None:
            self.source = "nvml"
            self.thread = threading.Thread(target=self._poll, args=(nv, h), daemon=True)
            self.thread.start()
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.local)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi"
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.stop = True
        if self.thread is not None:
            self.thread.join(timeout=5)
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for ln in out.splitlines():
                f = [x.strip() for x in ln.split(",")]
                if len(f) < 9:
                    continue
                try:
                    self.samples.append((float(f[1]), float(f[2]),
                                         {n for n, v in zip(names, f[5:9]) if v.lower().startswith("active")}))
                except ValueError:
                    continue

    def summary(self):
        if not self.samples:
            return None
        reasons = set()
        for _, _, r in self.samples:
            reasons |= r
        return {"sm_mhz": statistics.median(x[0] for x in self.samples), "sm_max_mhz": self.samples[-1][1],
                "reasons": sorted(reasons), "samples": len(self.samples), "source": self.source}


def mpix(W, H, ms):
    return W * H / (ms * 1e-3) / 1e6


# --------------------------------------------------------------------------- oracle arm

def oracle_frame_step(w, K):
    """One oracle pass over the full frame of the workload's first view, as the GPU step
    does it: conversion of every Gaussian, render, L1 against a blank target, reverse pass.
    Returns seconds."""
    import oracle
    cam = w.cameras[0]
    t0 = time.perf_counter()
    xyz, rgb, a = oracle.mesh_build(w.scene, K=K, cam_center=cam.C)
    xyz = xyz.astype(np.float32).astype(np.float64)
    tris = oracle.fan_tris(w.scene.n, K)
    img, _, _ = oracle.render(xyz, rgb, a, tris, cam)
    _, g = oracle.l1_loss_grad(img[..., :3], np.zeros_like(img[..., :3]))
    dL = np.zeros_like(img)
    dL[..., :3] = g
    oracle.render_backward(xyz, rgb, a, tris, cam, dL)
    return time.perf_counter() - t0


def cpu_baseline(w, K, passes=2):
    """The oracle on the host cores: `passes` full-frame steps (the first untimed)."""
    import oracle
    oracle_frame_step(w, K)
    ts = [oracle_frame_step(w, K) for _ in range(max(passes - 1, 1))]
    t = statistics.median(ts)
    cam = w.cameras[0]
    W, H = cam.width, cam.height
    return {"value": W * H / t / 1e6, "unit": "Mpix/s", "cores": oracle.threads_used(),
            "host_cores": os.cpu_count(), "affinity_cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": (f"the full {W}x{H} frame of the first view: conversion of all {w.scene.n} Gaussians "
                       f"(one thread), render, L1 and reverse pass (all cores); median of {len(ts)} timed "
                       f"passes after one untimed, {t:.2f} s each")}


def run_reference(args, ws, rank):
    import oracle
    import synthetic
    if rank != 0:
        return
    w = synthetic.workload(args.workload, n=args.gaussians or None)
    K = w.K
    cam = w.cameras[0]
    for _ in range(args.warmup):
        oracle_frame_step(w, K)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_frame_step(w, K)
    dt = (time.perf_counter() - t0) / args.steps
    W, H = cam.width, cam.height
    val = W * H / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "gaussians": w.scene.n, "K": K, "resolution": f"{W}x{H}",
                       "views_timed": 1, "parallelism": "replicas",
                       "step": "oracle conversion + full-frame render + L1 + reverse pass"},
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": oracle.threads_used(),
                             "host_cores": os.cpu_count(), "affinity_cores": len(os.sched_getaffinity(0)),
                             "kind": "oracle",
                             "sample": f"each step the full {W}x{H} frame of the first view, {dt:.2f} s"},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU arm

def stage_report(stage_ms, stage_n, info, sc, V, K, npx, local):
    """Per-stage achieved rate against its roofline, and the dominant stage's roofline
    entry.  Algorithmic work per launch: HBM bytes for the streaming stages, FP32
    lane-operations for the rasterisation / resolve (10 K per (pixel, fan) test and 40 per
    fragment forward, 420 per composited fragment backward)."""
    import torch
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    per_launch = {STAGES[i]: stage_ms[i] / max(stage_n[i], 1) for i in range(NSTAGE)}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sm * 128 * sm_max * 1e6 / 1e12           # FP32 lane-ops per second, TOP/s
    # the method's coverage work counted once (the count pass that sizes the fragment
    # buffer re-derives it, an implementation choice that is not counted)
    cov_ops = info.rect_tests * 10 * K + info.fragments * 40
    # backward: per composited fragment ~35 lane-ops of adjoint compositing and ~385 of the
    # chain to the vertices (double-float centre projection, two vertex offsets,
    # barycentrics and their adjoint); no coverage work
    comp_ops = {"raster": cov_ops, "raster_bwd": info.commits * 420}
    tc_flops = {"mlp": sc.n * MLP_FLOPS_PER_ROW}
    tc_peak = float(peaks.get("bf16_tflops", 1900.0))
    nb = (sc.sh_degree + 1) ** 2 * 3 * (2 if sc.sh_bf16 else 4)
    hbm_bytes = {"mesh_build": sc.n * (44 + nb) + V * 28,
                 "bin": V * 12 + info.pairs * 8,
                 # one histogram read, then per pass each 8-byte element read and written
                 "sort": info.pairs * (8 + 16 * ((info.sort_bits + 7) // 8)),
                 "loss": npx * 48,
                 "adam": V * 7 * 28}
    stages = {}
    for s_ in STAGES:
        t = per_launch[s_]
        if t <= 0:
            continue
        if s_ in hbm_bytes:
            ach = hbm_bytes[s_] / (t * 1e-3) / 1e9
            stages[s_] = {"ms": t, "bound": "hbm", "achieved": ach, "unit": "GB/s", "frac": ach / hbm}
        elif s_ in tc_flops:
            ach = tc_flops[s_] / (t * 1e-3) / 1e12
            stages[s_] = {"ms": t, "bound": "tensor", "achieved": ach, "unit": "TFLOP/s", "frac": ach / tc_peak}
        else:
            ach = comp_ops[s_] / (t * 1e-3) / 1e12
            stages[s_] = {"ms": t, "bound": "alu", "achieved": ach, "unit": "TOP/s", "frac": ach / alu_peak}
    dom = max(stages, key=lambda s_: stages[s_]["ms"])
    d = stages[dom]
    peak = {"hbm": hbm, "alu": alu_peak, "tensor": tc_peak}[d["bound"]]
    src = {"hbm": "measured hbm_gbs (MEASURED_PEAKS.json)", "tensor": "measured bf16_tflops (MEASURED_PEAKS.json)",
           "alu": f"{n_sm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz (max SM clock)"}[d["bound"]]
    roof = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": peak, "unit": d["unit"],
            "frac": d["frac"], "peak_source": src, "traffic": None}
    tr = TRAFFIC.get(dom)
    if tr is not None and tr["digest"] == kernel_digest() and sc.n == 1_000_000 and SPATIAL_ORDER:
        roof["traffic"] = tr["bytes"]
    return stages, roof


def prune_report(ms_, n_fans, K, kept):
    """Roofline entry of the pruning step: opacities read twice (4 (K+1) B per fan each),
    then 84 B read and 84 B written per kept vertex (position, colour, opacity and their
    two Adam moments).  The time includes the host read of the kept count."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    nbytes = n_fans * (K + 1) * 8 + kept * (K + 1) * 168
    ach = nbytes / (ms_ * 1e-3) / 1e9
    return {"ms": ms_, "bound": "hbm", "achieved": ach, "unit": "GB/s", "frac": ach / hbm, "fans": n_fans,
            "kept": kept}


def loss_report(ms_, npx):
    """Roofline entry of the full fine-tuning loss: two stencil passes over the image,
    algorithmic 152 B per pixel (image and target 32 B in each pass, nine gradient factor
    planes 36 B written and read, the gradient image 16 B written)."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ach = npx * 152 / (ms_ * 1e-3) / 1e9
    return {"ms": ms_, "bound": "hbm", "achieved": ach, "unit": "GB/s", "frac": ach / hbm,
            "bytes_per_pixel": 152, "loss": "0.6 L1 + 0.4 (1 - SSIM), 11x11 Gaussian window"}


def image_error(img, soup, K, cam, wins, tol=1e-4):
    """The GPU image against the FP64 oracle (FP64 coverage and order) on windows of the
    frame: max abs, mean abs and the count of channel values over 1e-4."""
    import oracle
    xyz, rgb, a = (np.asarray(t, np.float64) for t in soup)
    tris = oracle.fan_tris(xyz.shape[0] // (K + 1), K)
    worst, tot, over, n = 0.0, 0.0, 0, 0
    for x0, y0, x1, y1 in wins:
        ref, _, _ = oracle.render(xyz, rgb, a, tris, cam, window=(x0, y0, x1, y1))
        d = np.abs(img[y0:y1, x0:x1].astype(np.float64) - ref)
        worst = max(worst, float(d.max()))
        tot += float(d.sum())
        over += int((d > tol).sum())
        n += d.size
    return {"max_abs": worst, "mean_abs": tot / max(n, 1), "n_over_1e-4": over, "n_values": n,
            "windows": [list(map(int, w_)) for w_ in wins], "reference": "oracle, FP64 decisions"}


def error_windows(W, H, size=96, seed=7):
    """The image centre, a window right of it (the torus rim in the surface scenes) and a
    seeded random one."""
    rng = np.random.default_rng(seed)
    cx, cy = W // 2, H // 2
    x1, y1 = min(W - size, cx + W // 3), min(H - size, cy)
    wins = [(cx - size // 2, cy - size // 2, cx - size // 2 + size, cy - size // 2 + size),
            (x1, y1, x1 + size, y1 + size)]
    x0, y0 = int(rng.integers(0, W - size + 1)), int(rng.integers(0, H - size + 1))
    wins.append((x0, y0, x0 + size, y0 + size))
    return wins


# Gaussians are stored in the order ms_spatial_order gives (Morton order of the means), the
# way a scene is loaded for training: set by --input-order to keep the generator's order.
SPATIAL_ORDER = True


def stored_in_spatial_order(w):
    """The workload with its Gaussians (and the jittered target scene, by the same
    permutation) stored in the order the library's ms_spatial_order computes on the GPU;
    done once, before anything is timed.  The method does not depend on the order of its
    inputs (exact depth ties aside); the render's gathers and the adjoint's gradient sums
    do."""
    if not SPATIAL_ORDER:
        return w
    import torch
    import synthetic
    import paper_2502_07754_gb300 as ms
    p = ms.spatial_order(torch.from_numpy(np.ascontiguousarray(w.scene.means)).cuda()).cpu().numpy()
    reorder = lambda s_: synthetic.Scene(s_.means[p], s_.log_scales[p], s_.quats[p], s_.opacity[p], s_.sh[p],
                                         s_.sh_degree, s_.sh_bf16)
    w.scene = reorder(w.scene)
    if w.target_scene is not None:
        w.target_scene = reorder(w.target_scene)
    return w


def pipelined_e2e(run_step, hostG, devGs, steps, stream):
    """Milliseconds per step through the public API with each step's inputs copied from
    pinned host memory and its loss read back: the copy of step i + 1's inputs runs on a
    second stream into the other of two device input sets while step i computes (a
    double-buffered input pipeline).  One CUDA-event pair around all `steps` steps, the first
    copy inside it; no L2 flush (the 140 MB of inputs copied every step exceed L2)."""
    import torch
    cs = torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]
    loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    cs.wait_stream(stream)
    with torch.cuda.stream(cs):
        for d_, h_ in zip(devGs[0], hostG):
            d_.copy_(h_, non_blocking=True)
        copied[0].record(cs)
    for i in range(steps):
        k = i % 2
        stream.wait_event(copied[k])
        if i + 1 < steps:
            with torch.cuda.stream(cs):
                if i >= 1:
                    cs.wait_event(used[1 - k])   # step i - 1 has finished reading that set
                for d_, h_ in zip(devGs[1 - k], hostG):
                    d_.copy_(h_, non_blocking=True)
                copied[1 - k].record(cs)
        loss = run_step(k)
        loss_host.copy_(loss, non_blocking=True)
        used[k].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / steps


def timed(fn, steps, flush, stream):
    """Mean CUDA-event milliseconds of fn() over `steps` calls, L2 flushed before each."""
    import torch
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        e0[i].record(stream)
        fn()
        e1[i].record(stream)
    torch.cuda.synchronize()
    return sum(a_.elapsed_time(b_) for a_, b_ in zip(e0, e1)) / steps


def compact_single(idx, steps, warmup, flush):
    """Forward+backward fine-tune step (one captured CUDA graph) and forward-only render of a
    one-view workload (conversion, render, L1 against the same scene jittered by N(0, 1e-3),
    adjoint, Adam): Mpix/s of both and the image error of the render against the oracle."""
    import torch

    import synthetic
    import paper_2502_07754_gb300 as ms
    w = stored_in_spatial_order(synthetic.workload(idx))
    sc, K, cam = w.scene, w.K, w.cameras[0]
    tg = w.target_scene or synthetic.jittered(sc, 1e-3, 1100 + idx)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    shv = lambda s_: s_.sh.view(np.int16) if s_.sh_bf16 else s_.sh
    G = [dev(sc.means), dev(sc.log_scales), dev(sc.quats), dev(sc.opacity), dev(shv(sc))]
    tG = [dev(tg.means), dev(tg.log_scales), dev(tg.quats), dev(tg.opacity), dev(shv(tg))]
    rend = ms.Renderer(sc.n, K, cam)
    target = rend.forward(*ms.mesh_build(*tG, tg.sh_degree, K=K, cam_center=cam.C)).clone()
    xyz, rgb, a = ms.mesh_build(*G, sc.sh_degree, K=K, cam_center=cam.C)
    out = rend.forward(xyz, rgb, a).clone()
    err = image_error(out.cpu().numpy(), (xyz.cpu().numpy(), rgb.cpu().numpy(), a.cpu().numpy()), K, cam,
                      error_windows(cam.width, cam.height, size=min(96, cam.width, cam.height)))
    adam = ms.FanAdam(xyz, rgb, a, device_step=True)
    stream = torch.cuda.current_stream()

    def step():
        x, c, al = ms.mesh_build(*G, sc.sh_degree, K=K, cam_center=cam.C, out=(xyz, rgb, a))
        rend.forward(x, c, al, out=out, check_status=False)
        _, dL = ms.l1_loss(out, target)
        rend.backward(x, c, al, out, dL, into_workspace=True)
        adam.step_ws(x, c, al, rend)

    s_ = torch.cuda.Stream()
    s_.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s_):
        step()
    torch.cuda.current_stream().wait_stream(s_)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(warmup):
        graph.replay()
    ms_step = timed(graph.replay, steps, flush, stream)
    ms_fwd = timed(lambda: rend.forward(xyz, rgb, a, out=out, check_status=False), steps, flush, stream)
    st, _ = rend.info()
    from paper_2502_07754_gb300 import _lib
    _lib.check(st)
    W, H = cam.width, cam.height
    return {"workload": w.name, "gaussians": sc.n, "K": K, "resolution": f"{W}x{H}", "steps": steps,
            "warmup": warmup, "value": mpix(W, H, ms_step), "ms_per_step": ms_step, "fwd_mpix_s": mpix(W, H, ms_fwd),
            "fwd_ms": ms_fwd, "image_error": err, "target": "the scene jittered by N(0, 1e-3)", "step": "one CUDA graph"}


def compact_batch(idx, steps, warmup, flush):
    """Multi-view workloads: conversion (with the learned initializer's inference on
    workload 5), batch render of all views, L1, batch adjoint and Adam captured in one CUDA
    graph and replayed, after the autotuner picks tile and list capacities."""
    import torch

    import synthetic
    import paper_2502_07754_gb300 as ms
    w = stored_in_spatial_order(synthetic.workload(idx))
    sc, K, cams = w.scene, w.K, w.cameras
    centre = cams[0].C
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    shv = lambda s_: s_.sh.view(np.int16) if s_.sh_bf16 else s_.sh
    G = [dev(sc.means), dev(sc.log_scales), dev(sc.quats), dev(sc.opacity), dev(shv(sc))]
    tg = w.target_scene or synthetic.jittered(sc, 1e-3, 1100 + idx)
    tG = [dev(tg.means), dev(tg.log_scales), dev(tg.quats), dev(tg.opacity), G[4]]
    br = ms.BatchRenderer(sc.n, K, cams)
    target = br.forward(*ms.mesh_build(*tG, tg.sh_degree, K=K, cam_center=centre)).clone()
    del tG
    net = ms.FanMLP(K=K, seed=1) if idx == 5 else None
    xyz, rgb, a = ms.mesh_build(*G, sc.sh_degree, K=K, cam_center=centre, mlp=net)
    br.forward(xyz, rgb, a)
    br.autotune(xyz, rgb, a, reps=1, headroom=0.05)
    flat = br.new_flat()
    adam = ms.FanAdam(xyz, rgb, a, device_step=True)

    def step():
        x, c, al = ms.mesh_build(*G, sc.sh_degree, K=K, cam_center=centre, mlp=net, out=(xyz, rgb, a))
        br.forward(x, c, al, flat, check_status=False)
        _, dL = ms.l1_loss(flat, target)
        br.backward(x, c, al, flat, dL, into_workspace=True)
        adam.step_ws(x, c, al, br)

    s_ = torch.cuda.Stream()
    s_.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s_):
        step()
    torch.cuda.current_stream().wait_stream(s_)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(warmup):
        graph.replay()
    stream = torch.cuda.current_stream()
    ms_step = timed(graph.replay, steps, flush, stream)
    ms_fwd = timed(lambda: br.forward(xyz, rgb, a, flat, check_status=False), steps, flush, stream)
    st, _ = br.info()
    from paper_2502_07754_gb300 import _lib
    _lib.check(st)
    npx = br.n_pixels
    r = {"workload": w.name, "gaussians": sc.n, "K": K, "views": len(cams), "pixels": npx, "steps": steps,
         "warmup": warmup, "value": npx / (ms_step * 1e-3) / 1e6, "ms_per_step": ms_step,
         "fwd_mpix_s": npx / (ms_fwd * 1e-3) / 1e6, "fwd_ms": ms_fwd, "tile": int(br.params.tile),
         "kbuf": int(br.params.kbuf), "step": "one CUDA graph", "target": "the scene jittered by N(0, 1e-3)"}
    if net is not None:
        r["initializer"] = ("tensor-core MLP inference of every Gaussian fused into the conversion in the step, "
                            "untrained weights (the same work; bench.py --workload 5 runs the trained-network "
                            "experiment)")
    return r


def other_workloads(flush, steps=10, warmup=3):
    """Compact measurements of the other configurations, for the same JSON line."""
    import torch
    out = {}
    for idx, fn in ((1, compact_single), (2, compact_single), (4, compact_batch), (5, compact_batch)):
        t0 = time.perf_counter()
        try:
            r = fn(idx, steps, warmup, flush)
        except Exception as e:   # reported, not hidden: the headline line stays valid
            r = {"error": f"{type(e).__name__}: {e}"}
        r["wall_s"] = round(time.perf_counter() - t0, 1)
        out[str(idx)] = r
        torch.cuda.empty_cache()
    return out


def _scene_tensors(sc):
    import torch
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return [dev(sc.means), dev(sc.log_scales), dev(sc.quats), dev(sc.opacity),
            dev(sc.sh.view(np.int16) if sc.sh_bf16 else sc.sh)]


def row_full_fine_tune(flush, steps, warmup):
    """Next-row f1: the fine-tuning of Sec. 3 with the full loss of Eq. 3 (0.6 L1 +
    0.4 (1 - SSIM)) on the 1M-fan 1080p scene (FanFineTune: render, loss, adjoint, Adam),
    and one per-face pruning step (ms_prune_faces) of that soup with its moments."""
    import torch
    import synthetic
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300.finetune import FanFineTune
    w = stored_in_spatial_order(synthetic.workload(3))
    sc, K, cam = w.scene, w.K, w.cameras[0]
    G, tG = _scene_tensors(sc), _scene_tensors(w.target_scene)
    target = ms.Renderer(sc.n, K, cam).forward(*ms.mesh_build(*tG, sc.sh_degree, K=K, cam_center=cam.C)).clone()
    del tG
    xyz, rgb, a = ms.mesh_build(*G, sc.sh_degree, K=K, cam_center=cam.C)
    ft = FanFineTune(xyz, rgb, a, K, [cam], target.view(-1, 4), prune_every=0)
    for _ in range(warmup):
        ft.step()
    stream = torch.cuda.current_stream()
    t_step = timed(ft.step, steps, flush, stream)
    opt = ft.adam
    for _ in range(2):
        ms.prune_faces(ft.xyz, ft.rgb, ft.alpha, K, m=opt.m, v=opt.v)
    t_prune = timed(lambda: ms.prune_faces(ft.xyz, ft.rgb, ft.alpha, K, m=opt.m, v=opt.v), 3, flush, stream)
    kept = ms.prune_faces(ft.xyz, ft.rgb, ft.alpha, K, m=opt.m, v=opt.v)[6]
    W, H = cam.width, cam.height
    return {"workload": w.name, "step": "render+(0.6 L1 + 0.4 (1 - SSIM))+adjoint+adam (FanFineTune)",
            "value": mpix(W, H, t_step), "unit": "Mpix/s", "ms_per_step": t_step,
            "prune_faces_ms": t_prune, "fans": sc.n, "fans_kept": int(kept),
            "parity": "tests/test_gpu_finetune.py (the loop against the FP64 oracle loop)"}


def row_three_fan(flush, steps, warmup):
    """Next-row f2: the three-fan conversion of 3D Gaussians (ms_mesh_build_3d) and the
    fine-tune step of the three-fan mesh (render 3N fans, L1, adjoint, copies' gradients
    summed, Adam), on the 200k-Gaussian surface scene with the normal axis thickened to a
    third of the in-plane scale, 800x800; image error of the render against the oracle."""
    import torch
    import synthetic
    import paper_2502_07754_gb300 as ms
    w = stored_in_spatial_order(synthetic.workload(2))
    sc, K, cam = w.scene, w.K, w.cameras[0]
    ls = sc.log_scales.copy()
    ls[:, 0] = ls[:, 1] - np.log(3.0)
    sc = synthetic.Scene(sc.means, ls, sc.quats, sc.opacity, sc.sh, sc.sh_degree, sc.sh_bf16)
    tg = synthetic.jittered(sc, 1e-3, 1302)
    G, tG = _scene_tensors(sc), _scene_tensors(tg)
    N = sc.n
    rend = ms.Renderer(3 * N, K, cam)
    target = rend.forward(*ms.mesh_build_3d(*tG, tg.sh_degree, K=K, cam_center=cam.C)).clone()
    del tG
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ms.mesh_build_3d(*G, sc.sh_degree, K=K, cam_center=cam.C)
    t_conv = timed(lambda: ms.mesh_build_3d(*G, sc.sh_degree, K=K, cam_center=cam.C), steps, flush, stream)
    xyz, rgb, a = ms.mesh_build_3d(*G, sc.sh_degree, K=K, cam_center=cam.C)
    out = rend.forward(xyz, rgb, a).clone()
    err = image_error(out.cpu().numpy(), (xyz.cpu().numpy(), rgb.cpu().numpy(), a.cpu().numpy()), K, cam,
                      error_windows(cam.width, cam.height))
    adam = ms.FanAdam(xyz, rgb, a)

    def step():
        rend.forward(xyz, rgb, a, out=out, check_status=False)
        _, dL = ms.l1_loss(out, target)
        rend.backward(xyz, rgb, a, out, dL, into_workspace=True)
        ms.three_fan_sum_copies(N, K, renderer=rend)
        adam.step_ws(xyz, rgb, a, rend)

    for _ in range(warmup):
        step()
    t_step = timed(step, steps, flush, stream)
    st, _ = rend.info()
    from paper_2502_07754_gb300 import _lib
    _lib.check(st)
    nb = (sc.sh_degree + 1) ** 2 * 3 * 4
    conv_bytes = N * (44 + nb) + 3 * N * (K + 1) * 28
    W, H = cam.width, cam.height
    return {"workload": "surfaces-200k-3D-three-fan-K8-800px", "gaussians": N, "fans": 3 * N, "K": K,
            "conversion_ms": t_conv, "conversion_gbs": conv_bytes / (t_conv * 1e-3) / 1e9,
            "conversion_bytes": conv_bytes, "value": mpix(W, H, t_step), "unit": "Mpix/s", "ms_per_step": t_step,
            "step": "render+l1+adjoint+copies summed+adam", "image_error": err}


def row_mesh_prior(flush, steps, warmup):
    """Next-row f3: the mesh-prior mode on two tessellated spheres (S = 4 secondary
    triangles per face, midpoint subdivision), 1920x1080: secondary triangles built as
    centroid fans from the simplex weights, render, L1 against the same mesh with
    perturbed colours, adjoint, fold of the fan gradients to the weights and attributes;
    image error of the render against the oracle."""
    import torch
    import synthetic
    import paper_2502_07754_gb300 as ms
    V1, F1 = synthetic.sphere_mesh(160, 320, 0.8, (0.1, 0.0, 0.0), jitter=2e-4, seed=31)
    V2, F2 = synthetic.sphere_mesh(100, 200, 0.4, (-0.4, 0.3, 0.6), jitter=2e-4, seed=32)
    Vm = np.concatenate([V1, V2]).astype(np.float64)
    Fm = np.concatenate([F1, F2 + len(V1)])
    faces = Vm[Fm]                                    # F x 3 corners x 3
    S = 4
    wts = synthetic.mesh_prior_weights(faces.shape[0], S)   # midpoint subdivision of every face
    rng = np.random.Generator(np.random.PCG64(33))
    Fn = faces.shape[0]
    rgb = rng.uniform(0.1, 0.9, (Fn, S, 3, 3))
    alpha = rng.uniform(0.3, 0.9, (Fn, S, 3))
    dev = lambda a_: torch.from_numpy(np.ascontiguousarray(a_, dtype=np.float32)).cuda()
    Fd, Wd, Cd, Ad = dev(faces), dev(wts), dev(rgb), dev(alpha)
    cam = synthetic.make_camera(np.array([0.9, 0.7, 2.6]), 1920, 1080)
    rend = ms.Renderer(Fn * S, 3, cam)
    tgt = rend.forward(*ms.mesh_prior_build(Fd, Wd, dev(np.clip(rgb + rng.normal(0, 0.05, rgb.shape), 0, 1)),
                                            Ad)).clone()
    fx, fc, fa = ms.mesh_prior_build(Fd, Wd, Cd, Ad)
    out = rend.forward(fx, fc, fa).clone()
    err = image_error(out.cpu().numpy(), (fx.cpu().numpy(), fc.cpu().numpy(), fa.cpu().numpy()), 3, cam,
                      error_windows(cam.width, cam.height))
    grads = (torch.zeros_like(Wd), torch.zeros_like(Cd), torch.zeros_like(Ad))

    def step():
        x, c, a_ = ms.mesh_prior_build(Fd, Wd, Cd, Ad)
        rend.forward(x, c, a_, out=out, check_status=False)
        _, dL = ms.l1_loss(out, tgt)
        rend.backward(x, c, a_, out, dL, into_workspace=True)
        for g_ in grads:
            g_.zero_()
        ms.mesh_prior_backward(Fd, Wd, renderer=rend, out=grads)

    for _ in range(warmup):
        step()
    t_step = timed(step, steps, flush, torch.cuda.current_stream())
    st, _ = rend.info()
    from paper_2502_07754_gb300 import _lib
    _lib.check(st)
    return {"workload": "two-spheres-mesh-prior-S4-1080p", "faces": int(Fn), "secondary_triangles": int(Fn * S),
            "value": mpix(1920, 1080, t_step), "unit": "Mpix/s", "ms_per_step": t_step,
            "step": "prior build+render+l1+adjoint+fold to weights", "image_error": err}


def row_ray_tracing(flush, steps, warmup):
    """Next-row f4: ray tracing of the 200k-fan surface soup (1.6M triangles, 800x800):
    linear BVH build, primary rays alone and with a point light's shadows; the primary image
    against the FP64 oracle's rasterised composite (they differ only at pixel centres within
    rounding of an edge)."""
    import torch
    import synthetic
    import paper_2502_07754_gb300 as ms
    w = stored_in_spatial_order(synthetic.workload(2))
    sc, K, cam = w.scene, w.K, w.cameras[0]
    G = _scene_tensors(sc)
    xyz, rgb, a = ms.mesh_build(*G, sc.sh_degree, K=K, cam_center=cam.C)
    T = sc.n * K
    rt = ms.RayTracer(T, K)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        rt.build(xyz)
    t_build = timed(lambda: rt.build(xyz), steps, flush, stream)
    light = (2.5, 3.0, 3.5)
    out = torch.empty(cam.height, cam.width, 4, device="cuda")
    for _ in range(warmup):
        rt.trace(xyz, rgb, a, cam, out=out, T_eps=1e-5)
    t_prim = timed(lambda: rt.trace(xyz, rgb, a, cam, out=out, T_eps=1e-5), steps, flush, stream)
    prim = out.clone()
    t_shadow = timed(lambda: rt.trace(xyz, rgb, a, cam, light=light, ambient=0.3, out=out, T_eps=1e-5),
                     max(steps // 2, 1), flush, stream)
    st, ov = rt.status()
    from paper_2502_07754_gb300 import _lib
    _lib.check(st)
    err = image_error(prim.cpu().numpy(), (xyz.cpu().numpy(), rgb.cpu().numpy(), a.cpu().numpy()), K, cam,
                      error_windows(cam.width, cam.height, size=48))
    W, H = cam.width, cam.height
    return {"workload": w.name + "-raytraced", "triangles": T, "bvh_build_ms": t_build,
            "primary_ms": t_prim, "primary_mpix_s": mpix(W, H, t_prim), "shadow_ms": t_shadow,
            "value": mpix(W, H, t_shadow), "unit": "Mpix/s (primary + shadow rays)", "stack_overflows": ov,
            "image_error_primary_vs_raster_oracle": err}


def next_rows(flush, steps=10, warmup=3):
    """The rows built beyond the hot path (full-loss fine-tune with pruning, three-fan
    meshes, mesh prior, ray tracing), each timed on its own synthetic case."""
    import torch
    out = {}
    for name, fn in (("f1_full_loss_fine_tune", row_full_fine_tune), ("f2_three_fan", row_three_fan),
                     ("f3_mesh_prior", row_mesh_prior), ("f4_ray_tracing", row_ray_tracing)):
        t0 = time.perf_counter()
        try:
            r = fn(flush, steps, warmup)
        except Exception as e:   # reported, not hidden: the headline line stays valid
            r = {"error": f"{type(e).__name__}: {e}"}
        r["wall_s"] = round(time.perf_counter() - t0, 1)
        out[name] = r
        torch.cuda.empty_cache()
    return out


def run_ours(args, ws, rank, local):
    import torch

    import synthetic
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300 import _lib

    torch.cuda.set_device(local)
    if rank == 0:
        _lib.lib()
    barrier(ws)
    L = _lib.lib(build_if_missing=False)
    w = stored_in_spatial_order(synthetic.workload(args.workload, n=args.gaussians or None))
    sc, K, cam = w.scene, w.K, w.cameras[0]
    W, H = cam.width, cam.height
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sh_host = sc.sh.view(np.int16) if sc.sh_bf16 else sc.sh
    G = [dev(sc.means), dev(sc.log_scales), dev(sc.quats), dev(sc.opacity), dev(sh_host)]

    def convert(gs):
        return ms.mesh_build(*gs, sc.sh_degree, K=K, cam_center=cam.C)

    # target image: the jittered scene, rendered once (an input of the loss, untimed)
    tg = w.target_scene
    tG = [dev(tg.means), dev(tg.log_scales), dev(tg.quats), dev(tg.opacity), dev(sh_host)]
    rend = ms.Renderer(sc.n, K, cam, ms.render_params(tile=args.tile, kbuf=args.kbuf))
    txyz, trgb, ta = ms.mesh_build(*tG, tg.sh_degree, K=K, cam_center=cam.C)
    target = rend.forward(txyz, trgb, ta).clone()
    del txyz, trgb, ta, tG

    xyz, rgb, a = convert(G)
    rend.forward(xyz, rgb, a)           # sizes the pair capacity (host check, untimed)
    V = xyz.shape[0]
    adam = ms.FanAdam(xyz, rgb, a, device_step=True)
    out = torch.empty(H, W, 4, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(gs):
        x, c, al = ms.mesh_build(*gs, sc.sh_degree, K=K, cam_center=cam.C, out=(xyz, rgb, a))
        rend.forward(x, c, al, out=out, check_status=False)
        loss, dL = ms.l1_loss(out, target)
        rend.backward(x, c, al, out, dL, into_workspace=True)   # gradients stay in the workspace
        adam.step_ws(x, c, al, rend)
        return loss

    def capture(gs):
        # one step captured in a CUDA graph (after an eager run on a side stream)
        s_ = torch.cuda.Stream()
        s_.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s_):
            step(gs)
        torch.cuda.current_stream().wait_stream(s_)
        g_ = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_):
            loss_ = step(gs)
        return g_, loss_

    for _ in range(args.warmup):
        step(G)
    torch.cuda.synchronize()
    st, info = rend.info()
    _lib.check(st)
    launches0 = L.ms_kernel_launches()
    graph, _ = capture(G)
    launches = (L.ms_kernel_launches() - launches0) // 2   # the eager run and the capture
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()

    # ---- timed region: K full steps (graph replays), L2 flushed before each, per-step CUDA events
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev0[i].record(stream)
            graph.replay()
            ev1[i].record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    step_ms = sum(a_.elapsed_time(b_) for a_, b_ in zip(ev0, ev1)) / args.steps
    step_ms = max_over_ranks(step_ms, ws)
    st, info = rend.info()
    _lib.check(st)

    # per-stage times from eager steps with the stage profiler on (not the headline number)
    L.ms_profile_read(None, None, 0)
    L.ms_profile_enable(1)
    for _ in range(5):
        flush.zero_()
        step(G)
    torch.cuda.synchronize()
    L.ms_profile_enable(0)
    stage_ms = (C.c_double * NSTAGE)()
    stage_n = (C.c_int64 * NSTAGE)()
    _lib.check(L.ms_profile_read(stage_ms, stage_n, NSTAGE))

    # ---- forward-only throughput (render call alone)
    f0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    f1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    x, c, al = convert(G)
    for i in range(args.steps):
        flush.zero_()
        f0[i].record(stream)
        rend.forward(x, c, al, out=out, check_status=False)
        f1[i].record(stream)
    torch.cuda.synchronize()
    fwd_ms = max_over_ranks(sum(a_.elapsed_time(b_) for a_, b_ in zip(f0, f1)) / args.steps, ws)

    # ---- the full fine-tuning loss of Eq. 3 (lambda L1 + (1 - lambda)(1 - SSIM)) on the same
    # render and target, timed alone: not part of the step above, whose configuration names
    # the L1 loss
    lws = torch.empty(L.ms_fine_tune_loss_workspace_size(H, W), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        ms.fine_tune_loss(out, target, workspace=lws)
    s0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    s1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        s0[i].record(stream)
        ms.fine_tune_loss(out, target, workspace=lws)
        s1[i].record(stream)
    torch.cuda.synchronize()
    ssim_ms = max_over_ranks(sum(a_.elapsed_time(b_) for a_, b_ in zip(s0, s1)) / args.steps, ws)

    # ---- the pruning step (every 10 epochs in Sec. 3; not part of the step) on this soup
    # with its Adam moments
    px_ = None
    for _ in range(2):
        px_ = ms.prune_fans(x, c, al, K, m=adam.m, v=adam.v)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    flush.zero_()
    p0.record(stream)
    px_ = ms.prune_fans(x, c, al, K, m=adam.m, v=adam.v)
    p1.record(stream)
    torch.cuda.synchronize()
    prune_ms = max_over_ranks(p0.elapsed_time(p1), ws)
    kept = px_[5]
    del px_

    # ---- end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        hostG = [torch.from_numpy(np.ascontiguousarray(a_)).pin_memory() for a_ in
                 (sc.means, sc.log_scales, sc.quats, sc.opacity, sh_host)]
        devGs = [[torch.empty_like(h, device="cuda") for h in hostG] for _ in range(2)]
        loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
        h2d = sum(h.numel() * h.element_size() for h in hostG)
        for k in range(2):
            for d_, h_ in zip(devGs[k], hostG):
                d_.copy_(h_, non_blocking=True)
            step(devGs[k])
        torch.cuda.synchronize()
        # serial: copy, step and read-back one after the other (L2 flushed before each)
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ge = [capture(devGs[0]), capture(devGs[1])]   # one captured step per input set
        for k in (0, 1):
            ge[k][0].replay()
        torch.cuda.synchronize()
        devG = devGs[0]
        for i in range(args.steps):
            flush.zero_()
            e0[i].record(stream)
            for d_, h_ in zip(devG, hostG):
                d_.copy_(h_, non_blocking=True)
            ge[0][0].replay()
            loss_host.copy_(ge[0][1], non_blocking=True)
            e1[i].record(stream)
        torch.cuda.synchronize()
        serial_ms = max_over_ranks(sum(a_.elapsed_time(b_) for a_, b_ in zip(e0, e1)) / args.steps, ws)
        # pipelined: the next step's inputs copied while this one computes
        def run_step(k):
            ge[k][0].replay()
            return ge[k][1]

        e2e_ms = max_over_ranks(pipelined_e2e(run_step, hostG, devGs, args.steps, stream), ws)
        e2e = {"value": ws * mpix(W, H, e2e_ms), "unit": "Mpix/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": 4, "ms_per_step": e2e_ms,
               "pipeline": "step i + 1's inputs copied on a second stream during step i (two input sets)",
               "serial_ms_per_step": serial_ms, "serial_value": ws * mpix(W, H, serial_ms)}

    # image error of this run's render (the converted soup, forward-only loop above)
    # against the FP64 oracle on three 96 x 96 windows
    err = None
    if rank == 0:
        x, c, al = convert(G)
        rend.forward(x, c, al, out=out)
        torch.cuda.synchronize()
        err = image_error(out.cpu().numpy(), (x.cpu().numpy(), c.cpu().numpy(), al.cpu().numpy()), K, cam,
                          [(912, 492, 1008, 588), (1500, 560, 1596, 656)] + error_windows(W, H)[2:]
                          if (W, H) == (1920, 1080) else error_windows(W, H, size=min(96, W, H)))
    others = rows = None
    if not args.no_other_workloads and args.workload == 3 and not args.gaussians:
        del x, c, al
        torch.cuda.empty_cache()
        others = other_workloads(flush)
    if not args.no_next_rows and args.workload == 3 and not args.gaussians:
        torch.cuda.empty_cache()
        rows = next_rows(flush)

    if rank != 0:
        return
    stages, roof = stage_report(stage_ms, stage_n, info, sc, V, K, W * H, local)
    line = {"metric": METRIC, "value": ws * mpix(W, H, step_ms), "unit": "Mpix/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "gaussians": sc.n, "K": K, "resolution": f"{W}x{H}",
                       "sh": f"degree {sc.sh_degree} {'bf16' if sc.sh_bf16 else 'f32'}",
                       "step": "mesh_build+render+l1+render_backward+adam in one CUDA graph", "tile": args.tile, "kbuf": args.kbuf,
                       "l2": "flushed before every timed step (256 MB write)", "parallelism": "replicas",
                       "storage": ("Gaussians in Morton order of their means (ms_spatial_order, at load)"
                                   if SPATIAL_ORDER else "generator order")},
            "fwd_mpix_s": ws * mpix(W, H, fwd_ms), "fwd_ms": fwd_ms,
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(), "roofline": roof, "stages": stages,
            "work": {"pairs": info.pairs, "rect_tests": info.rect_tests, "fragments": info.fragments,
                     "commits": info.commits, "extra_passes": info.extra_passes, "sort_bits": info.sort_bits},
            "extra_stages": {"fine_tune_loss": loss_report(ssim_ms, W * H),
                             "prune": prune_report(prune_ms, sc.n, K, kept)},
            "image_error": err}
    if others is not None:
        line["other_workloads"] = others
    if rows is not None:
        line["next_rows"] = rows
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(w, K)
    print(json.dumps(line), flush=True)


def initializer_experiment(args, w, K, cams, centre, G):
    """Training pairs from fine-tunes of clustered-surface scenes (the fine-tune workload's
    generator, other seeds), training of the tensor-core MLP on all of them, then plain
    vs MLP-initialized conversion + the same fine-tune on the workload's scene, both judged
    by PSNR against its source-Gaussian render.  Returns (net, report, target)."""
    import torch

    import synthetic
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300 import initializer as I

    t0 = time.perf_counter()
    sets = []
    for i, n in enumerate(PAIR_SCENES):   # every scene gives the same share of the pairs
        psc = synthetic.surface_scene(n, 3000 + i, degree=3, clustered=True, bf16=True)
        sets.append(I.make_pairs(I.Gaussians.from_scene(psc), cams, K, args.finetune_steps, centre,
                                 keep_every=max(1, n // args.pairs_per_scene)))
    pairs = I.PairSet(torch.cat([p.X for p in sets]).contiguous(), torch.cat([p.T for p in sets]).contiguous())
    n_pairs = pairs.X.shape[0]
    t_pairs = time.perf_counter() - t0
    net = ms.FanMLP(K=K, seed=1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    l0, l1 = I.train(net, pairs, args.mlp_steps)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / (args.mlp_steps + 1)      # + the closing gradient pass
    Gs = I.Gaussians(G[0], G[1], G[2], G[3], G[4], w.scene.sh_degree)
    corr = torch.empty(Gs.n, 2 * (K + 1), device="cuda")
    for _ in range(3):
        net.forward(Gs.log_scales, Gs.quats, Gs.opacity, Gs.sh, Gs.sh_degree, out=corr)
    f0 = [torch.cuda.Event(enable_timing=True) for _ in range(10)]
    f1 = [torch.cuda.Event(enable_timing=True) for _ in range(10)]
    for i in range(10):
        f0[i].record()
        net.forward(Gs.log_scales, Gs.quats, Gs.opacity, Gs.sh, Gs.sh_degree, out=corr)
        f1[i].record()
    torch.cuda.synchronize()
    inf_ms = sum(a_.elapsed_time(b_) for a_, b_ in zip(f0, f1)) / 10
    # the same inference fused into the conversion (corrections stay on chip), against the
    # two launches it replaces
    fo = tuple(torch.empty(Gs.n * (K + 1), 3, device="cuda") for _ in range(2)) + \
        (torch.empty(Gs.n * (K + 1), device="cuda"),)
    conv = lambda **kw: ms.mesh_build(Gs.means, Gs.log_scales, Gs.quats, Gs.opacity, Gs.sh, Gs.sh_degree, K=K,
                                      cam_center=centre, out=fo, **kw)
    for _ in range(3):
        conv(mlp=net)
    for i in range(10):
        f0[i].record()
        conv(mlp=net)
        f1[i].record()
    torch.cuda.synchronize()
    fused_ms = sum(a_.elapsed_time(b_) for a_, b_ in zip(f0, f1)) / 10
    for i in range(10):
        f0[i].record()
        conv(corr=corr)
        f1[i].record()
    torch.cuda.synchronize()
    build_ms = sum(a_.elapsed_time(b_) for a_, b_ in zip(f0, f1)) / 10
    cmp = I.compare(Gs, cams, K, net, args.finetune_steps, centre, eval_every=10)
    target = I.source_targets(Gs, cams, centre)
    st, timeouts = net.status()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    tc_peak = float(peaks.get("bf16_tflops", 1900.0))
    inf_tf = Gs.n * MLP_FLOPS_PER_ROW / (inf_ms * 1e-3) / 1e12
    train_tf = 3 * n_pairs * MLP_FLOPS_PER_ROW / (train_ms * 1e-3) / 1e12
    report = {
        "pairs": n_pairs, "pair_scenes": PAIR_SCENES, "finetune_steps": args.finetune_steps,
        "finetune_lr_color": 5e-4,
        "pair_generation_s": round(t_pairs, 2),
        "mlp_train": {"steps": args.mlp_steps, "loss_first": l0, "loss_last": l1, "ms_per_step": train_ms,
                      "tflops": train_tf, "frac_of_measured_bf16": train_tf / tc_peak},
        "mlp_inference": {"rows": Gs.n, "ms": inf_ms, "rows_per_s": Gs.n / (inf_ms * 1e-3), "tflops": inf_tf,
                          "frac_of_measured_bf16": inf_tf / tc_peak},
        "fused_conversion": {"ms": fused_ms, "two_launch_ms": inf_ms + build_ms,
                             "tflops": Gs.n * MLP_FLOPS_PER_ROW / (fused_ms * 1e-3) / 1e12,
                             "corrections_hbm_bytes_saved": Gs.n * 2 * (K + 1) * 4 * 2},
        "psnr_db": {"plain": cmp["plain"], "mlp": cmp["mlp"]},
        "steps_to_plain_final": cmp["steps_to_plain_final"],
        "tensor_core_timeouts": timeouts,
    }
    return net, report, target


def run_batch(args, ws, rank, local):
    """The batched multi-view step: 16 cameras of mixed resolution over one fan soup.
    One step = fan conversion, batch render of all views, L1 over all views, batch
    adjoint and Adam, captured once in a CUDA graph and replayed; tile size, pending
    buffer and list capacities come from the autotuner.  `value` = pixels of all views
    per second of the forward+backward step."""
    import torch

    import synthetic
    import paper_2502_07754_gb300 as ms
    from paper_2502_07754_gb300 import _lib

    torch.cuda.set_device(local)
    if rank == 0:
        _lib.lib()
    barrier(ws)
    L = _lib.lib(build_if_missing=False)
    w = stored_in_spatial_order(synthetic.workload(args.workload, n=args.gaussians or None))
    sc, K, cams = w.scene, w.K, w.cameras
    centre = cams[0].C          # SH colours are evaluated once per step for the shared soup
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sh_host = sc.sh.view(np.int16) if sc.sh_bf16 else sc.sh
    G = [dev(sc.means), dev(sc.log_scales), dev(sc.quats), dev(sc.opacity), dev(sh_host)]
    # without the autotuner the tile and pending buffer come from the command line
    br = ms.BatchRenderer(sc.n, K, cams, ms.render_params(tile=args.tile, kbuf=args.kbuf)
                          if args.no_autotune else None)
    npx = br.n_pixels

    net, init_report = None, None
    if args.workload == 5:
        # the learned initializer: trained on pairs from fine-tunes of other scenes, judged
        # against the plain conversion on this one; its inference is part of every step
        net, init_report, target = initializer_experiment(args, w, K, cams, centre, G)
    else:
        tg = w.target_scene
        tG = [dev(tg.means), dev(tg.log_scales), dev(tg.quats), dev(tg.opacity), G[4]]
        target = br.forward(*ms.mesh_build(*tG, tg.sh_degree, K=K, cam_center=centre)).clone()
        del tG

    xyz, rgb, a = ms.mesh_build(*G, sc.sh_degree, K=K, cam_center=centre, mlp=net)
    br.forward(xyz, rgb, a)
    tune = None
    if not args.no_autotune:
        tune = br.autotune(xyz, rgb, a, reps=2, headroom=0.05)
    V = xyz.shape[0]
    flat = br.new_flat()
    adam = ms.FanAdam(xyz, rgb, a, device_step=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(gs):
        x, c, al = ms.mesh_build(*gs, sc.sh_degree, K=K, cam_center=centre, mlp=net, out=(xyz, rgb, a))
        br.forward(x, c, al, flat, check_status=False)
        loss, dL = ms.l1_loss(flat, target)
        br.backward(x, c, al, flat, dL, into_workspace=True)   # gradients stay in the workspace
        adam.step_ws(x, c, al, br)
        return loss

    # capture one step in a CUDA graph (after an eager warm-up on a side stream)
    s_ = torch.cuda.Stream()
    s_.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s_):
        step(G)
    torch.cuda.current_stream().wait_stream(s_)
    graph = torch.cuda.CUDAGraph()
    l0 = L.ms_kernel_launches()
    with torch.cuda.graph(graph):
        loss_g = step(G)
    launches = L.ms_kernel_launches() - l0
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    st, info = br.info()
    _lib.check(st)

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev0[i].record(stream)
            graph.replay()
            ev1[i].record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    step_ms = max_over_ranks(sum(a_.elapsed_time(b_) for a_, b_ in zip(ev0, ev1)) / args.steps, ws)
    st, info = br.info()
    _lib.check(st)

    # forward-only batch render (eager call)
    f0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    f1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        f0[i].record(stream)
        br.forward(xyz, rgb, a, flat, check_status=False)
        f1[i].record(stream)
    torch.cuda.synchronize()
    fwd_ms = max_over_ranks(sum(a_.elapsed_time(b_) for a_, b_ in zip(f0, f1)) / args.steps, ws)

    # per-stage times from eager steps with the stage profiler on (not the headline number)
    L.ms_profile_read(None, None, 0)
    L.ms_profile_enable(1)
    for _ in range(3):
        flush.zero_()
        step(G)
    torch.cuda.synchronize()
    L.ms_profile_enable(0)
    stage_ms = (C.c_double * NSTAGE)()
    stage_n = (C.c_int64 * NSTAGE)()
    _lib.check(L.ms_profile_read(stage_ms, stage_n, NSTAGE))

    e2e = None
    if not args.no_e2e:
        hostG = [torch.from_numpy(np.ascontiguousarray(a_)).pin_memory() for a_ in
                 (sc.means, sc.log_scales, sc.quats, sc.opacity, sh_host)]
        loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
        h2d = sum(h.numel() * h.element_size() for h in hostG)
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            e0[i].record(stream)
            for d_, h_ in zip(G, hostG):
                d_.copy_(h_, non_blocking=True)
            graph.replay()
            loss_host.copy_(loss_g, non_blocking=True)
            e1[i].record(stream)
        torch.cuda.synchronize()
        serial_ms = max_over_ranks(sum(a_.elapsed_time(b_) for a_, b_ in zip(e0, e1)) / args.steps, ws)
        # pipelined: a second input set with its own captured step, the next step's inputs
        # copied while this one computes
        G2 = [torch.empty_like(g_) for g_ in G]
        for d_, h_ in zip(G2, hostG):
            d_.copy_(h_)
        graph2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph2):
            loss_g2 = step(G2)
        graphs, losses = (graph, graph2), (loss_g, loss_g2)

        def run_step(k):
            graphs[k].replay()
            return losses[k]

        for k in (0, 1):
            run_step(k)
        e2e_ms = max_over_ranks(pipelined_e2e(run_step, hostG, (G, G2), args.steps, stream), ws)
        e2e = {"value": ws * npx / (e2e_ms * 1e-3) / 1e6, "unit": "Mpix/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": 4, "ms_per_step": e2e_ms,
               "pipeline": "step i + 1's inputs copied on a second stream during step i (two input sets)",
               "serial_ms_per_step": serial_ms, "serial_value": ws * npx / (serial_ms * 1e-3) / 1e6}
    if rank != 0:
        return
    stages, roof = stage_report(stage_ms, stage_n, info, sc, V, K, npx, local)
    res = sorted({(c.width, c.height) for c in cams})
    line = {"metric": METRIC, "value": ws * npx / (step_ms * 1e-3) / 1e6, "unit": "Mpix/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "gaussians": sc.n, "K": K, "views": len(cams), "pixels": npx,
                       "resolutions": [f"{a_}x{b_}" for a_, b_ in res],
                       "sh": f"degree {sc.sh_degree} {'bf16' if sc.sh_bf16 else 'f32'}",
                       "step": "mesh_build+batch_render+l1+batch_render_backward+adam in one CUDA graph",
                       "tile": int(br.params.tile), "kbuf": int(br.params.kbuf),
                       "l2": "flushed before every timed step (256 MB write)", "parallelism": "replicas",
                       "storage": ("Gaussians in Morton order of their means (ms_spatial_order, at load)"
                                   if SPATIAL_ORDER else "generator order")},
            "fwd_mpix_s": ws * npx / (fwd_ms * 1e-3) / 1e6, "fwd_ms": fwd_ms,
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(), "roofline": roof, "stages": stages,
            "work": {"pairs": info.pairs, "rect_tests": info.rect_tests, "fragments": info.fragments,
                     "commits": info.commits, "extra_passes": info.extra_passes, "sort_bits": info.sort_bits}}
    if init_report is not None:
        line["config"]["step"] = ("mesh_build_mlp (inference fused into the conversion)+batch_render+l1+"
                                  "batch_render_backward+adam in one CUDA graph")
        line["initializer"] = init_report
    if tune is not None:
        line["autotune"] = {"cand_ms": [round(x, 3) for x in tune.cand_ms], "best": tune.best,
                            "candidates": "tile 8<<(c//2) x kbuf 8<<(c%2); negative = skipped"}
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(w, K)
    print(json.dumps(line), flush=True)


def run_initializer_only(args):
    """The learned initializer's inference on one Gaussian set of the workload's generator:
    ms_mlp_forward (corrections to HBM), the conversion reading them, and the two fused
    (ms_mesh_build_mlp); untrained weights (the same work).  One JSON line."""
    import numpy as np
    import torch
    import synthetic
    import paper_2502_07754_gb300 as ms
    w = stored_in_spatial_order(synthetic.workload(5, n=args.gaussians or None))
    sc, K = w.scene, w.K
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    G = [dev(sc.means), dev(sc.log_scales), dev(sc.quats), dev(sc.opacity),
         dev(sc.sh.view(np.int16) if sc.sh_bf16 else sc.sh)]
    centre = w.cameras[0].C
    net = ms.FanMLP(K=K, seed=1)
    corr = torch.empty(sc.n, 2 * (K + 1), device="cuda")
    out = tuple(torch.empty(sc.n * (K + 1), 3, device="cuda") for _ in range(2)) + \
        (torch.empty(sc.n * (K + 1), device="cuda"),)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    fwd = lambda: net.forward(G[1], G[2], G[3], G[4], sc.sh_degree, out=corr)
    conv = lambda: ms.mesh_build(*G, sc.sh_degree, K=K, cam_center=centre, corr=corr, out=out)
    fused = lambda: ms.mesh_build(*G, sc.sh_degree, K=K, cam_center=centre, mlp=net, out=out)
    for _ in range(args.warmup):
        fwd(), conv(), fused()
    t_fwd = timed(fwd, args.steps, flush, stream)
    t_conv = timed(conv, args.steps, flush, stream)
    t_fused = timed(fused, args.steps, flush, stream)
    st, timeouts = net.status()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    tc_peak = float(peaks.get("bf16_tflops", 1900.0))
    tf = sc.n * MLP_FLOPS_PER_ROW / (t_fused * 1e-3) / 1e12
    line = {"metric": "initializer inference fused into the conversion", "value": sc.n / (t_fused * 1e-3) / 1e6,
            "unit": "M Gaussians/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_fused, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": w.name, "gaussians": sc.n, "K": K, "l2": "flushed before every timed call"},
            "mlp_forward_ms": t_fwd, "conversion_with_corrections_ms": t_conv, "fused_ms": t_fused,
            "roofline": {"kernel": "mlp_fwd (fused)", "bound": "tensor", "achieved": tf, "peak": tc_peak,
                         "unit": "TFLOP/s", "frac": tf / tc_peak},
            "forward_only_tflops": sc.n * MLP_FLOPS_PER_ROW / (t_fwd * 1e-3) / 1e12,
            "tensor_core_timeouts": timeouts}
    print(json.dumps(line), flush=True)


def main():
    global SPATIAL_ORDER
    args = parse()
    SPATIAL_ORDER = not args.input_order
    if args.initializer_only:
        run_initializer_only(args)
        return
    ws, rank, local = (1, 0, 0)
    if args.impl == "reference":
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, ws, rank)
        return
    ws, rank, local = dist_setup()
    if args.workload in (4, 5):
        run_batch(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
