#!/usr/bin/env python3
"""Benchmark of the MFA ray-casting hot path on one GB300 (or N independent replicas).

Workload (one step): degree-3 MFA model with 128^3 FP32 control points (64 Gaussians +
noise, clamped uniform knots), already resident on the device; one perspective 1024^2
frame with 1024 samples per ray, Phong shading and early termination at alpha 0.99; plus
one decode of 2^24 uniform random points (value + 3-component gradient).  Every sample
and every decode point is one MFA value+gradient query.

Printed metric (one JSON line on rank 0): MFA samples/s (value+grad) = (render samples
actually evaluated + decode queries) / step time, with frames/s at 1024^2 and p50/p99
frame latency beside it.  Steps are timed with CUDA events on the launching stream; a
256 MiB buffer is written between steps to flush L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the correctness reference; there is no
other implementation of this method to run) on bounded samples of the same workload.
Under torchrun (N > 1) each rank runs an independent replica of the workload on its own
GPU (the method is not sharded: no collective in the data path); value is the sum over
ranks of the work done, divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MFA samples/s (value+grad) & frames/s at 1024^2; p50/p99 frame latency vs plain FP32"
UNIT = "samples/s"
WORKLOAD = "mfa_p3_128cube_f32: persp 1024x1024, 1024 samples/ray, Phong, ERT 0.99 + decode 2^24 pts"
FP32_LANES = 128          # FP32 lanes per SM (sm_100 family)
DEFAULT_SM_MAX_MHZ = 2070.0


def device_sms(torch) -> int:
    """Streaming multiprocessors of the current device (cudaDeviceProp)."""
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sms * FP32_LANES * 2 * mhz * 1e6 / 1e12

# Algorithmic FP32 flops per value+grad query at degree p (q = p + 1):
#   contraction (sum-factorised)       2 (2q^3 + 3q^2 + 4q)
#   basis values + first derivatives   3 (2p(p+1) + 2p + 3q)   (span-local Cox-de Boor, 3 axes)
#   parameter map + chain rule         9
# A render sample adds 40 (transfer-function lerp, Phong, over).


def query_flops(p: int) -> int:
    q = p + 1
    return 2 * (2 * q ** 3 + 3 * q ** 2 + 4 * q) + 3 * (2 * p * (p + 1) + 2 * p + 3 * q) + 9


RENDER_EXTRA_FLOPS = 40
# window bytes a degree-p FP32 query gathers: q rows of its support, each row one load of
# every z-layer pair's entry (16 bytes at p = 1, 32 at p = 3, 32 + 16 at p = 4) or, at
# p = 2, one entry's layer pair and third-layer row (32 + 16 bytes)
DECODE_WINDOW_BYTES = {1: 1 * 2 * 16, 2: 1 * 3 * 48, 3: 2 * 4 * 32, 4: 3 * 5 * 48}

# DRAM bytes (read + write) of one k_render launch on this workload, measured by an ncu
# capture of the frame (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the
# kernel sources it was taken on (their SHA-256 is checked at run time; any change -> null).
RENDER_TRAFFIC = {"src_sha256": "13cd3d6a03f29cb15e04c80a34d78e612021b52189f4c082588db01198464555",
                  "bytes_per_launch": 120733696}
KERNEL_SOURCES = ["paper_2312_15073_gb300/csrc/render.cu", "paper_2312_15073_gb300/csrc/raycast.cuh",
                  "paper_2312_15073_gb300/csrc/bspline.cuh", "paper_2312_15073_gb300/csrc/mfa_internal.cuh"]


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def render_traffic():
    if RENDER_TRAFFIC["src_sha256"] and RENDER_TRAFFIC["src_sha256"] == kernel_sources_sha256():
        return RENDER_TRAFFIC["bytes_per_launch"]
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_replicas(total_s: float, units: float, dist, device: str):
    """Whole-job numbers of N independent replicas: the slowest rank's time and the sum
    of the work every rank did (the only collective; it is not in the data path)."""
    import torch
    t = torch.tensor([total_s], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def build_workload(with_points=True):
    import synth
    return synth.config2(decode_n=1 << 24, with_points=with_points)


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------

def oracle_rates(wl, budget_s: float, seed: int = 7):
    """Times the FP64 oracle on bounded samples of the workload: seeded pixels of the
    frame and seeded decode points.  Returns (render samples/s, decode queries/s, info)."""
    import oracle
    oracle.build()
    spec, job = wl.model, wl.render
    ref = oracle.Model.from_spec(spec)
    rng = np.random.default_rng(seed)
    W, H = job.width, job.height
    threads = oracle.default_threads()

    def run_pixels(npx):
        pix = rng.choice(W * H, npx, replace=False)
        t = time.perf_counter()
        _, ns = oracle.render(ref, job.camera, job.tf, W, H, job.n_samples, shading=job.shading, ka=job.ka, kd=job.kd,
                              ks=job.ks, shininess=job.shininess, ert_alpha=job.ert_alpha, pixels=pix,
                              nthreads=threads)
        return ns, time.perf_counter() - t

    # grow the pixel sample until it takes about 70 % of the budget
    npx = 256
    while True:
        ns1, t1 = run_pixels(npx)
        if t1 >= 0.35 * budget_s or npx >= W * H:
            break
        npx = int(min(W * H, npx * max(2.0, 0.7 * budget_s / max(t1, 1e-3))))
    rate0 = ns1 / t1
    n_dec = int(min(len(wl.decode_points) if wl.decode_points is not None else 1 << 20,
                    max(4096, 0.2 * budget_s * rate0)))
    pts = wl.decode_points[:n_dec] if wl.decode_points is not None else rng.random((n_dec, 3), dtype=np.float32)
    t = time.perf_counter()
    ref.decode(pts, nthreads=threads)
    td = time.perf_counter() - t
    # the same on one core, on a smaller sample (about 15 % of the budget)
    npx1 = max(64, min(W * H, int(0.1 * budget_s * rate0 / threads / max(1.0, ns1 / npx))))
    pix1 = rng.choice(W * H, npx1, replace=False)
    t = time.perf_counter()
    _, ns_1 = oracle.render(ref, job.camera, job.tf, W, H, job.n_samples, shading=job.shading, ka=job.ka, kd=job.kd,
                            ks=job.ks, shininess=job.shininess, ert_alpha=job.ert_alpha, pixels=pix1, nthreads=1)
    t_1 = time.perf_counter() - t
    pts1 = pts[:max(1024, len(pts) // threads // 4)]
    t = time.perf_counter()
    ref.decode(pts1, nthreads=1)
    td_1 = time.perf_counter() - t
    info = dict(pixels=npx, render_samples=ns1, render_s=t1, decode_points=len(pts), decode_s=td, threads=threads,
                one_core=dict(pixels=npx1, render_samples=ns_1, render_s=t_1, decode_points=len(pts1), decode_s=td_1,
                              render_rate=ns_1 / t_1, decode_rate=len(pts1) / td_1))
    return ns1 / t1, len(pts) / td, info


def oracle_checks(keep):
    """Errors of the kept GPU results against the FP64 oracle (part of the cpu_baseline leg):
    the small workload's full image; 4096 pixels of each of the 16 batched images; for the
    precision sweep, per storage type, the value and gradient errors of 2^22 decoded points
    and the image RMSE of a seeded pixel sample, each as kernel error (oracle on the same
    rounded control points) and total error (oracle on the FP64 values)."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from metrics import grad_error, image_rmse, value_error
    oracle.build()
    out = {}
    if "c1" in keep:
        wl = keep["c1"]["wl"]
        spec, job = wl.model, wl.render
        ref = oracle.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl64.astype(np.float32).astype(np.float64))
        r, _ = oracle.render(ref, job.camera, job.tf, job.width, job.height, job.n_samples, shading=job.shading,
                             ert_alpha=job.ert_alpha)
        rm = image_rmse(keep["c1"]["img"], r)
        out["c1_full_image_rmse"] = {"per_channel": rm.tolist(), "max": float(rm.max()), "gate": 1e-3}
    if "c4" in keep:
        rows = []
        for sp, job, pix, got in keep["c4"]:
            ref = oracle.Model(sp.degree, sp.nctrl, sp.knots, np.asarray(sp.ctrl, np.float64))
            r, _ = oracle.render(ref, job.camera, job.tf, job.width, job.height, job.n_samples, shading=job.shading,
                                 pixels=pix)
            rows.append(float(image_rmse(got, r).max()))
        out["c4_per_model_rmse"] = {"pixels_per_model": 4096, "max_channel_rmse": rows, "max": max(rows),
                                    "gate": 1e-3}
    if "c3" in keep:
        wl = keep["c3"]["wl"]
        spec, job = wl.model, wl.render
        pix, pts = keep["c3"]["pixels"], wl.decode_points
        exact = oracle.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl64)
        v_x, g_x = exact.decode(pts)
        r_x, _ = oracle.render(exact, job.camera, job.tf, job.width, job.height, job.n_samples, shading=True,
                               pixels=pix)
        del exact
        c3 = {"points": len(pts), "pixels": len(pix)}
        for name, rounding in (("f32", lambda P: P.astype(np.float32).astype(np.float64)),
                               ("f16", oracle.round_to_f16), ("bf16", oracle.round_to_bf16)):
            got = keep["c3"][name]
            stored = rounding(spec.ctrl64)
            ref = oracle.Model(spec.degree, spec.nctrl, spec.knots, stored)
            v_k, g_k = ref.decode(pts)
            r_k, _ = oracle.render(ref, job.camera, job.tf, job.width, job.height, job.n_samples, shading=True,
                                   pixels=pix)
            c3[name] = {"kernel": {"value": value_error(got["val"], v_k, stored), "gradient": grad_error(got["grad"], g_k),
                                   "image_rmse": float(image_rmse(got["img"], r_k).max())},
                        "total": {"value": value_error(got["val"], v_x, spec.ctrl64),
                                  "gradient": grad_error(got["grad"], g_x),
                                  "image_rmse": float(image_rmse(got["img"], r_x).max())}}
            del ref, stored
        c3["gates"] = {"value": 1e-5, "gradient": 1e-4, "image_rmse": 1e-3, "applies_to": "kernel error"}
        out["c3_precision_errors"] = c3
    return out


# ------------------------------------------------------------------------------------------
# reference arm: the oracle, as it stands
# ------------------------------------------------------------------------------------------

def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    wl = build_workload(with_points=True)
    import oracle
    oracle.build()
    spec, job = wl.model, wl.render
    ref = oracle.Model.from_spec(spec)
    threads = oracle.default_threads()
    rng = np.random.default_rng(11)
    W, H = job.width, job.height
    # per step: a bounded sample of the frame (pixels) and of the decode points, sized so
    # the whole run takes a few minutes
    total_steps = args.steps + args.warmup
    per_step_budget = min(20.0, 150.0 / max(total_steps, 1))
    _, _, cal = oracle_rates(wl, budget_s=min(8.0, per_step_budget))
    r_rate = cal["render_samples"] / cal["render_s"]
    px_per = cal["render_samples"] / cal["pixels"]
    npx = int(min(W * H, max(64, 0.85 * per_step_budget * r_rate / px_per)))
    nd = int(min(len(wl.decode_points) // 2, max(1024, 0.15 * per_step_budget * cal["decode_points"] / cal["decode_s"])))
    times, units = [], []
    for step in range(total_steps):
        pix = rng.choice(W * H, npx, replace=False)
        off = (step * nd) % (len(wl.decode_points) - nd)
        pts = wl.decode_points[off: off + nd]
        t = time.perf_counter()
        _, ns = oracle.render(ref, job.camera, job.tf, W, H, job.n_samples, shading=job.shading, ka=job.ka,
                              kd=job.kd, ks=job.ks, shininess=job.shininess, ert_alpha=job.ert_alpha, pixels=pix,
                              nthreads=threads)
        ref.decode(pts, nthreads=threads)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append(dt)
            units.append(ns + nd)
    value = sum(units) / sum(times)
    sample = (f"{npx} seeded pixels of the 1024^2 frame + {nd} decode points per step, "
              f"FP64 oracle on {threads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "oracle_sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

# the rows after the timed step, in the order they run
SIDE_ROWS = ["c1", "precision", "segments", "isosurface", "marschner_lobb", "encoding", "render_quality",
             "query_sweep", "c3_precision", "batch", "empty_space"]


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_2312_15073_gb300 as mfa
    from paper_2312_15073_gb300 import build as mfa_build
    if not os.path.exists(mfa.LIB_PATH):
        mfa_build.build()

    wl = build_workload(with_points=True)
    spec, job = wl.model, wl.render
    p = spec.degree[0]
    # the FP32 window plus each knot-span cell's polynomial (render variant 8, the autotuner's
    # candidate beside the others); decode and the side rows on this model use the window
    model = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl, window=mfa.MFA_WINDOW_PATCH)
    tf = mfa.transfer_fn(job.tf, shading=job.shading, ka=job.ka, kd=job.kd, ks=job.ks, shininess=job.shininess,
                         ert_alpha=job.ert_alpha)
    W, H, NS = job.width, job.height, job.n_samples
    n_pts = wl.decode_points.shape[0]
    stream = torch.cuda.current_stream()

    # device-resident inputs / outputs
    pts_d = torch.from_numpy(wl.decode_points).cuda()
    val_d = torch.empty(n_pts, device="cuda")
    grad_d = torch.empty((n_pts, 3), device="cuda")
    img_d = torch.empty((H, W, 4), device="cuda")
    cnt_d = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # measured denominators beside the derived FP32 peak (calibration kernels, untimed)
    peaks = mfa.measure_peaks()

    # the autotuner picks the kernel variant and ray-tile shape for this workload class
    # (outside the timed region); the timed renders then use its choice, unless the command
    # line fixes one
    if args.variant is None and args.tile_shape is None:
        tuned, _ = mfa.tune_render(model, job.camera, tf, W, H, NS, reps=3)
        kernel = dict(use_tuned=True)
    else:
        kernel = dict(variant=args.variant or 0, tile_shape=args.tile_shape or 0)
        tuned = dict(kernel, source="command line")

    def step(record=None):
        if record is not None:
            record[0].record(stream)
        mfa.render(model, job.camera, tf, W, H, NS, out=img_d, samples_out=cnt_d, **kernel)
        if record is not None:
            record[1].record(stream)
        mfa.decode(model, pts_d, val_d, grad_d)
        if record is not None:
            record[2].record(stream)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    cnt_d.zero_()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            step(evs[k])
            flush.zero_()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    render_ms = [e[0].elapsed_time(e[1]) for e in evs]
    decode_ms = [e[1].elapsed_time(e[2]) for e in evs]
    step_ms = [r + d for r, d in zip(render_ms, decode_ms)]
    samples = int(cnt_d.item())                      # evaluated render samples over the K steps
    units = samples + args.steps * n_pts
    total_s = sum(step_ms) / 1e3
    if dist:
        total_s, units = aggregate_replicas(total_s, units, dist, "cuda")
    value = units / total_s

    # end to end through the C ABI's host-buffer calls (page-locked host memory, the library
    # stages the copies): the render and the decode of a step are enqueued on two streams
    # and overlap; copies in and out are inside the timed region
    pts_h = torch.from_numpy(wl.decode_points).pin_memory()
    img_h = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
    val_h = torch.empty(n_pts, dtype=torch.float32).pin_memory()
    grad_h = torch.empty((n_pts, 3), dtype=torch.float32).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    e2e_ms = []
    cnt_e = torch.zeros(1, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    for k in range(e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        side.wait_event(a)
        mfa.render_host(model, job.camera, tf, W, H, NS, out=img_h, samples_out=cnt_e, sync=False, **kernel)
        with torch.cuda.stream(side):
            mfa.decode_host(model, pts_h, val_h, grad_h, sync=False)
        joined = torch.cuda.Event()
        joined.record(side)
        stream.wait_event(joined)
        b.record(stream)
        b.synchronize()
        if k > 0:                                          # first pass warms the copy engines
            e2e_ms.append(a.elapsed_time(b))
    e2e_samples = int(cnt_e.item()) * e2e_steps / (e2e_steps + 1)
    e2e_value = (e2e_samples + e2e_steps * n_pts) / (sum(e2e_ms) / 1e3)
    h2d = pts_h.numel() * 4
    d2h = (img_h.numel() + val_h.numel() + grad_h.numel()) * 4

    if rank != 0:
        return 0

    render_s = statistics.mean(render_ms) / 1e3
    samples_per_frame = samples / args.steps
    flops_sample = query_flops(p) + RENDER_EXTRA_FLOPS
    achieved_tflops = samples_per_frame * flops_sample / render_s / 1e12
    clk = clocks.summary()
    sms = device_sms(torch)
    sm_max_mhz = clk["sm_max_mhz"] or _peaks().get("sm_max_mhz") or DEFAULT_SM_MAX_MHZ
    peak_tflops = fp32_peak_tflops(sms, sm_max_mhz)
    sorted_ms = sorted(render_ms)

    def pct(q):
        return sorted_ms[min(len(sorted_ms) - 1, int(math.ceil(q * len(sorted_ms))) - 1)]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "model": "degree 3, 128^3 FP32 control points, 64 Gaussians + noise",
                   "layout": "FP32 layer-pair window + per-cell polynomial patches (MFA_WINDOW_PATCH, "
                             f"{model.info()['device_bytes'] / 1e6:.0f} MB on the device)",
                   "image": f"{W}x{H}", "n_samples": NS, "decode_points": n_pts,
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": f"replicas x{ws}"},
        "frames_per_s": 1.0 / render_s,
        "frame_latency_ms": {"p50": pct(0.5), "p99": pct(0.99), "mean": statistics.mean(render_ms)},
        "render_samples_per_frame": samples_per_frame,
        "nominal_samples_per_frame": W * H * NS,
        "render_samples_per_s": samples_per_frame / render_s,
        "decode_queries_per_s": n_pts / (statistics.mean(decode_ms) / 1e3),
        "roofline": {"bound": "alu", "kernel": "k_render", "achieved": achieved_tflops, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved_tflops / peak_tflops, "traffic": render_traffic(),
                     "traffic_note": "DRAM bytes per launch from ncu (variant 8: the patches of the cells the "
                                     "rays reach, 110 MB read, the rest of the 478 MiB patch array untouched or "
                                     "from L2; the 16 MiB image written)",
                     "tuned": tuned,
                     "flops_per_sample": flops_sample,
                     "flops_note": "algorithmic count (sum-factorised contraction + span-local Cox-de Boor "
                                   "basis and derivative + chain rule, + TF/Phong/over); on uniform knots the "
                                   "cardinal path executes 42 instead of 126 basis flops per sample, and variant 8 "
                                   "(per-cell polynomial patches) evaluates monomials instead of any basis",
                     "peak_basis": f"{sms} SMs (cudaDeviceProp) x {FP32_LANES} FP32 lanes x 2 flop x "
                                   f"{sm_max_mhz:.0f} MHz (max SM clock, nvidia-smi)",
                     "peak_at_median_clock": fp32_peak_tflops(sms, clk["sm_mhz"])
                     if clk["sm_mhz"] else None,
                     "measured_fma": {"tflops": peaks["fp32_tflops"], "fp32x2_tflops": peaks["fp32x2_tflops"],
                                      "clock_mhz": peaks["fma_clock_mhz"],
                                      "frac": achieved_tflops / peaks["fp32_tflops"],
                                      "note": "chip-wide FFMA / packed FFMA2 calibration kernels in this run"}},
        "decode_l2": {"bytes_per_query": DECODE_WINDOW_BYTES[spec.degree[0]],
                      "achieved_gbs": DECODE_WINDOW_BYTES[spec.degree[0]] * n_pts / (statistics.mean(decode_ms) / 1e3) / 1e9,
                      "l2_gather_peak_gbs": peaks["l2_gather_gbs"],
                      "frac": DECODE_WINDOW_BYTES[spec.degree[0]] * n_pts / (statistics.mean(decode_ms) / 1e3) / 1e9
                      / peaks["l2_gather_gbs"],
                      "note": "decode reads its support as random 32-byte window entries (8 at degree 3, FP32); "
                              "peak = random 32-byte gathers from an L2-resident buffer",
                      "fp32_frac": query_flops(spec.degree[0]) * n_pts / (statistics.mean(decode_ms) / 1e3) / 1e12
                      / peak_tflops,
                      "fp32_note": "the same decode against the FP32 peak (algorithmic flops per value+gradient query)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": statistics.mean(e2e_ms),
                "path": "mfa_render_host + mfa_decode_host (page-locked host buffers, library-staged "
                        "copies), enqueued on two streams so that they overlap"},
        # per step: the render (plus its visibility pass under variant 7) and the decode
        "gpu_launches": (3 if tuned.get("variant") == 7 else 2) * args.steps,
        "clocks": clk,
    }
    keep = {}   # GPU results the oracle checks in the cpu_baseline leg
    side = {
        "c1": lambda: c1_small(mfa, torch, keep),
        "precision": lambda: storage_throughput(mfa, torch, spec, job, tf),
        "segments": lambda: segments_throughput(mfa, torch, model, job, tf, render_s),
        "isosurface": lambda: iso_throughput(mfa, torch, spec, model, job, tf),
        "marschner_lobb": lambda: ml_throughput(mfa, torch, tf, peak_tflops),
        "encoding": lambda: encode_throughput(mfa, torch),
        "render_quality": lambda: render_quality(mfa, torch),
        "query_sweep": lambda: query_sweep(mfa, torch),
        "c3_precision": lambda: c3_precision(mfa, torch, keep),
        "batch": lambda: batch_throughput(mfa, torch, keep),
        "empty_space": lambda: empty_space(mfa, torch, spec, model, job),
    }
    if ws == 1 and not args.no_side_rows:
        for name in args.side_rows or SIDE_ROWS:
            line[name] = side[name]()
    if ws == 1 and not args.no_serve:
        line["serving"] = dict(run_serve(mfa, rates=args.serve_rates, duration=args.serve_duration,
                                         min_requests=args.serve_requests),
                               note="Poisson requests (sides 512..2048, 512..2048 samples) on 8 resident degree-3 "
                                    "models; served = FP16 control points (FP32 window and per-cell patches built "
                                    "from them), up to 16 requests in flight drawn tile by tile from the device "
                                    "work queue; plain_f32 = FP32 control points (default window), one request "
                                    "at a time in arrival order, one launch each; plain_f16 = the served models "
                                    "run as plain_f32 (the queue's own share of the difference); latency from "
                                    "scheduled arrival to completion")
    if ws == 1 and not args.no_cpu_baseline:
        r_rate, d_rate, info = oracle_rates(wl, budget_s=args.cpu_budget)
        cpu_step_s = samples_per_frame / r_rate + n_pts / d_rate
        o1 = info["one_core"]
        one_step_s = samples_per_frame / o1["render_rate"] + n_pts / o1["decode_rate"]
        line["cpu_baseline"] = {
            "value": (samples_per_frame + n_pts) / cpu_step_s, "unit": UNIT, "cores": info["threads"],
            "kind": "oracle",
            "sample": (f"FP64 oracle: {info['pixels']} seeded pixels of the frame ({info['render_samples']} samples, "
                       f"{info['render_s']:.1f} s) + {info['decode_points']} decode points ({info['decode_s']:.1f} s); "
                       "step time extrapolated from the two rates"),
            "one_core": {"value": (samples_per_frame + n_pts) / one_step_s, "unit": UNIT, "cores": 1,
                         "sample": (f"{o1['pixels']} seeded pixels ({o1['render_samples']} samples, "
                                    f"{o1['render_s']:.1f} s) + {o1['decode_points']} decode points "
                                    f"({o1['decode_s']:.1f} s) on one thread")},
        }
        if keep:
            line["oracle_checks"] = oracle_checks(keep)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def segments_throughput(mfa, torch, model, job, tf, single_s, frames=5):
    """The same frame with the object-space decomposition (blocks render their ray segments
    into partial images, merged with over): time per frame and samples evaluated, beside
    the single-pass render."""
    out = {"single_pass_ms": 1e3 * single_s}
    W, H, NS = job.width, job.height, job.n_samples
    img = torch.empty((H, W, 4), device="cuda")
    for g in ((2, 2, 2), (4, 4, 4)):
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        mfa.render_segments(model, job.camera, tf, W, H, NS, g, out=img)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(frames):
            mfa.render_segments(model, job.camera, tf, W, H, NS, g, out=img, samples_out=cnt)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / frames
        out["x".join(str(x) for x in g)] = {"ms_per_frame": ms, "samples_per_frame": int(cnt.item()) / frames,
                                            "samples_per_s": int(cnt.item()) / frames / (ms / 1e3)}
    return out


def ml_throughput(mfa, torch, tf, peak_tflops, frames=5):
    """The paper's scalability workload shape on the Marschner-Lobb signal: degree 2, 256^3
    control points (Greville-sampled), 768^2, 1024 samples per ray, Phong."""
    import synth
    spec = synth.marschner_lobb_model(256, 2)
    model = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.4, 0.6, 0.35, 32.0)
    W = H = 768
    NS = 1024
    ml_tf = mfa.transfer_fn(synth.ramp_tf(256, 0.06), shading=True)
    img = torch.empty((H, W, 4), device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    tuned, _ = mfa.tune_render(model, cam, ml_tf, W, H, NS, reps=3)
    mfa.render(model, cam, ml_tf, W, H, NS, out=img, use_tuned=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(frames):
        mfa.render(model, cam, ml_tf, W, H, NS, out=img, samples_out=cnt, use_tuned=True)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / frames
    samples = int(cnt.item()) / frames
    flops = samples * (query_flops(2) + RENDER_EXTRA_FLOPS)
    model.close()
    return {"model": "Marschner-Lobb, degree 2, 256^3 control points", "image": "768x768", "n_samples": NS,
            "tuned": tuned, "ms_per_frame": ms, "samples_per_frame": samples, "samples_per_s": samples / (ms / 1e3),
            "frac_fp32_peak": flops / (ms / 1e3) / 1e12 / peak_tflops}


def encode_throughput(mfa, torch):
    """MFA encoding of the Marschner-Lobb signal sampled on a 256^3 grid: one least-squares
    fit to 128^3 degree-2 control points, and the adaptive encoding to 1 % of the signal's
    range (time, control points, fits)."""
    import synth
    m = 256
    u = np.arange(m, dtype=np.float64) / (m - 1)
    data = torch.from_numpy(synth.MarschnerLobb().grid(u, u, u).astype(np.float32)).cuda()
    out = {"data": "Marschner-Lobb at 256^3 grid points"}
    mfa.fit_ctrl((2, 2, 2), (128, 128, 128), None, data)          # warm-up (pool, kernels)
    torch.cuda.synchronize()
    t = time.perf_counter()
    mfa.fit_ctrl((2, 2, 2), (128, 128, 128), None, data)
    torch.cuda.synchronize()
    out["fit_128cube_deg2_ms"] = 1e3 * (time.perf_counter() - t)
    t = time.perf_counter()
    model, res = mfa.model_encode((2, 2, 2), data, 0.01, max_ctrl=(256, 256, 256))
    torch.cuda.synchronize()
    out["adaptive"] = dict(res, err_max=0.01, seconds=time.perf_counter() - t,
                           compression=m ** 3 / float(np.prod(res["nctrl"])))
    model.close()
    return out


def render_quality(mfa, torch):
    """The render-quality comparison (Table II): the Marschner-Lobb signal sampled on a
    1024^3 grid, fitted by least squares to a degree-2 MFA of 256^3 control points (1/64 of
    the data), rendered at 768^2 with 1024 samples per ray, and scored (MSE, PSNR, SSIM on
    the 0..255 scale) against the direct render of the closed-form signal; the Greville-
    sampled 256^3 model of the throughput row is scored too."""
    import synth
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.4, 0.6, 0.35, 32.0)
    W = H = 768
    NS = 1024
    tf = mfa.transfer_fn(synth.ramp_tf(256, 0.06), shading=True, vmin=0.0, vmax=1.0)
    data = synth.MarschnerLobb().grid_device(1024)
    torch.cuda.synchronize()
    t = time.perf_counter()
    model, fit_err = mfa.model_fit((2, 2, 2), (256, 256, 256), None, data)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t
    del data
    truth = mfa.render_ml(cam, tf, W, H, NS)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    mfa.render_ml(cam, tf, W, H, NS, out=truth)
    b.record()
    b.synchronize()
    truth_ms = a.elapsed_time(b)
    fitted = mfa.image_compare(mfa.render(model, cam, tf, W, H, NS), truth)
    model.close()
    spec = synth.marschner_lobb_model(256, 2)
    greville = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
    sampled = mfa.image_compare(mfa.render(greville, cam, tf, W, H, NS), truth)
    greville.close()
    return {"data": "Marschner-Lobb (f_M = 6, alpha = 0.25) at 1024^3 grid points",
            "fit": {"degree": 2, "nctrl": 256, "seconds": fit_s, "max_err": fit_err},
            "image": f"{W}x{H}", "n_samples": NS, "ground_truth_ms": truth_ms,
            "fitted_vs_truth": fitted, "greville_vs_truth": sampled,
            "paper_table2_mfa": {"mse": 50.76, "psnr_db": 31.08, "ssim": 0.96,
                                 "note": "the paper's camera and transfer function are not given: context only"}}


def empty_space(mfa, torch, spec, model, job, frames=5):
    """Empty-space skipping (variant 7) against variant 6 on the same model and view with a
    transfer function transparent below the median control point: ms per frame and samples
    evaluated (the images agree to FP32 rounding)."""
    import synth
    W, H, NS = job.width, job.height, job.n_samples
    lo, hi = float(spec.ctrl.min()), float(spec.ctrl.max())
    cut = (float(np.median(spec.ctrl)) - lo) / (hi - lo)
    table = synth.ramp_tf(256, 0.05).copy()
    table[np.linspace(0.0, 1.0, len(table)) < cut, 3] = 0.0
    tf = mfa.transfer_fn(table, shading=True)
    img = torch.empty((H, W, 4), device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = {"transfer_function": "ramp, alpha 0 below the median control point"}
    for variant in (6, 7):
        mfa.render(model, job.camera, tf, W, H, NS, out=img, variant=variant)
        torch.cuda.synchronize()
        cnt.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(frames):
            mfa.render(model, job.camera, tf, W, H, NS, out=img, variant=variant, samples_out=cnt)
        b.record()
        b.synchronize()
        out[f"variant{variant}"] = {"ms_per_frame": a.elapsed_time(b) / frames,
                                    "samples_per_frame": int(cnt.item()) / frames}
    return out


def batch_throughput(mfa, torch, keep, reps=3):
    """The batched workload: 16 models (degrees 2, 3, 4; uniform and non-uniform knots;
    32..256 control points per axis), one image each (256^2..1024^2, 256..1024 samples):
    one CUDA-graph launch of the persistent batch kernels (tile shape from the batch
    autotuner) against the 16 images rendered one launch after another."""
    import synth
    pairs = synth.config4()
    models = [mfa.Model(sp.degree, sp.nctrl, sp.knots, sp.ctrl) for sp, _ in pairs]
    tfs = [mfa.transfer_fn(job.tf, shading=True) for _, job in pairs]
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    reqs = [mfa.Request(m, job.camera, tf, job.width, job.height, job.n_samples, samples_out=cnt)
            for m, tf, (_, job) in zip(models, tfs, pairs)]
    batch = mfa.Batch(len(reqs))
    tuned = mfa.tune_batch(batch, reqs)
    batch.configure(tile_shape=tuned["tile_shape"])

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        cnt.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps, int(cnt.item()) / reps

    ms_batch, samples = timed(lambda: batch.render(reqs))
    torch.cuda.synchronize()
    rng = np.random.default_rng(4004)
    keep["c4"] = []
    for (sp, job), q in zip(pairs, reqs):   # 4096 seeded pixels of each batched image
        pix = rng.choice(job.width * job.height, min(4096, job.width * job.height), replace=False)
        keep["c4"].append((sp, job, pix, q.out.cpu().numpy().reshape(-1, 4)[pix].astype(np.float64)))
    ms_single, _ = timed(lambda: [mfa.render(q.model, q.cam, q.tf, q.width, q.height, q.n_samples, out=q.out,
                                             samples_out=cnt) for q in reqs])
    batch.close()
    for m in models:
        m.close()
    return {"requests": len(reqs), "tile_shape": tuned["tile_shape"], "ms_per_batch": ms_batch,
            "samples_per_batch": samples, "samples_per_s": samples / (ms_batch / 1e3),
            "ms_separate_launches": ms_single}


def c3_precision(mfa, torch, keep, frames=3):
    """The precision-sweep workload: degree 3, 512x512x256 control points on non-uniform
    knots (turbulence), perspective 2048^2, 2048 samples per ray, Phong; one frame time and
    sample rate per storage type (FP32, FP16, BF16 from the same FP64 values), default
    kernel (variant 4: the record path).  The decode of 2^22 points and a seeded pixel sample
    of each frame are kept in `keep` for the oracle's error check."""
    import synth
    wl = synth.config3(dtype_in=np.float64)
    spec, job = wl.model, wl.render
    W, H, NS = job.width, job.height, job.n_samples
    tf = mfa.transfer_fn(job.tf, shading=True)
    img = torch.empty((H, W, 4), device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    pts = torch.from_numpy(wl.decode_points).cuda()
    rng = np.random.default_rng(3003)
    pix = np.concatenate([rng.choice(W * H, 16384, replace=False)] +
                         [r * W + np.arange(W) for r in rng.choice(H, 4, replace=False)])
    keep["c3"] = {"wl": wl, "pixels": pix}
    out = {"model": "degree 3, 512x512x256, non-uniform knots, turbulence", "image": f"{W}x{H}", "n_samples": NS}
    for storage, name in ((mfa.MFA_F32, "f32"), (mfa.MFA_F16, "f16"), (mfa.MFA_BF16, "bf16")):
        m = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl, storage=storage)
        mfa.render(m, job.camera, tf, W, H, NS, out=img)
        torch.cuda.synchronize()
        cnt.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(frames):
            mfa.render(m, job.camera, tf, W, H, NS, out=img, samples_out=cnt)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / frames
        samples = int(cnt.item()) / frames
        out[name] = {"ms_per_frame": ms, "samples_per_s": samples / (ms / 1e3),
                     "model_bytes": m.info()["device_bytes"]}
        v, g = mfa.decode(m, pts)
        keep["c3"][name] = {"val": v.cpu().numpy(), "grad": g.cpu().numpy(),
                            "img": img.cpu().numpy().reshape(-1, 4)[pix].astype(np.float64)}
        m.close()
    return out


def c1_small(mfa, torch, keep, frames=20):
    """The small workload: degree 3, 32^3 FP64 control points (stored FP32), orthographic
    256^2, 128 samples per ray, no shading; frames/s and samples/s, the image kept in `keep`
    for the oracle's full-image check."""
    import synth
    wl = synth.config1()
    spec, job = wl.model, wl.render
    m = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl)
    tf = mfa.transfer_fn(job.tf, shading=job.shading, ert_alpha=job.ert_alpha)
    img = torch.empty((job.height, job.width, 4), device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    mfa.render(m, job.camera, tf, job.width, job.height, job.n_samples, out=img)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(frames):
        mfa.render(m, job.camera, tf, job.width, job.height, job.n_samples, out=img, samples_out=cnt)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / frames
    samples = int(cnt.item()) / frames
    keep["c1"] = {"wl": wl, "img": img.cpu().numpy().astype(np.float64)}
    m.close()
    return {"model": "degree 3, 32^3 control points (FP64 input, FP32 storage), 8 Gaussians + noise",
            "image": f"{job.width}x{job.height} orthographic", "n_samples": job.n_samples, "ms_per_frame": ms,
            "frames_per_s": 1e3 / ms, "samples_per_frame": samples, "samples_per_s": samples / (ms / 1e3)}


def query_sweep(mfa, torch, n_pts=1 << 22, reps=5):
    """Value+gradient query rate against the control-point count and the degree (the
    paper's query-time study, Fig. 8, in spirit): 2^22 uniform random points per model,
    uniform knots, random control points (the rate does not depend on the values); the
    layer-pair window layout and the compact one (the control points once)."""
    rng = np.random.default_rng(20231215)
    pts = torch.rand((n_pts, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(8))
    val = torch.empty(n_pts, device="cuda")
    grad = torch.empty((n_pts, 3), device="cuda")
    rows = []
    for degree, n, storage, window in ((3, 32, 1, 0), (3, 64, 1, 0), (3, 128, 1, 0), (3, 256, 1, 0), (3, 512, 1, 0),
                                       (1, 128, 1, 0), (2, 128, 1, 0), (4, 128, 1, 0), (3, 128, 1, 2), (3, 256, 1, 2),
                                       (3, 512, 1, 2), (3, 256, 2, 0), (3, 256, 2, 2), (3, 256, 3, 2),
                                       (3, 512, 2, 2)):
        m = mfa.Model((degree,) * 3, (n,) * 3, None, rng.standard_normal((n, n, n), dtype=np.float32), storage=storage,
                      window=window)
        for _ in range(3):
            mfa.decode(m, pts, val, grad)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            mfa.decode(m, pts, val, grad)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        rows.append({"degree": degree, "nctrl": n, "storage": {1: "f32", 2: "f16", 3: "bf16"}[storage],
                     "layout": {0: "window", 2: "compact"}[window], "model_bytes": m.info()["device_bytes"],
                     "ms": ms, "queries_per_s": n_pts / (ms / 1e3)})
        m.close()
    return {"points": n_pts, "rows": rows}


def iso_throughput(mfa, torch, spec, model, job, tf, frames=5):
    """Isosurface frames of the same model and view (iso = the median control point):
    time per frame, samples per frame (samples examined -- with or without a query, as
    the cell bounds decide -- plus refinement queries), pixels hit."""
    W, H, NS = job.width, job.height, job.n_samples
    iso = float(np.median(spec.ctrl))
    img = torch.empty((H, W, 4), device="cuda")
    depth = torch.empty((H, W), device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    mfa.render_iso(model, job.camera, tf, W, H, NS, iso, out=img, depth=depth)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(frames):
        mfa.render_iso(model, job.camera, tf, W, H, NS, iso, out=img, depth=depth, samples_out=cnt)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / frames
    q = int(cnt.item()) / frames
    return {"iso": iso, "ms_per_frame": ms, "samples_per_frame": q, "samples_per_s": q / (ms / 1e3),
            "pixels_hit": int(torch.isfinite(depth).sum().item())}


def storage_throughput(mfa, torch, spec, job, tf, frames=5):
    """Samples/s of the same frame with FP32, FP16 and BF16 control points (the same
    FP64-rounded values, FP32 accumulation); 16-bit models with their own 16-bit window
    values and with FP32 window values (MFA_WINDOW_F32); the FP32 model with per-cell
    patches (MFA_WINDOW_PATCH, rendered by variant 8).  Default kernel of each model."""
    out = {}
    W, H, NS = job.width, job.height, job.n_samples
    img = torch.empty((H, W, 4), device="cuda")
    for storage, window, name in ((mfa.MFA_F32, 0, "f32"), (mfa.MFA_F16, 0, "f16"), (mfa.MFA_BF16, 0, "bf16"),
                                  (mfa.MFA_F16, mfa.MFA_WINDOW_F32, "f16_f32window"),
                                  (mfa.MFA_BF16, mfa.MFA_WINDOW_F32, "bf16_f32window"),
                                  (mfa.MFA_F32, mfa.MFA_WINDOW_PATCH, "f32_patches")):
        m = mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl, storage=storage, window=window)
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        mfa.render(m, job.camera, tf, W, H, NS, out=img)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(frames):
            mfa.render(m, job.camera, tf, W, H, NS, out=img, samples_out=cnt)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / frames
        out[name] = {"ms_per_frame": ms, "samples_per_s": int(cnt.item()) / frames / (ms / 1e3),
                     "model_bytes": m.info()["device_bytes"]}
        m.close()
    return out


# ------------------------------------------------------------------------------------------
# serving: Poisson camera-view requests, served FP16 path vs plain single-request FP32 path
# ------------------------------------------------------------------------------------------

def serve_models(mfa, size_scale=1.0):
    """The 8 serving models twice: FP16 control points with an FP32 window and per-cell
    patches built from them (served path) and FP32 with the default window (plain path)."""
    import synth
    specs = synth.config5_models(size_scale)
    f16 = [mfa.Model(s.degree, s.nctrl, s.knots, s.ctrl64, storage=mfa.MFA_F16, window=mfa.MFA_WINDOW_PATCH)
           for s in specs]
    f32 = [mfa.Model(s.degree, s.nctrl, s.knots, s.ctrl64, storage=mfa.MFA_F32) for s in specs]
    return specs, f16, f32


def serve_model_table(mfa, specs, f16, f32, tf, side=2048, ns=2048, frames=3):
    """Per serving model: control points, device bytes and the time of one 2048^2 frame
    with 2048 samples per ray (the largest serving view) for each way of holding it: FP32
    (the plain path's models), FP16 with per-cell patches (the served path's models), FP16
    with FP32 window values, FP16 with 16-bit window values, and the compact FP16 layout."""
    import torch
    import synth
    cam = synth.orbit_camera((0.5, 0.5, 0.5), 2.5, 0.7, 0.2, 30.0)
    img = torch.empty((side, side, 4), device="cuda")
    rows = []
    for spec, m16p, m32 in zip(specs, f16, f32):
        row = {"nctrl": list(spec.nctrl), "plain_values_bytes_f16": 2 * int(np.prod(spec.nctrl))}
        extra = [(name, mfa.Model(spec.degree, spec.nctrl, spec.knots, spec.ctrl64, storage=mfa.MFA_F16, window=w))
                 for name, w in (("f16_f32window", mfa.MFA_WINDOW_F32), ("f16", mfa.MFA_WINDOW_AUTO),
                                 ("f16_compact", mfa.MFA_WINDOW_COMPACT))]
        for name, m in [("f32", m32), ("f16_patches", m16p)] + extra:
            mfa.render(m, cam, tf, side, side, ns, out=img)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(frames):
                mfa.render(m, cam, tf, side, side, ns, out=img)
            b.record()
            b.synchronize()
            row[name] = {"device_bytes": m.info()["device_bytes"], "ms_per_frame": a.elapsed_time(b) / frames}
        for _, m in extra:
            m.close()
        rows.append(row)
    return rows


def serve_stream(mfa, server, models, tf, stream):
    """Submits the stream at its arrival times (a client thread sleeping until each one),
    waits for every ticket; returns (latencies ms, completed, rejected, wall seconds)."""
    import threading
    t0 = mfa.server_now() + 0.05
    tickets, rejected = [], 0
    lock = threading.Lock()

    def client():
        nonlocal rejected
        for r in stream:
            delay = t0 + r["t"] - mfa.server_now()
            if delay > 0:
                time.sleep(delay)
            try:
                tk = server.submit(models[r["model"]], r["camera"], tf, r["side"], r["side"], r["n_samples"],
                                   arrival_time=t0 + r["t"])
                with lock:
                    tickets.append(tk)
            except mfa.MfaError:
                rejected += 1

    th = threading.Thread(target=client)
    th.start()
    lat = []
    done = 0
    while th.is_alive() or done < len(tickets):
        with lock:
            pending = tickets[done:]
        for tk in pending:
            lat.append(server.wait(tk, 600000.0))
            server.release(tk)
            done += 1
        if not pending:
            time.sleep(0.002)
    th.join()
    wall = mfa.server_now() - t0
    return lat, done, rejected, wall


def run_serve(mfa, rates, duration, size_scale=1.0, max_slots=16, min_requests=0):
    """Each rate's stream lasts max(duration, min_requests / rate) seconds of arrivals."""
    import synth
    specs, f16, f32 = serve_models(mfa, size_scale)
    tf = mfa.transfer_fn(synth.ramp_tf(256, 0.05), shading=True)
    budget = 2 << 30
    out = {"models": serve_model_table(mfa, specs, f16, f32, tf), "hbm_budget_bytes": budget, "rates": {}}

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(math.ceil(q * len(v))) - 1)] if v else None

    for rate in rates:
        stream = synth.config5_requests(rate, max(duration, min_requests / rate))
        row = {"requests": len(stream)}
        for name, models, cfg in (("served_f16", f16, dict(max_slots=max_slots, mode=0)),
                                  ("plain_f32", f32, dict(max_slots=1, priority_levels=1, mode=1)),
                                  ("plain_f16", f16, dict(max_slots=1, priority_levels=1, mode=1))):
            srv = mfa.Server(hbm_budget_bytes=budget, max_queue=4096, **cfg)
            lat, done, rej, wall = serve_stream(mfa, srv, models, tf, stream)
            srv.close()
            row[name] = {"frames_per_s": done / wall if wall > 0 else None, "p50_ms": pct(lat, 0.5),
                         "p99_ms": pct(lat, 0.99), "completed": done, "rejected": rej, "wall_s": wall}
        out["rates"][str(rate)] = row
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving comparison")
    ap.add_argument("--no-side-rows", action="store_true",
                    help="skip the rows after the timed step (precision, segments, isosurface, Marschner-Lobb, "
                         "encoding, render quality), e.g. for profiling runs")
    ap.add_argument("--side-rows", nargs="+", choices=SIDE_ROWS, default=None,
                    help="run only these rows after the timed step (default: all of them, in this order: "
                         + ", ".join(SIDE_ROWS) + ")")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[20.0, 50.0, 100.0, 200.0],
                    help="request rates (1/s)")
    ap.add_argument("--serve-duration", type=float, default=5.0, help="minimum seconds of arrivals per rate")
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="minimum requests per rate (the stream lasts max(duration, requests / rate))")
    ap.add_argument("--variant", type=int, default=None, help="render kernel variant (skips the autotuner)")
    ap.add_argument("--tile-shape", type=int, default=None, help="ray-tile shape (skips the autotuner)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)      # at least three untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
