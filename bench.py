#!/usr/bin/env python3
"""Benchmark of the per-frame deformation solve on GB300.

A step is one frame of the 320x240 / 256-control-point / 2000-match sequence workload: frame
preparation, 1-point RANSAC preselection and 10 damped Gauss-Newton iterations (ICP + ORB +
dense ARAP, assembly, Cholesky, solves, update), warm-started from the previous frame.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32|fp32_refine]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

Prints one JSON line (rank 0). `value` is frames/s with inputs resident in device memory,
timed with CUDA events on the library's stream, L2 flushed before every step (outside the
events). `e2e` is the same metric through the C ABI with pinned host buffers: host->device
copy of the frame, the solve and the device->host read of the deformation, wall clock.
Multi-GPU runs are independent replicas (one stream per rank, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "seq_320x240_n256"
ITERS = 10
METRIC = "frames/s and p50/p99 frame latency vs plain GPU solve, at ≤1e-3 mm error"
PREC = {"fp64": 0, "fp32": 1, "fp32_refine": 2}
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 rate per GPU (nominal)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gen_frames(n_frames: int, seed: int):
    from synth import CONFIGS, make_scene
    return make_scene(CONFIGS[WORKLOAD], seed, n_frames=n_frames)


def cpu_baseline(sc):
    """The FP64 oracle on the host cores: one whole frame (prep, RANSAC, 10 iterations)."""
    from oracle import solver
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes)
    f = sc.frames[0]
    t0 = time.perf_counter()
    solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, iters=ITERS)
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": 1.0 / dt, "unit": "frames/s", "cores": cores, "kind": "oracle",
            "sample": f"one {WORKLOAD} frame (prep, RANSAC, {ITERS} GN iterations), "
                      f"{dt:.1f} s wall, numpy/LAPACK threads on {cores} cores"}


def measure_dgemm_tflops(torch, dev):
    """cuBLAS FP64 GEMM rate (context for the FP64 roofline)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 3
    for _ in range(reps):
        a @ b
    e1.record()
    torch.cuda.synchronize()
    return 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12


def run_gpu(args):
    import torch
    import torch.distributed as dist
    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl", rank=rank, world_size=world,
                                device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2007_08576_gb300 import build
    build.build()
    from paper_2007_08576_gb300 import defsolve as d

    K, W = args.steps, args.warmup
    n_frames = max(2, min(K + W, args.max_frames))
    sc = gen_frames(n_frames, 1000 + rank)
    prm = d.default_params(precision=PREC[args.precision])
    stream = torch.cuda.Stream(device=dev)
    h = d.ds_create_template(sc.template_depth, sc.W, sc.H, sc.K, prm, stream.cuda_stream)
    d.ds_set_control_points(h, sc.nodes)
    N, M = len(sc.nodes), len(sc.frames[0].match_idx)
    n = 6 * N
    # device-resident inputs of every frame
    dev_frames = [(torch.from_numpy(f.depth).to(dev), torch.from_numpy(f.match_idx).to(dev),
                   torch.from_numpy(np.ascontiguousarray(f.match_xyz)).to(dev),
                   torch.from_numpy(f.hyp).to(dev)) for f in sc.frames]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    torch.cuda.synchronize()

    def step(i):
        dep, mi, mx, hy = dev_frames[i % len(dev_frames)]
        d.ds_submit_frame(h, dep, mi, mx, M, hy)
        d.ds_solve(h, ITERS, False)

    d.ds_set_tracing(h, True)
    for i in range(W):
        step(i)
    torch.cuda.synchronize()
    # timed region: per-step CUDA events on the library's stream, L2 flushed outside them
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    k0 = d.ds_get_counters(h)
    step_ms, phase = [], np.zeros(4)
    with ClockSampler(local) as clk:
        for i in range(K):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(W + i)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            phase += d.ds_get_phase_times(h)
    torch.cuda.synchronize()
    launches = d.ds_get_counters(h) - k0
    total_s = sum(step_ms) * 1e-3
    if world > 1:
        t = torch.tensor([total_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * K / total_s
    lat = np.array(step_ms)

    # end to end through the C ABI with pinned host buffers
    pin = []
    for f in sc.frames:
        arrs = []
        for a in (f.depth, f.match_idx, np.ascontiguousarray(f.match_xyz), f.hyp):
            t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            arrs.append(t.numpy())
        pin.append(arrs)
    out_q = torch.empty((N, 4), dtype=torch.float32).pin_memory().numpy()
    out_t = torch.empty((N, 3), dtype=torch.float32).pin_memory().numpy()
    out_p = torch.empty((N, 3), dtype=torch.float32).pin_memory().numpy()
    d.ds_set_tracing(h, False)
    e2e_s = []
    for i in range(W + K):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        torch.cuda.synchronize()
        dep, mi, mx, hy = pin[i % len(pin)]
        t0 = time.perf_counter()
        d.ds_submit_frame(h, dep, mi, mx, M, hy)
        d.ds_solve(h, ITERS, False)
        d.ds_get_deformation(h, out_q, out_t, out_p)
        t1 = time.perf_counter()
        if i >= W:
            e2e_s.append(t1 - t0)
    e2e_tot = sum(e2e_s)
    if world > 1:
        t = torch.tensor([e2e_tot], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_tot = float(t.item())
    h2d = sc.frames[0].depth.nbytes + sc.frames[0].match_idx.nbytes + \
        np.ascontiguousarray(sc.frames[0].match_xyz).nbytes + sc.frames[0].hyp.nbytes
    d2h = out_q.nbytes + out_t.nbytes + out_p.nbytes

    # roofline of the dominant kernel: the Cholesky factorisation (FP64: DFMA-bound)
    flops_per_factor = n ** 3 / 3.0
    factor_ms = phase[1] / K                     # per frame (ITERS factorisations)
    achieved = ITERS * flops_per_factor / (factor_ms * 1e-3) / 1e12
    if args.precision == "fp64":
        peak, unit, bound = FP64_NOMINAL_TFLOPS, "TFLOP/s", "alu"
    else:
        peak, unit, bound = 72.0, "TFLOP/s", "alu"   # FP32 SIMT nominal (152 SM x 128 FMA x 2 x 1.85 GHz)
    dgemm = measure_dgemm_tflops(torch, dev) if args.precision == "fp64" else None

    result = None
    if rank == 0:
        cpu = cpu_baseline(sc) if world == 1 and not args.no_cpu else None
        result = {
            "metric": METRIC, "value": round(value, 3), "unit": "frames/s", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": round(float(total_s * 1e3 / K), 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f32 residuals/J^T J, f64 Cholesky+refine",
                      "fp32": "f32", "fp32_refine": "f32 Cholesky, f64 refine"}[args.precision],
            "data": "synthetic (seeded heightfield + deformation + camera motion, ray-cast depth)",
            "config": {"workload": WORKLOAD, "template": "320x240", "control_points": N,
                       "matches": M, "gn_iters": ITERS, "precision": args.precision,
                       "frames_cycled": len(sc.frames), "l2": "flushed (256 MB write) before each step",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 4),
                           "p99": round(float(np.percentile(lat, 99)), 4),
                           "mean": round(float(lat.mean()), 4)},
            "phase_ms_per_frame": {"linearize": round(phase[0] / K, 4), "factor": round(phase[1] / K, 4),
                                   "solve_refine": round(phase[2] / K, 4), "update": round(phase[3] / K, 4)},
            "e2e": {"value": round(world * K / e2e_tot, 3), "unit": "frames/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "roofline": {"bound": bound, "kernel": "Cholesky factorisation (panel + trailing update)",
                         "achieved": round(achieved, 4), "peak": peak, "unit": unit,
                         "frac": round(achieved / peak, 4), "traffic": None,
                         "peak_source": "nominal GB300 FP64 rate" if args.precision == "fp64" else "nominal FP32 SIMT rate",
                         "dgemm_measured_tflops": round(dgemm, 4) if dgemm else None},
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
    d.ds_destroy(h)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if result is not None:
        print(json.dumps(result), flush=True)


def run_reference(args):
    """The FP64 CPU oracle as it stands: a step is one Gauss-Newton iteration of the workload's
    frame; frames/s = 1 / (prep + RANSAC + 10 x mean iteration)."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    from oracle import ransac, solver
    sc = gen_frames(1, 1000)
    f = sc.frames[0]
    prm = solver.Params()
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    t0 = time.perf_counter()
    tgt = solver.prepare_target(f.depth, tpl.K)
    rs = ransac.ransac_1p(tpl.X0[f.match_idx], f.match_xyz, f.hyp, prm.H, prm.n_reweight,
                          prm.keep_frac)
    t_pre = time.perf_counter() - t0
    orb = (f.match_idx, f.match_xyz.astype(np.float64), rs["mask"], rs["what"])
    N = len(sc.nodes)
    q = np.tile([1.0, 0, 0, 0], (N, 1))
    t = np.zeros((N, 3))
    w_arap = None
    from oracle import dqb

    def it():
        nonlocal q, t, w_arap
        lin, w_arap = solver.linearize(tpl, tgt, q, t, orb, w_arap, prm)
        delta = solver.cholesky_solve(solver.damp(lin.A, prm), lin.b)
        q, t = dqb.apply_step(q, t, delta)

    for _ in range(args.warmup):
        it()
    ts = []
    for _ in range(args.steps):
        a = time.perf_counter()
        it()
        ts.append(time.perf_counter() - a)
    frame_s = t_pre + ITERS * float(np.mean(ts))
    value = 1.0 / frame_s
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "frames/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(float(np.mean(ts)) * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "template": "320x240", "control_points": N,
                   "matches": len(f.match_idx), "gn_iters": ITERS,
                   "step": "one oracle Gauss-Newton iteration; frame = prep + RANSAC + 10 steps"},
        "cpu_baseline": {"value": round(value, 5), "unit": "frames/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{args.steps} GN iterations of one {WORKLOAD} frame + its prep/RANSAC"},
        "e2e": {"value": round(value, 5), "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="fp64", choices=list(PREC))
    ap.add_argument("--max-frames", type=int, default=12, dest="max_frames")
    ap.add_argument("--no-cpu", action="store_true", dest="no_cpu")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
