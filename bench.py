#!/usr/bin/env python3
"""Benchmark of the per-frame deformation solve on GB300.

Workload: concurrent streams of the 320x240 / 256-control-point / 2000-match sequence. A frame is
frame preparation, 1-point RANSAC preselection and 10 damped Gauss-Newton iterations (ICP + ORB +
dense ARAP, assembly, Cholesky, solves, update), warm-started from the stream's previous frame.
A step is one frame of every one of S streams (default 32), solved as one batch in mixed
precision (FP32 J^T J and factorisation; two refinement steps whose residuals are accumulated
in double-float FP32 arithmetic, ~48 bits).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32_refine|fp32|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

Prints one JSON line (rank 0). `value` is frames/s with inputs resident in device memory,
timed with CUDA events on the library's stream, L2 flushed before every step (outside the
events). Next to it: the plain single-stream FP32 solve (the comparison the metric names), a
served run with Poisson arrivals (continuous batching, p50/p99 latency), `e2e` (the same metric
through the C ABI with pinned host buffers: host->device copies of the frames, the solve and the
device->host read of the deformations, wall clock), the factorisation's roofline and clocks.
Multi-GPU runs are independent replicas (one set of streams per rank, no collective).
"""
from __future__ import annotations

import argparse
import hashlib
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
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_chol_dag launch on this
# workload (32 problems, FP32 factor), from an ncu capture of one launch of the warm-up steps
# (`ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum -k regex:k_chol_dag -s 2 -c 1 ...`).
# It describes the kernel source it was taken on (first 16 hex digits of the sha256 of
# csrc/chol.cu + csrc/dev_util.cuh) and is reported as null for any other.
CHOL_TRAFFIC = {"chol_sha256": "a3f5333f6fac6ff8", "precision": 2, "streams": 32,
                "bytes": 663056896 + 355572480}


def max_over_ranks(x, world, dev):
    """The slowest rank's time: replicas run independent streams, the job ends with the last."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, total_s):
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / total_s


def replica_seeds(rank, n_scenes):
    """Scene seeds of a rank: every replica solves its own streams."""
    return [1000 + 100 * rank + k for k in range(n_scenes)]


def _measured_bf16():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0   # earlier GB300 measurement, used when the file is absent


def _measured_hbm():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0   # earlier GB300 measurement, used when the file is absent


def _chol_source_digest():
    """First 16 hex digits of the sha256 of the factorisation kernel's sources (chol.cu and the
    device helpers it includes)."""
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2007_08576_gb300",
                        "csrc")
    h = hashlib.sha256()
    for name in ("chol.cu", "dev_util.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _chol_traffic(prec, streams):
    digest = _chol_source_digest()
    c = CHOL_TRAFFIC
    if digest != c["chol_sha256"] or prec != c["precision"] or streams != c["streams"]:
        return None
    return c["bytes"]


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


def oracle_params(args):
    """The oracle's parameters for the method variant the GPU arm runs."""
    from oracle import solver
    return solver.Params(solver=args.solver, assoc=args.assoc, ransac_o1=args.ransac_o1)


def variant_params(d, args, prec):
    """The CUDA path's ds_params for the same variant."""
    return d.default_params(precision=prec, factor_tc=1 if args.factor_tc else 0,
                            solver=1 if args.solver == "block_jacobi" else 0,
                            assoc=1 if args.assoc == "bilinear" else 0,
                            ransac_o1=1 if args.ransac_o1 == "warm" else 0)


def cpu_baseline(sc, prm):
    """The FP64 oracle on the host cores: one whole frame (prep, RANSAC, 10 iterations)."""
    from oracle import solver
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    f = sc.frames[0]
    t0 = time.perf_counter()
    solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, prm, iters=ITERS)
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


def orb_frontend(d, torch, dev, S, K, W, n_scenes, flush):
    """Section 2.1's feature step for S streams: every step detects and describes each stream's
    live image (with its depth) and matches it against that stream's template features, on the
    streams' own CUDA streams at once; images resident on the device, L2 flushed before each step.
    Device time from an event before the fork to an event after the join."""
    from synth import CONFIGS, make_textured_scene, orb_pattern
    pat = orb_pattern(7)
    scenes = [make_textured_scene(CONFIGS[WORKLOAD], 1000 + j, n_frames=1) for j in range(n_scenes)]
    streams = [torch.cuda.Stream(device=dev) for _ in range(S)]
    tm, lv, imgs = [], [], []
    for j in range(S):
        ts = scenes[j % n_scenes]
        sc = ts.scene
        T = d.Orb(sc.W, sc.H, sc.K, pat, stream=streams[j].cuda_stream)
        T.detect(ts.template_image, np.ascontiguousarray(sc.template_depth, np.float32))
        L = d.Orb(sc.W, sc.H, sc.K, pat, stream=streams[j].cuda_stream)
        tm.append(T)
        lv.append(L)
        imgs.append((torch.from_numpy(ts.images[0]).to(dev),
                     torch.from_numpy(np.ascontiguousarray(sc.frames[0].depth, np.float32)).to(dev)))
    torch.cuda.synchronize()
    main = torch.cuda.current_stream(dev)

    def step():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for j in range(S):
            streams[j].wait_event(e0)
            lv[j].detect(imgs[j][0], imgs[j][1])
            d.ds_orb_match(tm[j].o, lv[j].o)
        for j in range(S):
            ev = torch.cuda.Event()
            ev.record(streams[j])
            main.wait_event(ev)
        e1.record(main)
        return e0, e1

    for _ in range(W):
        flush.fill_(0.0)
        step()
    torch.cuda.synchronize()
    n_launch0 = d.ds_get_counters()
    ms = []
    for i in range(K):
        flush.fill_(float(i))
        e0, e1 = step()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    launches = (d.ds_get_counters() - n_launch0) / K
    kp = [lv[j].keypoints()["pix"].size for j in range(S)]
    mt = [d.ds_orb_num_matches(lv[j].o) for j in range(S)]
    for o in tm + lv:
        o.close()
    med = float(np.median(ms))
    return {"streams": S, "image": f"{scenes[0].scene.W}x{scenes[0].scene.H}",
            "distinct_scenes": n_scenes, "ms_per_step": round(med, 4),
            "frames_per_s": round(S / (med * 1e-3), 1),
            "keypoints_per_frame": round(float(np.mean(kp)), 1),
            "matches_per_frame": round(float(np.mean(mt)), 1),
            "gpu_launches_per_step": int(launches),
            "step": f"detect + describe + match one live image of each of {S} streams",
            "l2": "flushed (256 MB write) before each step"}


def _stats_ms(xs):
    a = np.asarray(xs, dtype=np.float64)
    return {"p50": round(float(np.percentile(a, 50)), 4), "p99": round(float(np.percentile(a, 99)), 4),
            "mean": round(float(a.mean()), 4)}


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
    from paper_2007_08576_gb300.serve import FrameIn, GpuEngine, Server, StreamSpec, poisson_schedule

    K, W, S = args.steps, args.warmup, args.streams
    n_scenes = min(args.scenes, S)
    F = args.frames
    from synth import CONFIGS, make_scene
    scenes = [make_scene(CONFIGS[WORKLOAD], sd, n_frames=F) for sd in replica_seeds(rank, n_scenes)]
    N = len(scenes[0].nodes)
    M = len(scenes[0].frames[0].match_idx)
    n = 6 * N
    prec = PREC[args.precision]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def dev_frames(sc):
        return [(torch.from_numpy(f.depth).to(dev), torch.from_numpy(f.match_idx).to(dev),
                 torch.from_numpy(np.ascontiguousarray(f.match_xyz)).to(dev),
                 torch.from_numpy(f.hyp).to(dev)) for f in sc.frames]

    dframes = [dev_frames(sc) for sc in scenes]

    # ---------------------------------------------------------------- batched mixed precision
    solver_id = 1 if args.solver == "block_jacobi" else 0
    prm = variant_params(d, args, prec)
    handles, hstreams = [], []
    for j in range(S):
        sc = scenes[j % n_scenes]
        hs = torch.cuda.Stream(device=dev)    # per-stream frame work overlaps across streams
        h = d.ds_create_template(sc.template_depth, sc.W, sc.H, sc.K, prm, hs.cuda_stream)
        d.ds_set_control_points(h, sc.nodes)
        handles.append(h)
        hstreams.append(hs)
    batch = d.ds_batch_create(handles, stream.cuda_stream)
    d.ds_batch_set_tracing(batch, True)

    def step(i, e_start=None):
        for j, h in enumerate(handles):
            if e_start is not None:
                hstreams[j].wait_event(e_start)   # the frame work belongs to the timed step
            dep, mi, mx, hy = dframes[j % n_scenes][i % F]
            d.ds_submit_frame(h, dep, mi, mx, M, hy)
        d.ds_batch_solve(batch, ITERS)

    for i in range(W):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    k0 = d.ds_get_counters(None)
    # Steps run back to back as a stream of frames would: the host enqueues step i + 1 while the
    # device runs step i (no host synchronisation between steps). Each step's span is the device
    # time from its start event (after the L2 flush) to its end event; the throughput divides
    # the K steps' frames by the time from the first start event to the last end event.
    step_ms, phase, host_ms = [], np.zeros(4), []
    ev = []
    with ClockSampler(local) as clk:
        for i in range(K):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            th = time.perf_counter()
            # each step's frame work starts at its start event, after the previous solve: the
            # library lets submissions overlap the previous solve (two frame slots per handle),
            # but here that measured slower (the RANSAC CTAs take shared memory the persistent
            # factorisation needs)
            step(W + i, e0)
            host_ms.append((time.perf_counter() - th) * 1e3)
            e1.record(stream)
            ev.append((e0, e1))
        ev[-1][1].synchronize()
    d.ds_batch_status(batch)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    launches = d.ds_get_counters(None) - k0
    # phase split (linearise / factorise / solve / update, CUDA events inside the captured
    # graph, overwritten by every solve): K more steps, each read after it completes
    for i in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        step(W + K + i)
        torch.cuda.synchronize()
        phase += d.ds_batch_phase_times(batch)
    total_s = max_over_ranks(ev[0][0].elapsed_time(ev[-1][1]) * 1e-3, world, dev)
    value = job_throughput(world, S * K, total_s)

    # end to end through the C ABI: pinned host frames in, deformations out, every step
    pin = [[[torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
             for a in (f.depth, f.match_idx, f.match_xyz, f.hyp)] for f in sc.frames] for sc in scenes]
    outs = [[torch.empty(shape, dtype=torch.float32).pin_memory().numpy()
             for shape in ((N, 4), (N, 3), (N, 3))] for _ in range(S)]
    d.ds_batch_set_tracing(batch, False)

    def e2e_submit(i):
        for j, h in enumerate(handles):
            dep, mi, mx, hy = pin[j % n_scenes][i % F]
            d.ds_submit_frame(h, dep, mi, mx, M, hy)

    def e2e_read():
        for j, h in enumerate(handles):
            d.ds_get_deformation(h, *outs[j])

    # As a stream of frames runs: step i + 1's frames are submitted (host-to-device copies,
    # preparation and RANSAC, into each handle's other frame slot) while step i's batch solves,
    # then step i's deformations are read back, then step i + 1 is solved. Every step's input
    # copies and result reads lie inside the timed region, which spans the K steps.
    for i in range(W):
        e2e_submit(i)
        d.ds_batch_solve(batch, ITERS)
        e2e_read()
    with torch.cuda.stream(stream):
        flush.fill_(0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_submit(W)
    d.ds_batch_solve(batch, ITERS)
    for i in range(W, W + K):
        if i + 1 < W + K:
            e2e_submit(i + 1)
        e2e_read()
        if i + 1 < W + K:
            d.ds_batch_solve(batch, ITERS)
    e2e_tot = max_over_ranks(time.perf_counter() - t0, world, dev)
    f0 = scenes[0].frames[0]
    h2d = S * (f0.depth.nbytes + f0.match_idx.nbytes + np.ascontiguousarray(f0.match_xyz).nbytes +
               f0.hyp.nbytes)
    d2h = S * sum(o.nbytes for o in outs[0])
    d.ds_batch_destroy(batch)
    for h in handles:
        d.ds_destroy(h)

    # ---------------------------------------------------------------- plain single-stream FP32
    pprm = d.default_params(precision=PREC["fp32"])
    hp = d.ds_create_template(scenes[0].template_depth, scenes[0].W, scenes[0].H, scenes[0].K,
                              pprm, stream.cuda_stream)
    d.ds_set_control_points(hp, scenes[0].nodes)
    plain_ms = []
    for i in range(W + K):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dep, mi, mx, hy = dframes[0][i % F]
        d.ds_submit_frame(hp, dep, mi, mx, M, hy)
        d.ds_solve(hp, ITERS, False)
        e1.record(stream)
        e1.synchronize()
        if i >= W:
            plain_ms.append(e0.elapsed_time(e1))
    d.ds_destroy(hp)
    plain_fps = 1e3 * len(plain_ms) / sum(plain_ms)

    # ---------------------------------------------------------------- served, Poisson arrivals
    def serve_run(rate_scale, n_frames, seed):
        rng = np.random.default_rng(seed)
        rates = rng.uniform(15.0, 60.0, S) * rate_scale
        srv = Server(GpuEngine(variant_params(d, args, prec)),
                     budget_bytes=int(0.6 * torch.cuda.mem_get_info()[0]))
        for j in range(S):
            sc = scenes[j % n_scenes]
            srv.open_stream(j, StreamSpec(sc.template_depth, sc.K, sc.nodes, max_matches=M))
        sched = poisson_schedule(rng, rates, n_frames)
        cnt = [0] * S
        t_start = time.perf_counter()
        for t_arr, s_id in sched:
            now = time.perf_counter() - t_start
            while now < t_arr:
                srv.poll()
                now = time.perf_counter() - t_start
            f = scenes[s_id % n_scenes].frames[cnt[s_id] % F]
            cnt[s_id] += 1
            srv.submit(s_id, FrameIn(f.depth, f.match_idx, f.match_xyz, f.hyp),
                       t_arrival=t_start + t_arr)
            srv.poll()
        srv.drain()
        st = srv.stats()
        for j in range(S):
            srv.close_stream(j)
        return {"streams": S, "rates_hz": [round(float(r), 1) for r in rates[:4]] + ["..."],
                "offered_frames_per_s": round(float(rates.sum()), 1),
                "frames": st["frames"], "frames_per_s": round(st["frames_per_s"], 2),
                "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                "mean_batch": round(st["mean_batch"], 2), "batches": st["batches"]}

    served = served_low = None
    if rank == 0 and args.served_frames > 0:
        # the workload's rates (15-60 Hz per stream), then half of them (below saturation)
        served = serve_run(1.0, args.served_frames, 7)
        served_low = serve_run(0.5, args.served_frames // 2, 8)

    orb_fe = None
    if rank == 0 and not args.no_orb:
        orb_fe = orb_frontend(d, torch, dev, S, K, W, min(4, n_scenes), flush)

    # ---------------------------------------------------------------- roofline of the factorisation
    flops_per_step = S * ITERS * n ** 3 / 3.0
    factor_ms = phase[1] / K
    achieved = flops_per_step / (factor_ms * 1e-3) / 1e12
    bound = "alu"
    unit = "TFLOP/s"
    if solver_id == 1:
        # no factorisation: the linearisation dominates; its algorithmic bytes are the ICP pass's
        # 64 B per template point (32 B template point + weights, 32 B gathered live point +
        # normal) per iteration
        pts = sum(int((sc.template_depth > 0).sum()) for sc in scenes) * S / len(scenes)
        bytes_per_step = 64.0 * pts * ITERS
        achieved = bytes_per_step / (phase[0] / K * 1e-3) / 1e9
        bound, unit = "hbm", "GB/s"
        peak, peak_src = _measured_hbm(), "MEASURED_PEAKS.json hbm_gbs"
    elif prec == 0:
        peak, peak_src = FP64_NOMINAL_TFLOPS, "nominal GB300 FP64 rate"
    elif args.factor_tc:
        # tensor-pipe work: three TF32 products per FP32 product; peak = measured bf16 burst x the
        # nominal dense TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)
        bound = "tensor"
        achieved *= 3.0
        peak, peak_src = _measured_bf16() * 1.1 / 2.25, "measured bf16 burst x nominal tf32/bf16"
    else:
        peak, peak_src = FP32_SIMT_TFLOPS, "152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz"
    dgemm = measure_dgemm_tflops(torch, dev) if prec == 0 else None
    traffic = None if (args.factor_tc or solver_id == 1) else _chol_traffic(prec, S)

    result = None
    if rank == 0:
        cpu = cpu_baseline(scenes[0], oracle_params(args)) if world == 1 and not args.no_cpu else None
        result = {
            "metric": METRIC, "value": round(value, 3), "unit": "frames/s", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": round(float(total_s * 1e3 / K), 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f32 residuals/J^T J, f64 Cholesky, double-f32 refine residuals",
                      "fp32": "f32", "fp32_refine": "f32 J^T J + Cholesky, double-f32 (48-bit) refine residuals"}[args.precision],
            "data": "synthetic (seeded heightfield + deformation + camera motion, ray-cast depth)",
            "config": {"workload": WORKLOAD, "template": "320x240", "control_points": N,
                       "matches": M, "gn_iters": ITERS, "precision": args.precision,
                       "solver": args.solver, "icp_association": args.assoc,
                       "ransac_o1": args.ransac_o1,
                       "factor": "tensor cores (tcgen05, 3xTF32)" if args.factor_tc else "FP32 SIMT tile kernel",
                       "streams_per_batch": S, "distinct_scenes": n_scenes, "frames_per_scene": F,
                       "step": f"one frame of each of {S} streams, one batched solve",
                       "l2": "flushed (256 MB write) before each step", "parallelism": f"replicas x{world}"},
            "latency_ms": _stats_ms(step_ms),
            "plain_gpu_single_stream": {"precision": "fp32", "frames_per_s": round(plain_fps, 3),
                                        "latency_ms": _stats_ms(plain_ms)},
            "speedup_vs_plain": round(value / (world * plain_fps), 2),
            "served": served,
            "served_half_rate": served_low,
            "orb_frontend": orb_fe,
            "host_enqueue_ms_per_step": round(float(np.median(host_ms)), 3),
            "phase_ms_per_step": {"linearize": round(phase[0] / K, 4), "factor": round(phase[1] / K, 4),
                                  "solve_refine": round(phase[2] / K, 4), "update": round(phase[3] / K, 4)},
            "e2e": {"value": round(job_throughput(world, S * K, e2e_tot), 3), "unit": "frames/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "roofline": {"bound": bound,
                         "kernel": ("linearisation (k_icp + k_orb + k_arap_assemble diagonal blocks)"
                                    if solver_id == 1 else
                                    "k_chol_tc (persistent tile Cholesky on tcgen05, all problems)"
                                    if args.factor_tc and prec != 0 else
                                    "k_chol_dag (persistent tile Cholesky, all problems)"),
                         "achieved": round(achieved, 4), "peak": peak, "unit": unit,
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "traffic_unit": "DRAM bytes per launch (ncu)",
                         "algorithmic_bytes": int(2 * S * n * n * (8 if prec == 0 else 4)),
                         "peak_source": peak_src,
                         "algorithmic": ("64 B per template point per iteration (ICP)"
                                         if solver_id == 1 else
                                         "3 x n^3/3 TF32 flop per factorisation, 10 per frame"
                                         if bound == "tensor" else
                                         "n^3/3 flop per factorisation, 10 per frame"),
                         "dgemm_measured_tflops": round(dgemm, 4) if dgemm else None},
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
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
    prm = oracle_params(args)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    N = len(sc.nodes)
    q = np.tile([1.0, 0, 0, 0], (N, 1))
    t = np.zeros((N, 3))
    t0 = time.perf_counter()
    tgt = solver.prepare_target(f.depth, tpl.K)
    rs = ransac.ransac_1p(solver.ransac_o1(tpl, f.match_idx, q, t, prm), f.match_xyz, f.hyp,
                          prm.H, prm.n_reweight, prm.keep_frac)
    t_pre = time.perf_counter() - t0
    orb = (f.match_idx, f.match_xyz.astype(np.float64), rs["mask"], rs["what"])
    w_arap = None
    from oracle import dqb

    def it():
        nonlocal q, t, w_arap
        lin, w_arap = solver.linearize(tpl, tgt, q, t, orb, w_arap, prm)
        Ad = solver.damp(lin.A, prm)
        delta = (solver.block_jacobi_solve(Ad, lin.b) if prm.solver == "block_jacobi"
                 else solver.cholesky_solve(Ad, lin.b))
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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="fp32_refine", choices=list(PREC))
    ap.add_argument("--streams", type=int, default=32, help="concurrent streams per batch")
    ap.add_argument("--scenes", type=int, default=8, help="distinct seeded scenes behind them")
    ap.add_argument("--frames", type=int, default=4, help="frames per scene (cycled)")
    ap.add_argument("--served-frames", type=int, default=2000, dest="served_frames")
    ap.add_argument("--no-cpu", action="store_true", dest="no_cpu")
    ap.add_argument("--no-orb", action="store_true", dest="no_orb",
                    help="skip the ORB feature front-end measurement")
    ap.add_argument("--solver", default="dense", choices=["dense", "block_jacobi"],
                    help="dense 6N x 6N Cholesky, or per-node 6 x 6 solves (Section 2)")
    ap.add_argument("--factor-tc", action="store_true", dest="factor_tc",
                    help="FP32 factorisation on the tensor cores (tcgen05, 3xTF32)")
    ap.add_argument("--assoc", default="nearest", choices=["nearest", "bilinear"],
                    help="ICP association: nearest pixel or bilinear blend of 4 pixels")
    ap.add_argument("--ransac-o1", default="template", choices=["template", "warm"],
                    dest="ransac_o1", help="RANSAC o1: template points or warm-start warped points")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
