"""Continuous-batching server for many concurrent deformation streams on one GPU.

Each stream (one tissue surface seen by one camera) keeps its template, control points, blend
tables, normal-equation buffers and warm-start deformation resident in device memory. Frames
arrive asynchronously; every scheduler round (``poll``)

  1. completes the batches whose GPU work has finished (results read to the host, futures
     resolved, latency = result on the host - arrival),
  2. admits waiting streams while the device-memory budget allows,
  3. stages the next queued frame of every admitted stream that has none staged: the frame is
     submitted at once (copy to the device, frame preparation and RANSAC on the stream's own CUDA
     stream), into the frame slot its in-flight solve does not read, so this work overlaps the
     batch already on the GPU,
  4. launches one batch (one batched Gauss-Newton solve) over every admitted stream that has a
     staged frame and is not in flight, if no batch is on the GPU, or if fewer than max_inflight
     are and the ready streams make up at least min_fill of the admitted ones; otherwise the
     ready frames wait and join the next batch. Under load this keeps the batches full (two
     half-size groups taking turns would each pay a whole solve's fixed cost), while a burst
     still gets a batch of its own beside the running one.

Batches in flight together run on their own CUDA streams (their stream sets are disjoint), so
frames arriving while others are on the GPU are admitted into the next batch and their work
overlaps on the device. The GPU engine keeps two long-lived batch objects over every admitted
stream and solves each launch's streams as a masked solve, so a launch allocates and captures
nothing.

The engine is pluggable: ``GpuEngine`` drives libdefsolve; tests use a fake engine to check the
host logic without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from concurrent.futures import Future

import numpy as np


@dataclasses.dataclass
class StreamSpec:
    template_depth: np.ndarray      # (H, W) float32
    K: tuple                        # fx, fy, cx, cy
    nodes: np.ndarray               # (N,) int32 control-point pixels
    max_matches: int = 4096


@dataclasses.dataclass
class FrameIn:
    depth: np.ndarray
    match_idx: np.ndarray
    match_xyz: np.ndarray
    hyp: np.ndarray


@dataclasses.dataclass
class Result:
    q: np.ndarray                   # (N, 4)
    t: np.ndarray                   # (N, 3)
    pos: np.ndarray                 # (N, 3) control-point positions
    latency_s: float
    batch_size: int


def stream_bytes(W: int, H: int, N: int, M: int, precision: int) -> int:
    """Device bytes one stream holds (template, frame, blend tables, system buffers)."""
    npx, n = W * H, 6 * N
    nbp = 14 * N
    b = npx * (4 + 24 + 4 + 4 + 2 * (16 + 16) + 4)      # depths, FP64 template, 2 frame slots
    b += npx * (16 + 16 + 4)                            # sorted points, weights, rank
    # state, node tables, ARAP diagonal blocks, data blocks
    b += N * (8 * 7 + 64 + 96 + 48 * 4) + nbp * (36 * 4 + 12)
    b += n * n * 4                                      # FP32 system
    if precision == 0:
        b += n * n * 8                                  # FP64 factor
    elif precision == 2:
        b += n * n * 4                                  # FP32 factor
    b += n * (8 * 3 + 8 * 3 + 4)                        # vectors
    tb = 32 if precision == 0 else 64
    nt = (n + tb - 1) // tb
    tsz = 8 if precision == 0 else 4
    b += 4 * (nt + 2 * nt * nt) + tsz * nt * tb * tb
    # packed factor tiles: FP64 transposed padded tiles; FP32: the larger of the tensor-core
    # layouts (64 x 64 tiles of 8192 floats, 128 x 128 blocks of 32768 floats, hi / lo), which
    # also holds the SIMT kernel's tiles
    nb = (n + 127) // 128
    if precision == 0:
        b += tsz * nt * (nt + 1) // 2 * tb * (tb + 16 // tsz)
    else:
        b += tsz * max(nt * (nt + 1) // 2 * 8192, nb * (nb + 1) // 2 * 32768)
    b += nt * (nt + 1) // 2 * 16 * 2 + nb * (nb + 1) // 2 * 16   # task lists
    b += 2 * M * (4 + 12 + 4 + 4) + M * (8 * 3 + 4 * 6)  # 2 slots of matches + RANSAC results
    b += M * 64 * (7 * 8 + 4) + M * 8                   # RANSAC scratch, weights, bitsets
    return int(b)


class GpuEngine:
    """libdefsolve behind the server: one handle per admitted stream, and two long-lived batches
    over all admitted handles (one per batch in flight). A launch solves the ready streams as a
    masked solve of a free batch (ds_batch_solve_masked): the same captured graph serves every
    subset, so launching allocates and captures nothing. The batches are rebuilt when the
    admitted set changes."""

    def __init__(self, params=None, use_graph=True, n_batches=2):
        import torch
        from . import build, defsolve
        build.build()
        self.d = defsolve
        self.torch = torch
        self.params = params if params is not None else defsolve.default_params(precision=2)
        self.params.use_graph = 1 if use_graph else 0
        self.n_batches = n_batches
        self.handles = []          # admitted solvers, in batch order
        self.batches = []          # [batch, stream, in-flight token or None]
        self.dirty = True
        # per stream: two sets of pinned host staging of its frames, used in turn (a copy from
        # pageable memory would make the host wait for the stream's earlier work), and which set
        # the next frame takes
        self.staging = {}
        self.turn = {}

    @property
    def precision(self):
        return int(self.params.precision)

    def _drop_batches(self):
        for b, _, _ in self.batches:
            self.d.ds_batch_destroy(b)    # waits for the batch's stream
        self.batches = []
        self.dirty = True

    def create(self, spec: StreamSpec):
        s = self.d.Solver(spec.template_depth, spec.K, spec.nodes, self.params)
        H, W = spec.template_depth.shape
        M = spec.max_matches
        t = self.torch
        pin = lambda shape, dt: t.empty(shape, dtype=dt, pin_memory=True).numpy()
        self.staging[id(s)] = [(pin((H, W), t.float32), pin((M,), t.int32),
                                pin((M, 3), t.float32), pin((int(self.params.n_hyp),), t.int32))
                               for _ in range(2)]
        self.turn[id(s)] = 0
        self._drop_batches()
        self.handles.append(s)
        return s

    def destroy(self, s):
        self._drop_batches()
        self.handles = [h for h in self.handles if h is not s]
        self.staging.pop(id(s), None)
        self.turn.pop(id(s), None)
        s.close()

    def submit(self, s, f: FrameIn):
        """Copies the frame into one of the stream's two pinned staging sets and submits it
        from there (its copies to the device are asynchronous). The set is free again: the server
        keeps at most one frame staged and one in flight per stream, so the frame that used this
        set two submissions ago has been solved, after its copies."""
        k = self.turn[id(s)]
        self.turn[id(s)] = 1 - k
        dep, mi, mx, hy = self.staging[id(s)][k]
        M = len(f.match_idx)
        np.copyto(dep, f.depth)
        np.copyto(mi[:M], f.match_idx)
        np.copyto(mx[:M], f.match_xyz)
        np.copyto(hy[:len(f.hyp)], f.hyp)
        s.submit(dep, mi[:M], mx[:M], hy[:len(f.hyp)])

    def launch(self, solvers, iters):
        if self.dirty:
            for _ in range(self.n_batches):
                stream = self.torch.cuda.Stream()
                b = self.d.ds_batch_create([h.h for h in self.handles], stream.cuda_stream)
                self.batches.append([b, stream, None])
            self.dirty = False
        slot = next(x for x in self.batches if x[2] is None)
        on = {id(h) for h in solvers}
        mask = [1 if id(h) in on else 0 for h in self.handles]
        e0 = self.torch.cuda.Event(enable_timing=True)
        e0.record(slot[1])
        self.d.ds_batch_solve_masked(slot[0], mask, iters)
        ev = self.torch.cuda.Event(enable_timing=True)
        ev.record(slot[1])
        token = (slot, ev, e0)
        slot[2] = token
        return token

    def gpu_ms(self, token) -> float:
        """Device time of a completed launch (its batch stream, from the start of the solve)."""
        return token[2].elapsed_time(token[1])

    def done(self, token) -> bool:
        slot, ev = token[0], token[1]
        if ev.query():
            if slot[2] is token:
                slot[2] = None
            return True
        return False

    def read(self, s):
        q, t, p = s.deformation()
        return q, t, p

    def device_bytes(self, s) -> int:
        """Bytes the library reports the stream's handle holds now."""
        return self.d.ds_get_device_bytes(s.h)


class Server:
    def __init__(self, engine, budget_bytes: int, iters: int = 10, max_batch: int = 64,
                 max_inflight: int = 2, min_fill: float = 0.6, clock=time.perf_counter):
        self.engine = engine
        self.budget = int(budget_bytes)
        self.iters = iters
        self.max_batch = max_batch
        # batches on the GPU at once: frames that arrive meanwhile wait and join the next batch,
        # so batches grow with the load instead of splitting into many small concurrent ones
        self.max_inflight = max_inflight
        # share of the admitted streams that must be ready before a batch is launched beside
        # one already on the GPU (0: launch whenever a batch slot is free)
        self.min_fill = float(min_fill)
        slots = getattr(engine, "n_batches", None)
        if slots is not None and slots < max_inflight:
            raise ValueError(f"the engine keeps {slots} batches, fewer than max_inflight = "
                             f"{max_inflight}")
        self.clock = clock
        self.used = 0
        self.streams = {}                 # sid -> dict(spec, solver, queue, busy, bytes)
        self.waiting = collections.deque()  # sids waiting for admission
        self.in_flight = []               # (token, [sid], [(future, t_arrival)])
        self.latencies = []
        self.completed = 0
        self.t_first = None
        self.t_last = None
        self.batches = 0
        self.batch_sizes = []
        self.gpu_ms = []          # device time of each completed batch (when the engine reports it)
        self.done_batches = []    # (frames, device ms) of each completed batch, when reported
        self.host_ms = []         # host time of each launch (the batched solve's enqueue)
        self.submit_ms = []       # host time of each frame submission (staging)
        self.read_ms = []         # host time of each result read

    # -- streams
    def open_stream(self, sid, spec: StreamSpec) -> bool:
        """Registers a stream; returns True if it was admitted now, False if it waits for
        device memory (its frames queue up meanwhile)."""
        if sid in self.streams:
            raise KeyError(f"stream {sid} already open")
        H, W = spec.template_depth.shape
        nbytes = stream_bytes(W, H, len(spec.nodes), spec.max_matches, self.engine.precision)
        if nbytes > self.budget:
            raise ValueError(f"stream {sid} needs {nbytes} B, more than the whole budget")
        self.streams[sid] = dict(spec=spec, solver=None, queue=collections.deque(), busy=False,
                                 staged=None, bytes=nbytes)
        self.waiting.append(sid)
        self._admit()
        return self.streams[sid]["solver"] is not None

    def close_stream(self, sid):
        st = self.streams[sid]
        if st["busy"] or st["staged"] is not None:
            raise RuntimeError(f"stream {sid} has a frame in flight or staged")
        for fut, _, _ in st["queue"]:
            fut.cancel()
        if st["solver"] is not None:
            self.engine.destroy(st["solver"])
            self.used -= st.get("counted", 0)
        else:
            self.waiting.remove(sid)
        del self.streams[sid]
        self._admit()

    def _admit(self):
        while self.waiting:
            sid = self.waiting[0]
            st = self.streams[sid]
            if self.used + st["bytes"] > self.budget:
                break
            self.waiting.popleft()
            st["solver"] = self.engine.create(st["spec"])
            self._account(st)

    def _account(self, st):
        """Counts a stream at the larger of its estimate and what the engine reports it holds
        (the library's own allocation count), so growth the estimate missed is not lost."""
        actual = int(getattr(self.engine, "device_bytes", lambda s: 0)(st["solver"]))
        new = max(st["bytes"], actual)
        self.used += new - st.get("counted", 0)
        st["counted"] = new
        st["bytes"] = new

    # -- frames
    def submit(self, sid, frame: FrameIn, t_arrival=None) -> Future:
        """Queues a frame. A frame with more matches than the stream's max_matches is refused
        (ValueError): its buffers would outgrow the device bytes the stream was admitted with."""
        st = self.streams[sid]
        if frame.match_idx is not None and len(frame.match_idx) > st["spec"].max_matches:
            raise ValueError(f"stream {sid}: {len(frame.match_idx)} matches exceed its "
                             f"max_matches = {st['spec'].max_matches}")
        fut = Future()
        t = self.clock() if t_arrival is None else t_arrival
        if self.t_first is None:
            self.t_first = t
        st["queue"].append((fut, t, frame))
        return fut

    def poll(self) -> int:
        """One scheduler round; returns the number of frames completed."""
        n_done = 0
        still = []
        for token, sids, items in self.in_flight:
            if self.engine.done(token):
                now_batch = len(sids)
                if hasattr(self.engine, "gpu_ms"):
                    g = self.engine.gpu_ms(token)
                    self.gpu_ms.append(g)
                    self.done_batches.append((now_batch, g))
                for sid, (fut, t_arr) in zip(sids, items):
                    st = self.streams[sid]
                    r0 = self.clock()
                    q, t, p = self.engine.read(st["solver"])
                    self.read_ms.append((self.clock() - r0) * 1e3)
                    now = self.clock()
                    lat = now - t_arr
                    self.latencies.append(lat)
                    st["busy"] = False
                    fut.set_result(Result(q, t, p, lat, now_batch))
                    self.completed += 1
                    self.t_last = now
                    n_done += 1
            else:
                still.append((token, sids, items))
        self.in_flight = still
        self._admit()
        self._stage()
        ready = [sid for sid, st in self.streams.items()
                 if st["staged"] is not None and not st["busy"]]
        ready = ready[: self.max_batch]
        admitted = sum(1 for st in self.streams.values() if st["solver"] is not None)
        if ready and len(self.in_flight) < self.max_inflight and (
                not self.in_flight or len(ready) >= self.min_fill * admitted):
            h0 = self.clock()
            solvers, items = [], []
            for sid in ready:
                st = self.streams[sid]
                items.append(st["staged"])
                st["staged"] = None
                st["busy"] = True
                solvers.append(st["solver"])
            token = self.engine.launch(solvers, self.iters)
            self.host_ms.append((self.clock() - h0) * 1e3)
            self.in_flight.append((token, ready, items))
            self.batches += 1
            self.batch_sizes.append(len(ready))
            self._stage()       # the launched streams' next frames overlap their solve
        return n_done

    def _stage(self):
        """Submits the next queued frame of every admitted stream that has none staged (one
        frame staged and one in flight per stream at most: the handle's two frame slots)."""
        for st in self.streams.values():
            if st["solver"] is None or st["staged"] is not None or not st["queue"]:
                continue
            fut, t_arr, frame = st["queue"].popleft()
            h0 = self.clock()
            self.engine.submit(st["solver"], frame)
            self.submit_ms.append((self.clock() - h0) * 1e3)
            self._account(st)
            st["staged"] = (fut, t_arr)

    def pending(self) -> int:
        return sum(len(st["queue"]) + (st["staged"] is not None)
                   for st in self.streams.values()) + sum(len(s) for _, s, _ in self.in_flight)

    def drain(self, idle_sleep=0.0):
        """Polls until every queued frame is done. Raises RuntimeError instead of spinning when
        the only frames left belong to streams still waiting for admission while nothing is on
        the GPU: no batch will complete to free memory for them (close a stream first)."""
        while self.pending():
            if self.poll() == 0 and idle_sleep:
                time.sleep(idle_sleep)
            if not self.in_flight and not any(
                    st["solver"] is not None and (st["queue"] or st["staged"] is not None)
                    for st in self.streams.values()) and self.pending():
                raise RuntimeError("frames left only on streams waiting for device memory; "
                                   "close a stream to admit them")

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        span = (self.t_last - self.t_first) if self.completed and self.t_last else float("nan")
        return {"frames": self.completed, "frames_per_s": self.completed / span if span else None,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "batches": self.batches,
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "mean_gpu_ms_per_batch": float(np.mean(self.gpu_ms)) if self.gpu_ms else None,
                "mean_host_ms_per_launch": float(np.mean(self.host_ms)) if self.host_ms else None,
                "mean_host_ms_per_submit": float(np.mean(self.submit_ms)) if self.submit_ms else None,
                "mean_read_ms_per_frame": float(np.mean(self.read_ms)) if self.read_ms else None,
                "device_bytes": self.used, "full_batches": self._full_batches()}

    def _full_batches(self):
        """The batches that carried every admitted stream (the load the server saturates at): how
        many, and their frames per second of device time."""
        if not self.done_batches:
            return None
        top = max(n for n, _ in self.done_batches)
        full = [(n, g) for n, g in self.done_batches if n == top]
        ms = sum(g for _, g in full)
        return {"size": top, "batches": len(full),
                "frames_per_s_device": sum(n for n, _ in full) / (ms * 1e-3) if ms > 0 else None}


def poisson_schedule(rng: np.random.Generator, rates_hz, n_total: int):
    """Merged arrival schedule of independent Poisson streams: list of (t, stream index), the
    first n_total arrivals."""
    events = []
    horizon = 1.0
    while True:
        events = []
        for s, r in enumerate(rates_hz):
            t = 0.0
            while True:
                t += rng.exponential(1.0 / r)
                if t > horizon:
                    break
                events.append((t, s))
        if len(events) >= n_total:
            break
        horizon *= 2.0
    events.sort()
    return events[:n_total]
