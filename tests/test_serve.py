"""Serving loop: host logic on the CPU with a fake engine; on the GPU, each stream's results in
the served mix equal the same stream solved alone."""
import numpy as np
import pytest

from paper_2007_08576_gb300.serve import (FrameIn, Server, StreamSpec, poisson_schedule,
                                          stream_bytes)


class FakeEngine:
    """Completes a launched batch after `delay` polls; 'solves' by counting frames. Models the
    library's two frame slots per handle: a solve takes the latest submitted frame, a stream has
    at most one solve in flight, and a frame may be submitted while one is (into the other
    slot), but never two frames beyond the last launched one."""

    precision = 2

    def __init__(self, delay=2):
        self.delay = delay
        self.launches = []
        self.polls = 0
        self.live = set()

    def create(self, spec):
        s = {"frames": 0, "submitted": 0, "launched": 0, "spec": spec}
        self.live.add(id(s))
        return s

    def destroy(self, s):
        self.live.discard(id(s))

    def submit(self, s, f):
        assert s["submitted"] == s["launched"], "a frame submitted over an unsolved one"
        s["submitted"] += 1

    def launch(self, solvers, iters):
        for s in solvers:
            assert s["launched"] == s["frames"], "a second solve of a stream in flight"
            assert s["submitted"] > s["launched"], "a solve without a new frame"
            s["launched"] = s["submitted"]
        tok = {"left": self.delay, "ids": [id(s) for s in solvers], "solvers": solvers,
               "upto": [s["submitted"] for s in solvers]}
        self.launches.append(tok)
        return tok

    def done(self, tok):
        tok["left"] -= 1
        if tok["left"] < 0:
            for s, u in zip(tok["solvers"], tok["upto"]):
                s["frames"] = u
            return True
        return False

    def read(self, s):
        N = len(s["spec"].nodes)
        return np.zeros((N, 4)), np.full((N, 3), float(s["frames"])), np.zeros((N, 3))


def _spec(W=80, H=60, N=32):
    return StreamSpec(np.full((H, W), 100.0, np.float32), (W, W, (W - 1) / 2, (H - 1) / 2),
                      np.arange(N, dtype=np.int32), max_matches=200)


def _frame():
    return FrameIn(None, None, None, None)


def test_admission_by_memory_budget():
    one = stream_bytes(80, 60, 32, 200, 2)
    eng = FakeEngine()
    srv = Server(eng, budget_bytes=int(2.5 * one))
    assert srv.open_stream("a", _spec())
    assert srv.open_stream("b", _spec())
    assert not srv.open_stream("c", _spec())         # waits: budget holds two streams
    assert srv.used == 2 * one and len(eng.live) == 2
    fc = srv.submit("c", _frame())                  # queued while not admitted
    srv.close_stream("a")                           # frees memory -> c admitted
    assert srv.streams["c"]["solver"] is not None and srv.used == 2 * one
    srv.drain()
    assert fc.result().t[0, 0] == 1.0
    with pytest.raises(ValueError):
        Server(eng, budget_bytes=one // 2).open_stream("x", _spec())


def test_continuous_batching_overlaps_and_keeps_order():
    eng = FakeEngine(delay=3)
    srv = Server(eng, budget_bytes=1 << 40, min_fill=0.0)
    for s in "abcd":
        srv.open_stream(s, _spec())
    f1 = [srv.submit(s, _frame()) for s in "ab"]
    srv.poll()                                       # batch 1: a, b
    assert eng.launches[-1]["ids"] and len(srv.in_flight) == 1
    f2 = [srv.submit(s, _frame()) for s in "cd"] + [srv.submit("a", _frame())]
    srv.poll()                                       # batch 2: c, d (a still busy)
    assert len(srv.in_flight) == 2
    ids2 = set(eng.launches[-1]["ids"])
    assert ids2 == {id(srv.streams["c"]["solver"]), id(srv.streams["d"]["solver"])}
    srv.drain()
    assert all(f.done() for f in f1 + f2)
    # stream a got its two frames in order (warm-start chain)
    assert f1[0].result().t[0, 0] == 1.0 and f2[2].result().t[0, 0] == 2.0
    st = srv.stats()
    assert st["frames"] == 5 and st["batches"] >= 3 and st["p99_ms"] >= st["p50_ms"]


def test_poisson_schedule():
    rng = np.random.default_rng(0)
    ev = poisson_schedule(rng, [15.0, 60.0], 200)
    assert len(ev) == 200 and all(a[0] <= b[0] for a, b in zip(ev, ev[1:]))
    counts = np.bincount([s for _, s in ev], minlength=2)
    assert counts[1] > 2 * counts[0]                 # rate ratio 4


@pytest.mark.gpu
def test_served_results_equal_alone():
    from gpu_common import lib
    from paper_2007_08576_gb300.serve import GpuEngine
    from synth import make_scene
    from synth.scene import Config
    d = lib()
    cfgs = [Config("s80", 80, 60, 32, 200, 5, 0.3, 0.3, 0.0, 4.0, 1.0, 0.3, 0.5, 3),
            Config("s120", 120, 90, 40, 300, 8, 0.4, 0.5, 0.1, 8.0, 1.0, 0.3, 0.5, 3),
            Config("s150", 150, 110, 50, 333, 8, 0.35, 0.5, 0.05, 6.0, 1.0, 0.2, 0.5, 3)]
    scenes = [make_scene(c, 500 + i, n_frames=3) for i, c in enumerate(cfgs)]
    p = d.default_params(precision=2)
    # alone: each stream's frames in order on its own handle
    alone = []
    for sc in scenes:
        s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
        outs = []
        for f in sc.frames:
            s.submit(f.depth, f.match_idx, f.match_xyz, f.hyp)
            s.solve(10, stats=False)
            outs.append(s.deformation()[2])
        alone.append(outs)
        s.close()
    # served: Poisson arrivals, continuous batching
    srv = Server(GpuEngine(d.default_params(precision=2)), budget_bytes=1 << 33)
    for i, sc in enumerate(scenes):
        srv.open_stream(i, StreamSpec(sc.template_depth, sc.K, sc.nodes, max_matches=400))
    rng = np.random.default_rng(3)
    sched = poisson_schedule(rng, [40.0, 25.0, 60.0], 9)
    nxt = [0, 0, 0]
    futs = {i: [] for i in range(3)}
    for _, s in sched:
        if nxt[s] >= 3:
            continue
        f = scenes[s].frames[nxt[s]]
        futs[s].append(srv.submit(s, FrameIn(f.depth, f.match_idx, f.match_xyz, f.hyp)))
        nxt[s] += 1
        srv.poll()
    for s in range(3):
        while nxt[s] < 3:
            f = scenes[s].frames[nxt[s]]
            futs[s].append(srv.submit(s, FrameIn(f.depth, f.match_idx, f.match_xyz, f.hyp)))
            nxt[s] += 1
    srv.drain()
    for s in range(3):
        for k, fut in enumerate(futs[s]):
            assert np.abs(fut.result().pos - alone[s][k]).max() <= 1e-4
    st = srv.stats()
    assert st["frames"] == 9
    for i in range(3):
        srv.close_stream(i)
    # the served results also equal the FP64 oracle's warm-started sequence of each stream
    from gpu_common import POS_TOL_MM, oracle_params
    from oracle import solver
    prm = oracle_params(p)
    for s, sc in enumerate(scenes):
        tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
        q0 = t0 = None
        for k, f in enumerate(sc.frames):
            res = solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, prm, 10,
                                     q0=q0, t0=t0)
            q0, t0 = res.q, res.t
            assert np.abs(futs[s][k].result().pos - res.pos).max() <= POS_TOL_MM, (s, k)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,ftc", [(0, 0), (1, 0), (2, 0), (2, 1), (2, 2), (2, 3)])
def test_admission_estimate_covers_the_librarys_allocations(prec, ftc):
    """The admitter's per-stream estimate (stream_bytes) against the bytes the library reports
    the handle holds (ds_get_device_bytes, its own allocation count) after a full-size frame
    (320x240 template, 256 control points, 2000 matches) is submitted and solved: never below
    it, and within 10 % above it. The device's free memory (cudaMemGetInfo) drops by at least
    the library's count."""
    torch = pytest.importorskip("torch")
    from gpu_common import lib
    from synth import CONFIGS, make_scene
    d = lib()
    sc = make_scene(CONFIGS["seq_320x240_n256"], 1000, n_frames=1)
    f = sc.frames[0]
    M = len(f.match_idx)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, d.default_params(precision=prec,
                                                                      factor_tc=ftc))
    s.submit(f.depth, f.match_idx, f.match_xyz, f.hyp)
    s.solve(10, stats=True)
    actual = d.ds_get_device_bytes(s.h)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    est = stream_bytes(sc.W, sc.H, len(sc.nodes), M, prec)
    s.close()
    assert actual > 0
    assert est >= actual, (est, actual)
    assert est <= 1.10 * actual, (est, actual)
    assert free0 - free1 >= actual, (free0 - free1, actual)


def test_inflight_cap_coalesces_waiting_frames():
    """With at most one batch on the GPU, frames that arrive meanwhile wait and then go out
    together as one larger batch."""
    eng = FakeEngine(delay=2)
    srv = Server(eng, budget_bytes=1 << 40, max_inflight=1)
    for s in "abcd":
        srv.open_stream(s, _spec())
    srv.submit("a", _frame())
    srv.poll()                                   # batch 1: a
    assert len(eng.launches) == 1 and len(srv.in_flight) == 1
    for s in "bcd":
        srv.submit(s, _frame())
    srv.poll()                                   # capped: b, c, d wait
    assert len(eng.launches) == 1
    srv.drain()
    assert len(eng.launches) == 2 and len(eng.launches[1]["ids"]) == 3
    assert srv.stats()["frames"] == 4


def test_frames_beyond_max_matches_are_refused():
    srv = Server(FakeEngine(), budget_bytes=1 << 40)
    srv.open_stream("a", _spec())                    # max_matches = 200
    ok = FrameIn(None, np.zeros(200, np.int32), np.zeros((200, 3), np.float32), None)
    srv.submit("a", ok)
    big = FrameIn(None, np.zeros(201, np.int32), np.zeros((201, 3), np.float32), None)
    with pytest.raises(ValueError):
        srv.submit("a", big)
    srv.drain()
    assert srv.stats()["frames"] == 1


def test_accounting_follows_the_engines_reported_bytes():
    """A stream is counted at the larger of its estimate and the bytes the engine reports it
    holds (the library's own allocation count), after admission and after every submission;
    closing it returns exactly what was counted."""
    class Reporting(FakeEngine):
        extra = 0

        def device_bytes(self, s):
            return stream_bytes(80, 60, 32, 200, 2) + self.extra

    eng = Reporting()
    one = stream_bytes(80, 60, 32, 200, 2)
    srv = Server(eng, budget_bytes=10 * one)
    srv.open_stream("a", _spec())
    assert srv.used == one
    eng.extra = 1000                                  # the library holds more than estimated
    srv.submit("a", _frame())
    srv.poll()
    assert srv.used == one + 1000
    srv.drain()
    srv.close_stream("a")
    assert srv.used == 0


def test_inflight_cap_needs_as_many_engine_batches():
    """A server may not keep more batches on the GPU than its engine has batch slots."""
    eng = FakeEngine()
    eng.n_batches = 2
    Server(eng, budget_bytes=1 << 40, max_inflight=2)
    with pytest.raises(ValueError):
        Server(eng, budget_bytes=1 << 40, max_inflight=3)


def test_full_batch_rate_from_device_times():
    class Timed(FakeEngine):
        def gpu_ms(self, tok):
            return 10.0 * len(tok["ids"])

    eng = Timed(delay=1)
    srv = Server(eng, budget_bytes=1 << 40, max_inflight=1)
    for s in "abc":
        srv.open_stream(s, _spec())
    for s in "abc":
        srv.submit(s, _frame())
    srv.poll()                                   # batch of 3
    srv.drain()
    srv.submit("a", _frame())
    srv.drain()                                  # batch of 1
    fb = srv.stats()["full_batches"]
    assert fb["size"] == 3 and fb["batches"] == 1
    assert fb["frames_per_s_device"] == pytest.approx(3 / 0.030)


def test_next_frame_is_staged_while_the_previous_solves():
    """A stream's next frame is submitted (its copies, preparation and RANSAC start) while its
    previous frame's solve is on the GPU; the solve of the new frame waits for that one, and the
    results come out in order."""
    eng = FakeEngine(delay=3)
    srv = Server(eng, budget_bytes=1 << 40)
    srv.open_stream("a", _spec())
    f1 = srv.submit("a", _frame())
    srv.poll()                                       # staged and launched
    s = srv.streams["a"]["solver"]
    assert s["submitted"] == 1 and s["launched"] == 1
    f2 = srv.submit("a", _frame())
    f3 = srv.submit("a", _frame())
    srv.poll()                                       # frame 2 staged beside the running solve
    assert s["submitted"] == 2 and s["launched"] == 1 and len(eng.launches) == 1
    assert srv.streams["a"]["staged"] is not None and len(srv.streams["a"]["queue"]) == 1
    srv.drain()
    assert [f.result().t[0, 0] for f in (f1, f2, f3)] == [1.0, 2.0, 3.0]
    assert len(eng.launches) == 3


def test_batches_beside_a_running_one_need_min_fill():
    """With a batch on the GPU, a second one is launched only when the ready streams make up at
    least min_fill of the admitted ones; otherwise they wait and go out with the first batch's
    streams as one full batch."""
    eng = FakeEngine(delay=2)
    srv = Server(eng, budget_bytes=1 << 40, max_inflight=2, min_fill=0.6)
    for sid in "abcde":
        srv.open_stream(sid, _spec())
    for sid in "ab":
        srv.submit(sid, _frame())
    srv.poll()                                       # nothing on the GPU: a, b go at once
    assert len(eng.launches) == 1
    for sid in "cd":
        srv.submit(sid, _frame())
    srv.poll()                                       # 2 ready < 0.6 x 5: they wait
    assert len(eng.launches) == 1
    for sid in "ab":
        srv.submit(sid, _frame())
    srv.drain()
    assert len(eng.launches) == 2 and len(eng.launches[1]["ids"]) == 4
    srv2 = Server(FakeEngine(delay=2), budget_bytes=1 << 40, max_inflight=2, min_fill=0.6)
    for sid in "abcde":
        srv2.open_stream(sid, _spec())
    srv2.submit("a", _frame())
    srv2.poll()
    for sid in "bcd":
        srv2.submit(sid, _frame())
    srv2.poll()                                      # 3 ready >= 0.6 x 5: a second batch
    assert len(srv2.in_flight) == 2
    srv2.drain()
    assert srv2.stats()["frames"] == 4


@pytest.mark.parametrize("seed", range(6))
def test_random_schedules_keep_the_slot_discipline_and_order(seed):
    """Random arrivals, batch delays, fill rules and in-flight caps: the fake engine asserts the
    library's slot model on every submission and launch (one frame staged and one in flight per
    stream at most, a solve only over a new frame), every frame completes, and each stream's
    results come out in arrival order."""
    rng = np.random.default_rng(seed)
    eng = FakeEngine(delay=int(rng.integers(1, 5)))
    eng.n_batches = 2
    srv = Server(eng, budget_bytes=1 << 40, max_inflight=int(rng.integers(1, 3)),
                 min_fill=float(rng.choice([0.0, 0.3, 0.6, 1.0])))
    sids = list(range(int(rng.integers(2, 7))))
    for sid in sids:
        srv.open_stream(sid, _spec())
    futs = {sid: [] for sid in sids}
    for _ in range(60):
        for sid in sids:
            if rng.random() < 0.3:
                futs[sid].append(srv.submit(sid, _frame()))
        for _ in range(int(rng.integers(0, 3))):
            srv.poll()
    srv.drain()
    total = 0
    for sid in sids:
        got = [f.result().t[0, 0] for f in futs[sid]]
        assert got == [float(k + 1) for k in range(len(got))]
        total += len(got)
    st = srv.stats()
    assert st["frames"] == total and srv.pending() == 0
    assert all(not s["busy"] and s["staged"] is None for s in srv.streams.values())


def test_drain_refuses_to_spin_on_streams_that_cannot_be_admitted():
    """Frames of a stream that waits for device memory, with nothing on the GPU to free any:
    drain raises instead of polling forever; once a stream is closed the waiting one is admitted
    and its frames complete."""
    one = stream_bytes(80, 60, 32, 200, 2)
    srv = Server(FakeEngine(), budget_bytes=int(1.5 * one))
    srv.open_stream("a", _spec())
    assert not srv.open_stream("b", _spec())
    fa = srv.submit("a", _frame())
    fb = srv.submit("b", _frame())
    with pytest.raises(RuntimeError):
        srv.drain()
    assert fa.done() and not fb.done()
    srv.close_stream("a")
    srv.drain()
    assert fb.result().t[0, 0] == 1.0
