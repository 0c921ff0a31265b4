"""The multi-GPU path is replicas only (independent streams per rank, no collective on the data
path): the host logic that combines ranks, run as 2 gloo processes on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(times[rank], world, "cpu")
    from synth.workloads import mixed_problems
    seeds = bench.replica_seeds(rank, mixed_problems(3))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, seeds))


def test_two_replicas_take_the_slowest_rank_and_own_seeds():
    world, port = 2, _free_port()
    times = [1.25, 2.5]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert all(t == max(times) for _, t, _ in out)          # max over ranks
    assert set(out[0][2]).isdisjoint(out[1][2])             # each replica its own streams
    import bench
    assert bench.job_throughput(world, 64 * 20, max(times)) == pytest.approx(2 * 1280 / 2.5)
