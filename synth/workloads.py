"""Problem lists of the batched and served workloads (inputs only, no solve arithmetic).

Batched workload: 64 independent sequences whose template size is drawn from {160x120,
320x240, 640x480}, whose control-point count is uniform in [64, 1024] and whose outlier rate is
uniform in [20 %, 60 %]. The match count and the deformation follow the single-size workloads of
the same template size (2000 matches and 10 mm at 320x240, 4000 matches and 15 mm at 640x480;
500 matches, the 320x240 count per pixel, and 10 mm at 160x120). Served workload: 32 of those
sequences as streams with Poisson frame arrivals at rates uniform in [15, 60] Hz.

Seeds follow the convention config index x 1000 + stream (batched: 4, served: 5); the draws of
the problem list itself use config index x 10000.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .scene import Config, make_scene

SIZES = [(160, 120), (320, 240), (640, 480)]
MATCHES = {160: 500, 320: 2000, 640: 4000}
AMPLITUDE = {160: 10.0, 320: 10.0, 640: 15.0}


@dataclasses.dataclass
class Problem:
    cfg: Config
    seed: int          # scene seed
    rate_hz: float     # frame arrival rate when served


def mixed_problems(n: int, config_index: int = 4) -> list[Problem]:
    """n problems drawn as the batched workload describes (see the module docstring)."""
    rng = np.random.default_rng(config_index * 10000)
    out = []
    for k in range(n):
        W, H = SIZES[int(rng.integers(0, 3))]
        N = int(rng.integers(64, 1025))
        outlier = float(rng.uniform(0.2, 0.6))
        rate = float(rng.uniform(15.0, 60.0))
        cfg = Config(f"mix{k}_{W}x{H}_n{N}", W, H, N, MATCHES[W], 20, outlier, 0.5, 0.10,
                     AMPLITUDE[W], 1.0, 0.2, 0.5, 300)
        out.append(Problem(cfg, config_index * 1000 + k, rate))
    return out


def _make(args):
    cfg, seed, n_frames = args
    return make_scene(cfg, seed, n_frames=n_frames)


def make_scenes(problems: list[Problem], n_frames: int, processes: int = 1):
    """The scenes of a problem list (n_frames frames each), built in `processes` spawned worker
    processes when processes > 1 (spawned, so a CUDA context of the caller is not inherited)."""
    jobs = [(p.cfg, p.seed, n_frames) for p in problems]
    if processes <= 1:
        return [_make(j) for j in jobs]
    import multiprocessing as mp
    # largest templates first so that the pool's tail is short
    order = sorted(range(len(jobs)), key=lambda i: -jobs[i][0].W * jobs[i][0].H)
    with mp.get_context("spawn").Pool(processes) as pool:
        built = pool.map(_make, [jobs[i] for i in order], chunksize=1)
    out = [None] * len(jobs)
    for i, sc in zip(order, built):
        out[i] = sc
    return out
