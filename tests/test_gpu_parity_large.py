"""GPU parity at the workloads' full sizes, every Gauss-Newton iteration of a frame:

* the 320x240 template / 256 control points / 2000 matches frame in the mixed precision the
  batched benchmark runs (FP32 J^T J and factor, two refinement steps with ~48-bit residuals,
  nearest-pixel association) and in FP64, against one FP64 oracle solve;
* the 640x480 / 1024 control points (6144 unknowns) / 4000 matches frame, 10 iterations, in the
  mixed precision and in FP64;
* a batch of uneven problems drawn like the batched workload (templates 160x120 to 640x480,
  64 to 1024 control points, 20-60 % outliers): every problem against its own oracle solve.

The oracle runs of the larger cases take minutes; they are computed once per module, the mixed
batch's in parallel processes (spawned, so no CUDA state is inherited)."""
import multiprocessing as mp

import numpy as np
import pytest

from gpu_common import (COST_RTOL, POS_TOL_MM, gpu_frame, lib, oracle_params, ransac_listed,
                        scene)
from oracle import solver
from synth import CONFIGS

pytestmark = pytest.mark.gpu


def _oracle_pos_costs(args):
    """Oracle solve of one frame in a worker process: (node positions g, control-point
    positions, costs, RANSAC result)."""
    cfg, seed, prm, iters = args
    sc = scene(cfg, seed)
    fr = sc.frames[0]
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    res = solver.solve_frame(tpl, fr.depth, fr.match_idx, fr.match_xyz, fr.hyp, prm, iters)
    return tpl.g, res.pos, np.array(res.costs), res.ransac


@pytest.fixture(scope="module")
def d():
    return lib()


def _case(name, seed, d):
    sc = scene(CONFIGS[name], seed)
    fr = sc.frames[0]
    prm = oracle_params(d.default_params())
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    res = solver.solve_frame(tpl, fr.depth, fr.match_idx, fr.match_xyz, fr.hyp, prm, 10)
    return sc, tpl, res


@pytest.fixture(scope="module")
def c2(d):
    return _case("seq_320x240_n256", 1000, d)


@pytest.fixture(scope="module")
def c3(d):
    return _case("seq_640x480_n1024", 2000, d)


def _check(d, case, p):
    sc, tpl, res = case
    fr = sc.frames[0]
    s, st, q, t = gpu_frame(d, sc, fr, p, iters=10)
    mask = s.mask()
    listed, _ = ransac_listed(res.ransac, p.H_mm)
    assert np.array_equal(mask[~listed], res.ransac["mask"][~listed])
    err = np.abs(tpl.g + t - res.pos).max()
    assert err <= POS_TOL_MM, err
    rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
    assert rel.max() <= COST_RTOL, rel
    s.close()
    return err, rel.max()


@pytest.mark.parametrize("prec,ftc", [(2, 0), (0, 0), (2, 1), (2, 2), (2, 3), (2, 4), (2, 5),
                                      (2, -1)],
                         ids=["fp32_refine", "fp64", "fp32_refine_tc64", "fp32_refine_tc128",
                              "fp32_refine_tc128q", "fp32_refine_tc128p", "fp32_refine_tc128pipe",
                              "fp32_refine_auto"])
def test_320x240_n256_all_iterations(d, c2, prec, ftc):
    _check(d, c2, d.default_params(precision=prec, factor_tc=ftc))


@pytest.mark.parametrize("prec,ftc", [(2, 0), (0, 0), (2, 1), (2, 2), (2, 3), (2, 4), (2, 5)],
                         ids=["fp32_refine", "fp64", "fp32_refine_tc64", "fp32_refine_tc128",
                              "fp32_refine_tc128q", "fp32_refine_tc128p", "fp32_refine_tc128pipe"])
def test_640x480_n1024_all_iterations(d, c3, prec, ftc):
    _check(d, c3, d.default_params(precision=prec, factor_tc=ftc))


def test_mixed_size_batch_every_problem_matches_oracle(d):
    """Five problems drawn like the batched workload, solved as one batch in the mixed precision
    (10 iterations): each problem's control points within the parity bar of its own oracle solve,
    its RANSAC mask bit-exact outside the listed band."""
    from synth.scene import Config
    rng = np.random.default_rng(64)
    sizes = [(160, 120), (320, 240), (640, 480)]
    cfgs = []
    for k in range(5):
        W, H = sizes[k % 3]
        N = int(rng.integers(64, 1025))
        out = float(rng.uniform(0.2, 0.6))
        M = int(min(4000, W * H // 20))
        cfgs.append(Config(f"mix{k}_{W}x{H}_n{N}", W, H, N, M, 20, out, 0.5, 0.1, 10.0, 1.0,
                           0.2, 0.5, 1))
    p = d.default_params(precision=2)
    prm = oracle_params(p)
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(cfgs)) as pool:
        pending = pool.map_async(_oracle_pos_costs,
                                 [(c, 6400 + k, prm, 10) for k, c in enumerate(cfgs)])
        scenes = [scene(c, 6400 + k) for k, c in enumerate(cfgs)]
        solvers = []
        for sc in scenes:
            s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
            fr = sc.frames[0]
            s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
            solvers.append(s)
        d.ds_solve_batch([s.h for s in solvers], 10)
        got = [(s.deformation64()[1], s.mask()) for s in solvers]
        for s in solvers:
            s.close()
        want = pending.get(timeout=1800)
    for k, ((t, mask), (g, pos, costs, rs)) in enumerate(zip(got, want)):
        err = np.abs(g + t - pos).max()
        assert err <= POS_TOL_MM, (k, cfgs[k].name, err)
        listed, _ = ransac_listed(rs, p.H_mm)
        assert np.array_equal(mask[~listed], rs["mask"][~listed]), (k, cfgs[k].name)
