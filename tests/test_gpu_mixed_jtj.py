"""The mixed-precision ICP term: J^T W J from BF16 Jacobian rows on the tensor cores with FP32
accumulation (ds_params.jtj = 1), the gradient J^T W r in FP32.

Bounds: each Jacobian entry rounded to BF16 (unit roundoff u = 2^-8) moves a product of two
entries by at most 2u of its size, so an entry (a, b) of the data-term J^T W J moves by at most
2u sum_p |J_pa| |J_pb| <= 2u sqrt(A_aa A_bb) (Cauchy-Schwarz over the points), i.e. 2^-7 of the
largest diagonal entry; the gradient is unchanged (FP32). The Gauss-Newton fixed point is then
the FP64 oracle's, and the control points after 10 iterations are held to the parity bar."""
import numpy as np
import pytest

from gpu_common import (COST_RTOL, MID, POS_TOL_MM, gpu_frame, lib, oracle_params, scene)
from oracle import ransac, solver
from synth import CONFIGS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def d():
    return lib()


@pytest.mark.parametrize("which", ["tiny", "mid"])
def test_bf16_normal_equations_within_their_bound(d, which):
    sc = scene(CONFIGS["frame_80x60_n32"], 1000) if which == "tiny" else scene(MID, 4242)
    fr = sc.frames[0]
    p = d.default_params(jtj=1)
    prm = oracle_params(p)
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    n = 6 * len(sc.nodes)
    A = np.zeros((n, n))
    b = np.zeros(n)
    c3 = np.zeros(3)
    w_arap = d.ds_linearize(s.h, 0.0, A, b, c3)
    s.close()
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    tgt = solver.prepare_target(fr.depth, tpl.K)
    rs = ransac.ransac_1p(tpl.X0[fr.match_idx], fr.match_xyz, fr.hyp, prm.H, prm.n_reweight,
                          prm.keep_frac)
    orb = (fr.match_idx, fr.match_xyz.astype(np.float64), rs["mask"], rs["what"])
    N = len(sc.nodes)
    lin, wo = solver.linearize(tpl, tgt, np.tile([1.0, 0, 0, 0], (N, 1)), np.zeros((N, 3)),
                               orb, None, prm)
    assert abs(w_arap - wo) <= 1e-5 * wo
    scale = np.abs(lin.A).max()
    dev = np.abs(A - lin.A).max() / scale
    assert dev <= 2.0 ** -7 + 2e-5, dev
    assert dev > 0.0                                   # the BF16 path did run
    assert np.abs(b - lin.b).max() <= 2e-5 * np.abs(lin.b).max()


@pytest.mark.parametrize("prec", [0, 2])
def test_bf16_jtj_solve_matches_oracle(d, prec):
    """Tiny and ragged frames, 10 iterations: control points within the parity bar, the cost at
    each linearisation within the parity tolerance."""
    for sc in (scene(CONFIGS["frame_80x60_n32"], 1000), scene(MID, 4242)):
        fr = sc.frames[0]
        p = d.default_params(precision=prec, jtj=1)
        s, st, q, t = gpu_frame(d, sc, fr, p)
        tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, oracle_params(p))
        res = solver.solve_frame(tpl, fr.depth, fr.match_idx, fr.match_xyz, fr.hyp,
                                 oracle_params(p), 10)
        err = np.abs(tpl.g + t - res.pos).max()
        assert err <= POS_TOL_MM, err
        rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
        assert rel[-1] <= COST_RTOL, rel
        s.close()


def test_batch_rejects_mixed_jtj(d):
    sc = scene(CONFIGS["frame_80x60_n32"], 1000)
    a = d.Solver(sc.template_depth, sc.K, sc.nodes, d.default_params(precision=2))
    b = d.Solver(sc.template_depth, sc.K, sc.nodes, d.default_params(precision=2, jtj=1))
    with pytest.raises(d.DsError) as e:
        d.ds_batch_create([a.h, b.h])
    assert e.value.status == d.DS_ERR_ARG
    a.close()
    b.close()
