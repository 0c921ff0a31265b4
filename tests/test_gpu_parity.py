"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs, element by element, at sizes the oracle finishes in seconds (several tiles, ragged
tails) and at the full 320x240 / 256-node size the benchmark times."""
import numpy as np
import pytest

from gpu_common import (BAND_MM, COST_RTOL, MID, POS_TOL_MM, gpu_frame, lib, oracle_params,
                        ransac_listed, scene, unpack_bits)
from oracle import frame as oframe
from oracle import solver
from synth import CONFIGS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def d():
    return lib()


@pytest.fixture(scope="module")
def tiny():
    return scene(CONFIGS["frame_80x60_n32"], 1000)


@pytest.fixture(scope="module")
def mid():
    return scene(MID, 4242)


def _oracle(sc, fr, prm, iters=10, q0=None, t0=None):
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    res = solver.solve_frame(tpl, fr.depth, fr.match_idx, fr.match_xyz, fr.hyp, prm, iters,
                             q0=q0, t0=t0)
    return tpl, res


# ----------------------------------------------------------------------------- set-up tables


@pytest.mark.parametrize("which", ["tiny", "mid"])
def test_blend_table_bit_exact(d, which, tiny, mid):
    sc = tiny if which == "tiny" else mid
    p = d.default_params()
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, oracle_params(p))
    P = d.ds_get_blend_table(s.h)
    pix = np.zeros(P, np.int32)
    nid = np.zeros((P, 4), np.int32)
    al = np.zeros((P, 4), np.float32)
    d.ds_get_blend_table(s.h, pix, nid, al)
    assert np.array_equal(pix, tpl.pidx)
    assert np.array_equal(nid, tpl.nid)          # index work: bit-exact
    assert np.abs(al - tpl.alpha).max() < 1e-6   # FP32 rounding of FP64 weights
    s.close()


def test_frame_points_and_normals(d, mid):
    sc = mid
    fr = sc.frames[0]
    p = d.default_params()
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    pts = np.zeros((sc.H * sc.W, 4), np.float32)
    nrm = np.zeros((sc.H * sc.W, 4), np.float32)
    d.ds_get_frame_points(s.h, pts, nrm)
    X, valid = oframe.backproject(fr.depth, sc.K)
    n, ok = oframe.target_normals(X, valid)
    assert np.array_equal(pts[:, 3] > 0, ok.reshape(-1))
    okf = ok.reshape(-1)
    assert np.abs(pts[okf, :3] - X.reshape(-1, 3)[okf]).max() < 1e-4      # mm
    assert np.abs(nrm[okf, :3] - n.reshape(-1, 3)[okf]).max() < 1e-4
    s.close()


# ----------------------------------------------------------------------------- RANSAC


@pytest.mark.parametrize("which", ["tiny", "mid", "full"])
def test_ransac_mask_bit_exact(d, which, tiny, mid):
    if which == "full":
        sc = scene(CONFIGS["seq_320x240_n256"], 1000)
    else:
        sc = tiny if which == "tiny" else mid
    fr = sc.frames[0]
    p = d.default_params()
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    from oracle import ransac
    X0, _ = oframe.backproject(sc.template_depth, sc.K)
    rs = ransac.ransac_1p(X0.reshape(-1, 3)[fr.match_idx], fr.match_xyz, fr.hyp, p.H_mm,
                          p.n_reweight, p.keep_frac)
    _check_ransac(d, s, p, rs, len(fr.match_idx))
    s.close()


def _check_ransac(d, s, p, rs, M):
    """The handle's last RANSAC against the oracle's: kept references and masks bit-exact outside
    the listed band, scores and weights to rounding."""
    bits = np.zeros((M + 31) // 32, np.uint32)
    d.ds_get_inlier_mask(s.h, bits)
    w = np.zeros(M, np.float32)
    kept = np.zeros(2, np.uint32)
    score = np.zeros(p.n_hyp, np.float64)
    d.ds_get_ransac(s.h, w, kept, score)
    gmask = unpack_bits(bits, M)
    gkept = unpack_bits(kept, p.n_hyp)
    listed, amb = ransac_listed(rs, p.H_mm)
    assert np.array_equal(gkept[~amb], rs["kept"][~amb])
    assert np.array_equal(gmask[~listed], rs["mask"][~listed]), np.flatnonzero(gmask != rs["mask"])
    assert np.abs(score - rs["score"]).max() <= 1e-9 * np.abs(rs["score"]).max()
    assert np.abs(w[~listed] - rs["what"][~listed]).max() < 1e-6
    assert listed.sum() <= max(1, M // 100)


# ----------------------------------------------------------------------------- linearisation


@pytest.mark.parametrize("which", ["tiny", "mid"])
def test_normal_equations_match_oracle(d, which, tiny, mid):
    sc = tiny if which == "tiny" else mid
    fr = sc.frames[0]
    p = d.default_params()
    prm = oracle_params(p)
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    n = 6 * len(sc.nodes)
    A = np.zeros((n, n))
    b = np.zeros(n)
    c3 = np.zeros(3)
    w_arap = d.ds_linearize(s.h, 0.0, A, b, c3)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    tgt = solver.prepare_target(fr.depth, tpl.K)
    from oracle import ransac
    rs = ransac.ransac_1p(tpl.X0[fr.match_idx], fr.match_xyz, fr.hyp, prm.H, prm.n_reweight,
                          prm.keep_frac)
    orb = (fr.match_idx, fr.match_xyz.astype(np.float64), rs["mask"], rs["what"])
    N = len(sc.nodes)
    q = np.tile([1.0, 0, 0, 0], (N, 1))
    t = np.zeros((N, 3))
    lin, wo = solver.linearize(tpl, tgt, q, t, orb, None, prm)
    assert abs(w_arap - wo) <= 1e-5 * wo
    scale = np.abs(lin.A).max()
    assert np.abs(A - lin.A).max() <= 2e-5 * scale, np.abs(A - lin.A).max() / scale
    assert np.abs(b - lin.b).max() <= 2e-5 * np.abs(lin.b).max()
    ref = np.array([lin.cost_icp, lin.cost_orb, lin.cost_arap])
    # relative to the total: the ARAP cost is exactly 0 at the identity, FP32 leaves ~1e-9
    assert np.all(np.abs(c3 - ref) <= COST_RTOL * ref.sum())
    s.close()


# ----------------------------------------------------------------------------- whole solves


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_solve_matches_oracle_tiny(d, tiny, prec):
    sc = tiny
    fr = sc.frames[0]
    p = d.default_params(precision=prec)
    prm = oracle_params(p)
    s, st, q, t = gpu_frame(d, sc, fr, p)
    tpl, res = _oracle(sc, fr, prm)
    pos = tpl.g + t
    err = np.abs(pos - res.pos).max()
    assert err <= POS_TOL_MM, err
    cost = np.array(st.cost[:10])
    rel = np.abs(cost - np.array(res.costs)) / np.array(res.costs)
    assert rel.max() <= COST_RTOL, rel
    assert abs(st.w_arap - res.w_arap) <= 1e-6 * res.w_arap
    s.close()


def test_solve_matches_oracle_mid_ragged(d, mid):
    sc = mid
    fr = sc.frames[0]
    p = d.default_params()
    s, st, q, t = gpu_frame(d, sc, fr, p)
    tpl, res = _oracle(sc, fr, oracle_params(p))
    err = np.abs(tpl.g + t - res.pos).max()
    assert err <= POS_TOL_MM, err
    rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
    assert rel.max() <= COST_RTOL, rel
    s.close()


def test_warm_started_sequence(d):
    """Three consecutive frames, each warm-started from the previous result on both sides."""
    from synth.scene import Config
    cfg = Config("seq_120x90_n40", 120, 90, 40, 300, 8, 0.4, 0.5, 0.1, 8.0, 1.0, 0.3, 0.5, 3)
    sc = scene(cfg, 77, n_frames=3)
    p = d.default_params()
    prm = oracle_params(p)
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    q0 = t0 = None
    for fr in sc.frames:
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
        s.solve(10, stats=False)
        res = solver.solve_frame(tpl, fr.depth, fr.match_idx, fr.match_xyz, fr.hyp, prm, 10,
                                 q0=q0, t0=t0)
        q0, t0 = res.q, res.t
        _, t = s.deformation64()
        assert np.abs(tpl.g + t - res.pos).max() <= POS_TOL_MM
    s.close()


def test_no_matches_frame(d, tiny):
    sc = tiny
    fr = sc.frames[0]
    p = d.default_params()
    prm = oracle_params(p)
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    d.ds_submit_frame(s.h, fr.depth, None, None, 0, None)
    st = d.ds_solve(s.h, 10, True)
    _, t = s.deformation64()
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    res = solver.solve_frame(tpl, fr.depth, np.zeros(0, np.int32), np.zeros((0, 3)), [], prm, 10)
    assert np.abs(tpl.g + t - res.pos).max() <= POS_TOL_MM
    assert st.n_inliers == 0
    s.close()


def test_batch_equals_individual(d, tiny, mid):
    p = d.default_params()
    solvers = []
    for sc in (tiny, mid, tiny):
        s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
        fr = sc.frames[0]
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
        solvers.append(s)
    d.ds_solve_batch([s.h for s in solvers], 10)
    outs = [s.deformation64()[1] for s in solvers]
    for s, sc, o in zip(solvers, (tiny, mid, tiny), outs):
        s2, st, q, t = gpu_frame(d, sc, sc.frames[0], p)
        assert np.abs(o - t).max() <= 1e-4
        s2.close()
        s.close()


# ----------------------------------------------------------------------------- errors


def test_error_codes(d, tiny):
    sc = tiny
    fr = sc.frames[0]
    p = d.default_params()
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    with pytest.raises(d.DsError) as e:
        d.ds_solve(s.h, 10)
    assert e.value.status == d.DS_ERR_STATE
    bad = sc.nodes.copy()
    bad[1] = bad[0]
    with pytest.raises(d.DsError) as e:
        d.ds_set_control_points(s.h, bad)
    assert e.value.status == d.DS_ERR_ARG
    with pytest.raises(d.DsError) as e:
        d.ds_submit_frame(s.h, fr.depth, np.full(len(fr.match_idx), 10 ** 7, np.int32),
                          fr.match_xyz, len(fr.match_idx), fr.hyp)
    assert e.value.status == d.DS_ERR_ARG
    dep = fr.depth.copy()
    dep[3, 3] = np.nan
    d.ds_submit_frame(s.h, dep, fr.match_idx, fr.match_xyz, len(fr.match_idx), fr.hyp)
    with pytest.raises(d.DsError) as e:
        d.ds_solve(s.h, 10, True)
    assert e.value.status == d.DS_ERR_BAD_INPUT
    tdep = sc.template_depth.copy()
    tdep[0, 0] = np.inf
    with pytest.raises(d.DsError) as e:
        d.ds_create_template(tdep, sc.W, sc.H, sc.K)
    assert e.value.status == d.DS_ERR_BAD_INPUT
    s.close()


def test_resume_from_saved_state(d, tiny):
    """get_deformation / set_deformation round trip resumes the same trajectory."""
    sc = tiny
    fr = sc.frames[0]
    p = d.default_params()
    s, st, q, t = gpu_frame(d, sc, fr, p, iters=4)
    qf, tf, _ = s.deformation()
    s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    s.solve(3, stats=False)
    _, ta = s.deformation64()
    s2 = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    d.ds_set_deformation(s2.h, qf, tf)
    s2.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    s2.solve(3, stats=False)
    _, tb = s2.deformation64()
    assert np.abs(ta - tb).max() <= 1e-4
    s.close()
    s2.close()


# ----------------------------------------------------------------------------- batches


def test_batch_of_uneven_problems_matches_oracle(d, tiny, mid):
    """One batch over problems of different template sizes, node counts and match counts: every
    problem's result equals its own oracle solve."""
    from synth.scene import Config
    cfg3 = Config("seq_120x90_n40", 120, 90, 40, 300, 8, 0.4, 0.5, 0.1, 8.0, 1.0, 0.3, 0.5, 1)
    scenes = [tiny, mid, scene(cfg3, 99), tiny]
    p = d.default_params(precision=2)
    solvers = []
    for sc in scenes:
        s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
        fr = sc.frames[0]
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
        solvers.append(s)
    b = d.ds_batch_create([s.h for s in solvers])
    d.ds_batch_solve(b, 10)
    d.ds_batch_status(b)
    for s, sc in zip(solvers, scenes):
        _, t = s.deformation64()
        fr = sc.frames[0]
        tpl, res = _oracle(sc, fr, oracle_params(p))
        assert np.abs(tpl.g + t - res.pos).max() <= POS_TOL_MM
    # a second solve of the same batch (graph replay) on new frames continues from the warm start
    for s, sc in zip(solvers, scenes):
        fr = sc.frames[0]
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    d.ds_batch_solve(b, 3)
    d.ds_batch_status(b)
    d.ds_batch_destroy(b)
    for s in solvers:
        s.close()


def test_batch_result_equals_alone(d, tiny, mid):
    """Each problem's result is the same alone and inside a batch (within the parity
    tolerance; the reduction order of the data-term atomics may differ)."""
    p = d.default_params(precision=2)
    alone = []
    for sc in (tiny, mid):
        s, st, q, t = gpu_frame(d, sc, sc.frames[0], p)
        alone.append(t)
        s.close()
    solvers = []
    for sc in (mid, tiny, mid):
        s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
        fr = sc.frames[0]
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
        solvers.append(s)
    d.ds_solve_batch([s.h for s in solvers], 10)
    outs = [s.deformation64()[1] for s in solvers]
    assert np.abs(outs[0] - alone[1]).max() <= 1e-4
    assert np.abs(outs[1] - alone[0]).max() <= 1e-4
    assert np.abs(outs[2] - alone[1]).max() <= 1e-4
    for s in solvers:
        s.close()


def test_batch_rejects_mixed_precision(d, tiny):
    sc = tiny
    a = d.Solver(sc.template_depth, sc.K, sc.nodes, d.default_params(precision=0))
    b = d.Solver(sc.template_depth, sc.K, sc.nodes, d.default_params(precision=1))
    with pytest.raises(d.DsError) as e:
        d.ds_batch_create([a.h, b.h])
    assert e.value.status == d.DS_ERR_ARG
    a.close()
    b.close()


def test_batch_membership(d, tiny):
    """A handle appears once per batch; new control points or a destroyed handle stop every
    batch that lists it (DS_ERR_STATE) instead of running on stale tables; batches and handles
    may be destroyed in either order."""
    sc, fr = tiny, tiny.frames[0]
    p = d.default_params(precision=2)
    a = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    c = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    for s in (a, c):
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    with pytest.raises(d.DsError) as e:
        d.ds_batch_create([a.h, c.h, a.h])
    assert e.value.status == d.DS_ERR_ARG
    b1 = d.ds_batch_create([a.h, c.h])
    b2 = d.ds_batch_create([c.h])
    d.ds_batch_solve(b1, 2)
    d.ds_batch_status(b1)
    d.ds_set_control_points(a.h, sc.nodes)        # same nodes, new tables: b1 is stale
    with pytest.raises(d.DsError) as e:
        d.ds_batch_solve(b1, 2)
    assert e.value.status == d.DS_ERR_STATE
    d.ds_batch_solve(b2, 2)                       # b2 does not list a
    d.ds_batch_status(b2)
    a.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    a.solve(2, stats=False)                       # a alone still works (its own batch)
    a.deformation64()
    c.close()                                     # destroyed before its batches
    for b in (b1, b2):
        with pytest.raises(d.DsError) as e:
            d.ds_batch_solve(b, 2)
        assert e.value.status == d.DS_ERR_STATE
        d.ds_batch_destroy(b)
    a.close()


def test_bounded_waits_give_up_and_the_context_stays_usable(d, tiny):
    """Failure detection without a GPU fault: a wait on a flag that nothing sets gives up after
    its budget with DS_ERR_TIMEOUT (both wait helpers of the hand-offs between CTAs); with the
    error word already raised by a peer it ends at once; afterwards a frame still solves to the
    oracle."""
    for kind in (0, 1):
        st, ms = d.ds_selftest_bounded_wait(kind, 2_000_000)
        assert st == d.DS_ERR_TIMEOUT
        assert 2.0 <= ms < 1000.0
        st, ms = d.ds_selftest_bounded_wait(kind, 50_000_000, peer_error=1)
        assert st == d.DS_ERR_TIMEOUT
        assert ms < 5.0
    sc, fr = tiny, tiny.frames[0]
    p = d.default_params(precision=2)
    s, st, q, t = gpu_frame(d, sc, fr, p)
    tpl, res = _oracle(sc, fr, oracle_params(p))
    assert np.abs(tpl.g + t - res.pos).max() <= POS_TOL_MM
    s.close()


# ----------------------------------------------------------------------------- tensor-core factor


@pytest.mark.parametrize("ftc", [1, 2, 3, 4, 5],
                         ids=["tiles64", "blocks128", "blocks128q", "blocks128p", "blocks128pipe"])
@pytest.mark.parametrize("prec", [1, 2])
def test_tensor_core_factor_matches_oracle_tiny_and_ragged(d, tiny, mid, prec, ftc):
    """FP32 factorisation on tcgen05 (three TF32 terms per product): the same parity bar, with
    64 x 64 tiles, with 128 x 128 blocks and with the 128-block columns taken in pairs."""
    for sc in (tiny, mid):
        fr = sc.frames[0]
        p = d.default_params(precision=prec, factor_tc=ftc)
        s, st, q, t = gpu_frame(d, sc, fr, p)
        tpl, res = _oracle(sc, fr, oracle_params(p))
        err = np.abs(tpl.g + t - res.pos).max()
        assert err <= POS_TOL_MM, err
        rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
        assert rel.max() <= COST_RTOL, rel
        s.close()


@pytest.mark.parametrize("ftc", [1, 2, 3, 4, 5],
                         ids=["tiles64", "blocks128", "blocks128q", "blocks128p", "blocks128pipe"])
def test_tensor_core_factor_full_size_frame(d, ftc):
    sc = scene(CONFIGS["seq_320x240_n256"], 1000)
    fr = sc.frames[0]
    p = d.default_params(precision=2, factor_tc=ftc)
    s, st, q, t = gpu_frame(d, sc, fr, p)
    tpl, res = _oracle(sc, fr, oracle_params(p))
    err = np.abs(tpl.g + t - res.pos).max()
    assert err <= POS_TOL_MM, err
    rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
    assert rel.max() <= COST_RTOL, rel
    s.close()


def test_tensor_core_factor_batch_equals_simt_and_agreement_rule(d, tiny, mid):
    """An uneven batch factored on the tensor cores gives the SIMT batch's result within the
    parity tolerance; handles that disagree on the factor kernel cannot share a batch."""
    outs = {}
    for ftc in (0, 1, 2, 3, 4, 5):
        p = d.default_params(precision=2, factor_tc=ftc)
        solvers = []
        for sc in (mid, tiny, mid):
            s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
            fr = sc.frames[0]
            s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
            solvers.append(s)
        d.ds_solve_batch([s.h for s in solvers], 10)
        outs[ftc] = [s.deformation64()[1] for s in solvers]
        for s in solvers:
            s.close()
    for ftc in (1, 2, 3, 4, 5):
        for a, b in zip(outs[0], outs[ftc]):
            assert np.abs(a - b).max() <= POS_TOL_MM
    a = d.Solver(tiny.template_depth, tiny.K, tiny.nodes, d.default_params(precision=2))
    b = d.Solver(tiny.template_depth, tiny.K, tiny.nodes,
                 d.default_params(precision=2, factor_tc=1))
    with pytest.raises(d.DsError) as e:
        d.ds_batch_create([a.h, b.h])
    assert e.value.status == d.DS_ERR_ARG
    a.close()
    b.close()


# ----------------------------------------------------------------------------- block-Jacobi solver


@pytest.mark.parametrize("prec", [0, 2])
def test_block_jacobi_matches_oracle(d, tiny, mid, prec):
    """Per-node 6 x 6 solves (Section 2's independent W_i updates): same parity bar."""
    for sc in (tiny, mid):
        fr = sc.frames[0]
        p = d.default_params(precision=prec, solver=1)
        s, st, q, t = gpu_frame(d, sc, fr, p)
        tpl, res = _oracle(sc, fr, oracle_params(p))
        err = np.abs(tpl.g + t - res.pos).max()
        assert err <= POS_TOL_MM, err
        rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
        assert rel.max() <= COST_RTOL, rel
        s.close()


def test_block_jacobi_full_size_frame_and_batch_rule(d, tiny):
    sc = scene(CONFIGS["seq_320x240_n256"], 1000)
    fr = sc.frames[0]
    p = d.default_params(precision=2, solver=1)
    s, st, q, t = gpu_frame(d, sc, fr, p)
    tpl, res = _oracle(sc, fr, oracle_params(p))
    assert np.abs(tpl.g + t - res.pos).max() <= POS_TOL_MM
    rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
    assert rel.max() <= COST_RTOL, rel
    s.close()
    a = d.Solver(tiny.template_depth, tiny.K, tiny.nodes, d.default_params(precision=2))
    b = d.Solver(tiny.template_depth, tiny.K, tiny.nodes, d.default_params(precision=2, solver=1))
    with pytest.raises(d.DsError) as e:
        d.ds_batch_create([a.h, b.h])
    assert e.value.status == d.DS_ERR_ARG
    a.close()
    b.close()


# ----------------------------------------------------------------------------- largest sizes


@pytest.mark.gpu
def test_mixed_size_batch():
    """Batched uneven solves as in the batched workload: templates drawn from 160x120, 320x240
    and 640x480, control points uniform in [64, 1024], outlier rates uniform in [20 %, 60 %];
    one batch equals every problem solved alone, and the smallest problem equals the oracle."""
    from gpu_common import lib
    from synth.scene import Config
    d = lib()
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
    scenes = [scene(c, 6400 + k) for k, c in enumerate(cfgs)]
    p = d.default_params(precision=2)
    alone = []
    for sc in scenes:
        s, st, q, t = gpu_frame(d, sc, sc.frames[0], p)
        alone.append(t)
        s.close()
    solvers = []
    for sc in scenes:
        s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
        fr = sc.frames[0]
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
        solvers.append(s)
    d.ds_solve_batch([s.h for s in solvers], 10)
    for s, t in zip(solvers, alone):
        assert np.abs(s.deformation64()[1] - t).max() <= 1e-4
        s.close()
    k = int(np.argmin([c.W * c.H * c.N for c in cfgs]))
    sc = scenes[k]
    tpl, res = _oracle(sc, sc.frames[0], oracle_params(p))
    assert np.abs(tpl.g + alone[k] - res.pos).max() <= POS_TOL_MM


# ----------------------------------------------------------------------------- association and RANSAC variants


@pytest.mark.parametrize("prec", [0, 2])
def test_bilinear_association_matches_oracle(d, tiny, mid, prec):
    """ICP with the target point and normal blended from the 4 pixels around the projection."""
    for sc in (tiny, mid):
        fr = sc.frames[0]
        p = d.default_params(precision=prec, assoc=1)
        s, st, q, t = gpu_frame(d, sc, fr, p)
        tpl, res = _oracle(sc, fr, oracle_params(p))
        err = np.abs(tpl.g + t - res.pos).max()
        assert err <= POS_TOL_MM, err
        rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
        assert rel.max() <= COST_RTOL, rel
        assert abs(st.w_arap - res.w_arap) <= 1e-6 * res.w_arap
        s.close()


def test_bilinear_normal_equations_match_oracle(d, mid):
    sc = mid
    fr = sc.frames[0]
    p = d.default_params(assoc=1)
    prm = oracle_params(p)
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    n = 6 * len(sc.nodes)
    A = np.zeros((n, n))
    b = np.zeros(n)
    c3 = np.zeros(3)
    w_arap = d.ds_linearize(s.h, 0.0, A, b, c3)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    tgt = solver.prepare_target(fr.depth, tpl.K)
    from oracle import ransac
    rs = ransac.ransac_1p(tpl.X0[fr.match_idx], fr.match_xyz, fr.hyp, prm.H, prm.n_reweight,
                          prm.keep_frac)
    orb = (fr.match_idx, fr.match_xyz.astype(np.float64), rs["mask"], rs["what"])
    N = len(sc.nodes)
    lin, wo = solver.linearize(tpl, tgt, np.tile([1.0, 0, 0, 0], (N, 1)), np.zeros((N, 3)), orb,
                               None, prm)
    assert abs(w_arap - wo) <= 1e-5 * wo
    scale = np.abs(lin.A).max()
    assert np.abs(A - lin.A).max() <= 2e-5 * scale, np.abs(A - lin.A).max() / scale
    assert np.abs(b - lin.b).max() <= 2e-5 * np.abs(lin.b).max()
    s.close()


def test_bilinear_association_full_size_frame(d):
    sc = scene(CONFIGS["seq_320x240_n256"], 1000)
    fr = sc.frames[0]
    p = d.default_params(precision=2, assoc=1)
    s, st, q, t = gpu_frame(d, sc, fr, p)
    tpl, res = _oracle(sc, fr, oracle_params(p))
    assert np.abs(tpl.g + t - res.pos).max() <= POS_TOL_MM
    rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
    assert rel.max() <= COST_RTOL, rel
    s.close()


@pytest.mark.parametrize("which", ["tiny", "full"])
def test_warm_start_ransac_bit_exact(d, which, tiny):
    """RANSAC o1 = the template points warped by the handle's current state (FP64 on both
    sides): the state is set through the ABI, read back in FP64 and given to the oracle."""
    sc = tiny if which == "tiny" else scene(CONFIGS["seq_320x240_n256"], 1000)
    fr = sc.frames[0]
    p = d.default_params(ransac_o1=1)
    prm = oracle_params(p)
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    rng = np.random.default_rng(5)
    N = len(sc.nodes)
    from oracle.quat import qexp_half
    ax = rng.normal(size=(N, 3))
    q = qexp_half(ax / np.linalg.norm(ax, axis=1, keepdims=True) * rng.uniform(0, 0.1, (N, 1)))
    t = rng.normal(scale=1.5, size=(N, 3))
    d.ds_set_deformation(s.h, q.astype(np.float32), t.astype(np.float32))
    q64, t64 = s.deformation64()
    s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    from oracle import ransac
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    o1 = solver.ransac_o1(tpl, fr.match_idx, q64, t64, prm)
    assert np.abs(o1 - tpl.X0[fr.match_idx]).max() > 1.0     # the warm start moved the points
    rs = ransac.ransac_1p(o1, fr.match_xyz, fr.hyp, p.H_mm, p.n_reweight, p.keep_frac)
    _check_ransac(d, s, p, rs, len(fr.match_idx))
    s.close()


def test_warm_started_sequence_with_both_variants(d):
    """Three consecutive frames with bilinear association and warm-start RANSAC; each frame of
    the oracle starts from the state the CUDA path starts from (read back in FP64)."""
    from synth.scene import Config
    cfg = Config("seq_120x90_n40", 120, 90, 40, 300, 8, 0.4, 0.5, 0.1, 8.0, 1.0, 0.3, 0.5, 3)
    sc = scene(cfg, 77, n_frames=3)
    p = d.default_params(precision=2, assoc=1, ransac_o1=1)
    prm = oracle_params(p)
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    for fr in sc.frames:
        q0, t0 = s.deformation64()
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
        st = s.solve(10, stats=True)
        res = solver.solve_frame(tpl, fr.depth, fr.match_idx, fr.match_xyz, fr.hyp, prm, 10,
                                 q0=q0, t0=t0)
        _check_ransac(d, s, p, res.ransac, len(fr.match_idx))
        _, t = s.deformation64()
        assert np.abs(tpl.g + t - res.pos).max() <= POS_TOL_MM
        rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
        assert rel.max() <= COST_RTOL, rel
    s.close()


def test_batch_mixes_association_variants(d, tiny, mid):
    """Handles of one batch may use different associations; each result equals its own solve."""
    ps = [d.default_params(precision=2, assoc=a) for a in (1, 0, 1)]
    scs = (tiny, mid, mid)
    solvers = []
    for sc, p in zip(scs, ps):
        s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
        fr = sc.frames[0]
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
        solvers.append(s)
    d.ds_solve_batch([s.h for s in solvers], 10)
    outs = [s.deformation64()[1] for s in solvers]
    for sc, p, o in zip(scs, ps, outs):
        s2, st, q, t = gpu_frame(d, sc, sc.frames[0], p)
        assert np.abs(o - t).max() <= 1e-4
        s2.close()
    assert np.abs(outs[1] - outs[2]).max() > 1e-6      # the two associations differ
    for s in solvers:
        s.close()


# ----------------------------------------------------------------------------- pipelined frames


def test_pipelined_batch_frames_match_sequential(d):
    """Each handle keeps two frame slots: frame k + 1 is submitted (prepared, RANSAC) while the
    batch still solves frame k, with no host synchronisation; the results equal solving each
    frame after the previous one finished, and the getters return the latest frame's RANSAC."""
    from synth.scene import Config
    cfg = Config("seq_120x90_n40", 120, 90, 40, 300, 8, 0.4, 0.5, 0.1, 8.0, 1.0, 0.3, 0.5, 3)
    scs = [scene(cfg, 91 + j, n_frames=3) for j in range(3)]
    p = d.default_params(precision=2)
    seq, seq_masks = [], []
    for sc in scs:
        s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
        for fr in sc.frames:
            s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
            s.solve(10, stats=False)
            s.deformation64()                       # synchronises
        seq.append(s.deformation64()[1])
        seq_masks.append(s.mask())
        s.close()
    solvers = [d.Solver(sc.template_depth, sc.K, sc.nodes, p) for sc in scs]
    b = d.ds_batch_create([s.h for s in solvers])
    for k in range(3):
        for s, sc in zip(solvers, scs):
            fr = sc.frames[k]
            s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
        d.ds_batch_solve(b, 10)
        if k == 1:
            # frame 2 submitted while frame 1 solves: its RANSAC is what the getters return
            fr = scs[0].frames[2]
            solvers[0].submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
            ref = d.Solver(scs[0].template_depth, scs[0].K, scs[0].nodes, p)
            ref.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
            assert np.array_equal(solvers[0].mask(), ref.mask())
            ref.close()
            # and the earlier frame the batch is solving is not disturbed: resubmit frame 1 so
            # that the next batch solve sees the same sequence as the sequential run
            fr = scs[0].frames[1]
            solvers[0].submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    d.ds_batch_status(b)
    for s, t_seq, m_seq in zip(solvers, seq, seq_masks):
        _, t = s.deformation64()
        assert np.abs(t - t_seq).max() <= 1e-4
        assert np.array_equal(s.mask(), m_seq)
    d.ds_batch_destroy(b)
    for s in solvers:
        s.close()


def test_ransac_degenerate_fit_is_the_identity(d, tiny):
    """Every match on the same template pixel: S1 = 0 for every reference, M = sum w S2 S1^T = 0,
    and both sides take R = I (Horn's matrix vanishes; the oracle's SVD has no singular value
    above zero), so d_k = |S2(k)| decides each mask bit."""
    sc = tiny
    fr = sc.frames[0]
    rng = np.random.default_rng(12)
    j = int(sc.nodes[3])
    M = 60
    midx = np.full(M, j, np.int32)
    X0, _ = oframe.backproject(sc.template_depth, sc.K)
    o1 = X0.reshape(-1, 3)[midx]
    off = rng.normal(size=(M, 3))
    off *= rng.uniform(0.0, 6.0, (M, 1)) / np.linalg.norm(off, axis=1, keepdims=True)
    xyz = (o1 + off).astype(np.float32)
    hyp = rng.choice(M, size=30, replace=False).astype(np.int32)
    p = d.default_params()
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    s.submit(fr.depth, midx, xyz, hyp)
    from oracle import ransac
    rs = ransac.ransac_1p(o1, xyz, hyp, p.H_mm, p.n_reweight, p.keep_frac)
    assert np.array_equal(ransac.kabsch(o1 - o1[0], xyz - xyz[0], np.ones(M)), np.eye(3))
    assert rs["mask"].any() and not rs["mask"].all()
    _check_ransac(d, s, p, rs, M)
    s.close()


# ----------------------------------------------------------------------------- factor-kernel tuner


def test_factor_tuner_picks_the_fastest_and_auto_batches_stay_at_parity(d, tiny, mid):
    """ds_batch_tune times the three FP32 factor kernels on the batch's sizes and keeps the
    fastest; a batch of DS_FACTOR_AUTO handles tunes itself (or takes the cached choice) at its
    first solve, and its results equal the SIMT batch's and the oracle within the parity bar."""
    from synth.scene import Config
    cfg3 = Config("seq_120x90_n40", 120, 90, 40, 300, 8, 0.4, 0.5, 0.1, 8.0, 1.0, 0.3, 0.5, 1)
    scenes = [mid, tiny, scene(cfg3, 99)]
    outs = {}
    for ftc in (0, d.DS_FACTOR_AUTO):
        p = d.default_params(precision=2, factor_tc=ftc)
        solvers = []
        for sc in scenes:
            s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
            fr = sc.frames[0]
            s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
            solvers.append(s)
        b = d.ds_batch_create([s.h for s in solvers])
        if ftc == d.DS_FACTOR_AUTO:
            choice, ms = d.ds_batch_tune(b, 2)
            assert choice in range(6) and (ms > 0).all()
            assert ms[choice] == ms.min()
            assert d.ds_batch_factor_kernel(b)[0] == choice
        d.ds_batch_solve(b, 10)
        d.ds_batch_status(b)
        outs[ftc] = [s.deformation64()[1] for s in solvers]
        d.ds_batch_destroy(b)
        for s in solvers:
            s.close()
    for a, c in zip(outs[0], outs[d.DS_FACTOR_AUTO]):
        assert np.abs(a - c).max() <= POS_TOL_MM
    sc = scenes[0]
    tpl, res = _oracle(sc, sc.frames[0], oracle_params(d.default_params(precision=2)))
    assert np.abs(tpl.g + outs[d.DS_FACTOR_AUTO][0] - res.pos).max() <= POS_TOL_MM
    # an auto handle solving alone tunes its batch of one at the first solve
    s, st, q, t = gpu_frame(d, sc, sc.frames[0],
                            d.default_params(precision=2, factor_tc=d.DS_FACTOR_AUTO))
    assert np.abs(tpl.g + t - res.pos).max() <= POS_TOL_MM
    s.close()


def test_masked_batch_solves_only_the_active_handles(d, tiny, mid):
    """ds_batch_solve_masked: the active handles get the same result as solved alone, a handle
    left out keeps its state untouched (even with a newer frame submitted), and the same batch
    (and captured graph) then serves the complementary mask; two batches over the same handles
    run disjoint masks in flight at once."""
    from synth.scene import Config
    cfg3 = Config("seq_120x90_n40", 120, 90, 40, 300, 8, 0.4, 0.5, 0.1, 8.0, 1.0, 0.3, 0.5, 1)
    scenes = [tiny, mid, scene(cfg3, 99)]
    p = d.default_params(precision=2)
    alone = []
    for sc in scenes:
        s, st, q, t = gpu_frame(d, sc, sc.frames[0], p)
        alone.append(t)
        s.close()
    solvers = []
    for sc in scenes:
        s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
        fr = sc.frames[0]
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
        solvers.append(s)
    b = d.ds_batch_create([s.h for s in solvers])
    d.ds_batch_solve_masked(b, [1, 0, 1], 10)
    d.ds_batch_status(b)
    assert np.abs(solvers[0].deformation64()[1] - alone[0]).max() <= 1e-4
    assert np.abs(solvers[2].deformation64()[1] - alone[2]).max() <= 1e-4
    assert np.abs(solvers[1].deformation64()[1]).max() == 0.0      # untouched: identity
    d.ds_batch_solve_masked(b, [0, 1, 0], 10)
    d.ds_batch_status(b)
    assert np.abs(solvers[1].deformation64()[1] - alone[1]).max() <= 1e-4
    with pytest.raises(d.DsError) as e:
        d.ds_batch_solve_masked(b, [0, 0, 0], 10)
    assert e.value.status == d.DS_ERR_ARG
    # two batches over the same handles, disjoint masks in flight together (fresh states)
    b2 = d.ds_batch_create([s.h for s in solvers])
    for s, sc in zip(solvers, scenes):
        N = len(sc.nodes)
        d.ds_set_deformation(s.h, np.tile(np.float32([1, 0, 0, 0]), (N, 1)),
                             np.zeros((N, 3), np.float32))
        fr = sc.frames[0]
        s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    d.ds_batch_solve_masked(b, [1, 1, 0], 10)
    d.ds_batch_solve_masked(b2, [0, 0, 1], 10)
    d.ds_batch_status(b)
    d.ds_batch_status(b2)
    for s, t in zip(solvers, alone):
        assert np.abs(s.deformation64()[1] - t).max() <= 1e-4
    d.ds_batch_destroy(b)
    d.ds_batch_destroy(b2)
    for s in solvers:
        s.close()
