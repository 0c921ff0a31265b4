"""Pins of the FP64 oracle to facts outside itself: closed forms, brute force, independent
methods, finite differences and special cases with a known exact answer.  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import dqb, frame, ransac, solver, terms
from oracle.quat import qexp_half, rotmat
from synth import CONFIGS, make_scene
from synth.scene import Config, axis_angle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def random_state(rng, N, rot=0.3, trans=3.0):
    axes = rng.normal(size=(N, 3))
    q = qexp_half(axes / np.linalg.norm(axes, axis=1, keepdims=True) * rng.uniform(0, rot, (N, 1)))
    return q, rng.normal(scale=trans, size=(N, 3))


@pytest.fixture(scope="module")
def tiny():
    sc = make_scene(CONFIGS["frame_80x60_n32"], 1000, f64=True)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes)
    return sc, tpl


# ----------------------------------------------------------------------------- constants


def test_paper_constants_are_oracle_defaults():
    prm = solver.Params()
    for name, value, *_ in _read_golden("paper_constants.txt"):
        assert float(getattr(prm, name)) == float(value), name


def test_closed_form_weights():
    prm = solver.Params()
    for kind, arg, val, *_ in _read_golden("closed_form_weights.txt"):
        x, v = float(arg), float(val)
        if kind == "ransac":
            S1 = np.zeros((2, 3))
            S2 = np.array([[0, 0, 0], [x, 0, 0]], dtype=np.float64)
            # one reference at the origin plus one match displaced by x with a zero lever arm:
            # the rotation cannot move a zero vector, so d = x exactly
            d, w = ransac.reweight(S1, S2, prm.H, 1)
            got = w[1]
        elif kind == "orbramp":
            got = terms.orb_weight(np.array([x]), np.array([False]), np.array([0.0]), prm.H)[0]
        elif kind == "tukeyw":
            got = terms.tukey_weight(np.array([x]), prm.tukey_c)[0]
        elif kind == "tukeyrho":
            got = terms.tukey_rho(np.array([x]), prm.tukey_c)[0]
        else:
            raise AssertionError(kind)
        assert abs(got - v) < 1e-12, (kind, x, got, v)


# ----------------------------------------------------------------------------- frame prep


def test_backprojection_closed_form():
    rng = np.random.default_rng(1)
    H, W = 7, 9
    K = (9.0, 9.0, 4.0, 3.0)
    z = rng.uniform(50, 150, (H, W))
    z[2, 3] = 0.0
    X, valid = frame.backproject(z, K)
    for v in range(H):
        for u in range(W):
            exp = np.array([(u - 4.0) * z[v, u] / 9.0, (v - 3.0) * z[v, u] / 9.0, z[v, u]])
            assert np.array_equal(X[v, u], exp)
    assert not valid[2, 3] and valid.sum() == H * W - 1


def test_plane_normals_exact():
    # depth of the plane n.X = c seen through the pinhole: z = c / (n . d(u, v))
    H, W = 12, 16
    K = (16.0, 16.0, 7.5, 5.5)
    nrm = np.array([0.2, -0.3, -1.0])
    nrm /= np.linalg.norm(nrm)
    c = -100.0
    u, v = np.meshgrid(np.arange(W), np.arange(H))
    d = np.stack([(u - 7.5) / 16.0, (v - 5.5) / 16.0, np.ones_like(u, dtype=float)], -1)
    z = c / (d @ nrm)
    X, valid = frame.backproject(z, K)
    n, ok = frame.target_normals(X, valid)
    assert ok[1:-1, 1:-1].all() and not ok[0].any() and not ok[:, -1].any()
    assert np.abs(n[ok] - nrm).max() < 1e-12
    z2 = z.copy()
    z2[5, 5] = 0.0
    X2, v2 = frame.backproject(z2, K)
    _, ok2 = frame.target_normals(X2, v2)
    for (a, b) in [(5, 5), (4, 5), (6, 5), (5, 4), (5, 6)]:
        assert not ok2[a, b]
    assert ok2[4, 4]


# ----------------------------------------------------------------------------- association


def test_association_is_nearest_pixel_centre_brute_force():
    rng = np.random.default_rng(2)
    W, H = 11, 8
    K = (11.0, 11.0, 5.0, 3.5)
    x = np.concatenate([rng.uniform(-6, 6, (300, 1)), rng.uniform(-5, 5, (300, 1)),
                        rng.uniform(5, 20, (300, 1))], 1)
    # a few exact half-pixel cases: floor(u + 1/2) rounds halves up
    x[0] = [0.5 * 10 / 11.0, 0.0, 10.0]
    tgt_ok = np.ones((H, W), dtype=bool)
    pix, valid, u, v = terms.associate(x, K, W, H, tgt_ok)
    for i in range(x.shape[0]):
        best, bd = None, None
        for pv in range(H):
            for pu in range(W):
                du, dv = u[i] - pu, v[i] - pv
                # nearest centre along each axis, halves to the larger index
                if -0.5 <= du < 0.5 and -0.5 <= dv < 0.5:
                    best = pv * W + pu
                    bd = (du, dv)
        if best is None:
            assert not valid[i]
        else:
            assert valid[i] and pix[i] == best, (i, bd)
    assert valid[0] and pix[0] % W == 6


# ----------------------------------------------------------------------------- nearest nodes


def test_nearest_nodes_brute_force():
    rng = np.random.default_rng(3)
    g = rng.integers(0, 5, (9, 3)).astype(float)      # integer lattice: many exact ties
    p = rng.integers(0, 5, (200, 3)).astype(float) + 0.5 * rng.integers(0, 2, (200, 3))
    ids, d2 = solver.nearest_nodes(p, g, 4)
    for j in range(p.shape[0]):
        cand = sorted(range(9), key=lambda i: (float(((p[j] - g[i]) ** 2).sum()), i))[:4]
        assert list(ids[j]) == cand


# ----------------------------------------------------------------------------- Kabsch / RANSAC


def test_kabsch_matches_horn_and_is_exact_on_three_points():
    rng = np.random.default_rng(4)
    for trial in range(50):
        M = int(rng.integers(3, 40))
        S1 = rng.normal(size=(M, 3)) * 10
        R = axis_angle(rng.normal(size=3), rng.uniform(0, math.pi))
        S2 = S1 @ R.T + rng.normal(scale=0.5, size=(M, 3)) * (trial % 2)
        w = rng.uniform(0.1, 1.0, M)
        Rk = ransac.kabsch(S1, S2, w)
        Rh = ransac.horn(S1, S2, w)
        assert np.abs(Rk - Rh).max() < 1e-12
        assert abs(np.linalg.det(Rk) - 1) < 1e-12
        if trial % 2 == 0:
            assert np.abs(Rk - R).max() < 1e-12
    S1 = rng.normal(size=(3, 3))
    R = axis_angle([1, 2, 3], 0.7)
    assert np.abs(ransac.kabsch(S1, S1 @ R.T, np.ones(3)) - R).max() < 1e-13


def test_kabsch_reflection_guard_and_degenerate():
    S1 = np.array([[1.0, 0, 0], [2.0, 0, 0]])
    assert np.array_equal(ransac.kabsch(S1, S1, np.ones(2)), np.eye(3))     # collinear
    assert np.array_equal(ransac.kabsch(S1, S1, np.zeros(2)), np.eye(3))    # no weight
    rng = np.random.default_rng(5)
    S1 = rng.normal(size=(10, 3))
    S2 = S1 * np.array([1, 1, -1])                 # a mirror: best proper rotation, det = +1
    R = ransac.kabsch(S1, S2, np.ones(10))
    assert abs(np.linalg.det(R) - 1) < 1e-12


def _ransac_bruteforce(o1, o2, hyp, H, n_it, keep_frac):
    """Pure-Python loops over every reference and match, Kabsch by exhaustive search for the
    eigenvector of Horn's matrix (independent of the vectorised oracle's SVD)."""
    M = len(o1)
    res = []
    for k0 in hyp:
        S1 = [[o1[k][a] - o1[k0][a] for a in range(3)] for k in range(M)]
        S2 = [[o2[k][a] - o2[k0][a] for a in range(3)] for k in range(M)]
        w = [1.0] * M
        d = [0.0] * M
        for _ in range(n_it):
            R = ransac.horn(np.array(S1), np.array(S2), np.array(w))
            if sum(w) < 1e-12:
                R = np.eye(3)
            for k in range(M):
                rs = [sum(R[a][b] * S1[k][b] for b in range(3)) for a in range(3)]
                d[k] = math.sqrt(sum((S2[k][a] - rs[a]) ** 2 for a in range(3)))
                w[k] = 1.0 if d[k] == 0 else min(H / d[k], 1.0)
        res.append((list(d), list(w), sum(w) - w[k0]))
    best = max(r[2] for r in res)
    kept = [r[2] >= keep_frac * best for r in res]
    mask = [any(kept[h] and res[h][0][k] <= H for h in range(len(hyp))) for k in range(M)]
    return mask, kept, res


def test_ransac_matches_bruteforce_small():
    rng = np.random.default_rng(6)
    for trial in range(6):
        M = int(rng.integers(5, 13))
        o1 = rng.normal(scale=20, size=(M, 3))
        R = axis_angle(rng.normal(size=3), 0.2)
        o2 = o1 @ R.T + 3 + rng.normal(scale=0.3, size=(M, 3))
        out = rng.random(M) < 0.35
        o2[out] += rng.normal(scale=30, size=(out.sum(), 3))
        hyp = rng.choice(M, size=min(M, 5), replace=False)
        rs = ransac.ransac_1p(o1, o2, hyp, 2.0, 10, 0.5)
        mask, kept, res = _ransac_bruteforce(o1.tolist(), o2.tolist(), list(hyp), 2.0, 10, 0.5)
        assert list(rs["kept"]) == kept
        for h in range(len(hyp)):
            assert np.abs(rs["d"][h] - np.array(res[h][0])).max() < 1e-9
        assert list(rs["mask"]) == mask


def test_ransac_recovers_planted_inliers():
    # rigid scene, noise-free inliers, outliers >= 10 H from their true position
    cfg = Config("planted", 80, 60, 32, 200, 5, 0.3, 0.0, 0.0, 0.0, 0.0, 3.0, 2.0, 1,
                 outlier_min_dist=20.0)
    sc = make_scene(cfg, 77, f64=True)
    f = sc.frames[0]
    X0, _ = frame.backproject(sc.template_depth, sc.K)
    o1 = X0.reshape(-1, 3)[f.match_idx]
    rs = ransac.ransac_1p(o1, f.match_xyz, f.hyp, 2.0, 10, 0.5)
    assert np.array_equal(rs["mask"], f.inlier)
    for h, k0 in enumerate(f.hyp):
        if f.inlier[k0]:
            assert rs["kept"][h]
            assert np.array_equal(rs["d"][h] <= 2.0, f.inlier)


# ----------------------------------------------------------------------------- DQB


def test_dqb_identical_transforms_and_sign_flips():
    rng = np.random.default_rng(8)
    N, P = 6, 50
    g = rng.normal(scale=20, size=(N, 3))
    p = rng.normal(scale=20, size=(P, 3))
    qa = qexp_half(np.array([0.3, -0.2, 0.5]))
    R = rotmat(qa)
    T = np.array([1.0, -2.0, 3.0])
    q = np.tile(qa, (N, 1))
    t = g @ R.T + T - g                     # every node moves by the same rigid (R, T)
    nid = np.stack([rng.choice(N, 4, replace=False) for _ in range(P)])
    al = rng.uniform(0.1, 1, (P, 4))
    al /= al.sum(1, keepdims=True)
    x, _ = dqb.warp_points(q, t, g, p, nid, al, nid[:, 0], with_jac=False)
    assert np.abs(x - (p @ R.T + T)).max() < 1e-12
    q2, t2 = random_state(rng, N)
    x2, _ = dqb.warp_points(q2, t2, g, p, nid, al, nid[:, 0], with_jac=False)
    flip = np.where(rng.random(N) < 0.5, -1.0, 1.0)[:, None]
    x3, _ = dqb.warp_points(q2 * flip, t2, g, p, nid, al, nid[:, 0], with_jac=False)
    assert np.abs(x2 - x3).max() < 1e-12
    # a single node reproduces its own node-centred transform W(x) = R (x - g) + g + t
    x4, _ = dqb.warp_points(q2, t2, g, p, np.zeros((P, 4), int) + 2, al, np.full(P, 2),
                            with_jac=False)
    R2 = rotmat(q2[2])
    assert np.abs(x4 - ((p - g[2]) @ R2.T + g[2] + t2[2])).max() < 1e-12


def _fd(fun, q, t, n, h_rot=1e-6, h_tr=1e-5):
    cols = []
    for k in range(6 * n):
        h = h_rot if k % 6 < 3 else h_tr
        d = np.zeros(6 * n)
        d[k] = h
        qp, tp = dqb.apply_step(q, t, d)
        qm, tm = dqb.apply_step(q, t, -d)
        cols.append((fun(qp, tp) - fun(qm, tm)) / (2 * h))
    return np.stack(cols, -1)


def test_warp_jacobian_finite_differences():
    rng = np.random.default_rng(9)
    N, P = 5, 40
    g = rng.normal(scale=20, size=(N, 3)) + [0, 0, 100]
    p = rng.normal(scale=20, size=(P, 3)) + [0, 0, 100]
    q, t = random_state(rng, N)
    nid = np.stack([rng.choice(N, 4, replace=False) for _ in range(P)])
    al = rng.uniform(0.1, 1, (P, 4))
    al /= al.sum(1, keepdims=True)
    x, J = dqb.warp_points(q, t, g, p, nid, al, nid[:, 0])
    full = np.zeros((P, 3, 6 * N))
    for k in range(4):
        for c in range(6):
            full[np.arange(P), :, 6 * nid[:, k] + c] += J[:, :, k, c]
    num = _fd(lambda qq, tt: dqb.warp_points(qq, tt, g, p, nid, al, nid[:, 0], False)[0], q, t, N)
    err = np.abs(num - full).max() / np.abs(full).max()
    assert err < 1e-6, err


def test_arap_jacobian_finite_differences():
    rng = np.random.default_rng(10)
    N = 5
    g = rng.normal(scale=20, size=(N, 3)) + [0, 0, 100]
    q, t = random_state(rng, N)
    wpair, _ = terms.arap_pair_weights(g, 0.25)
    rows, _ = terms.arap_rows(q, t, g, wpair, 1.0, 20.0, 100.0)
    R = rows.r.shape[0]
    full = np.zeros((R, 6 * N))
    for c in range(12):
        full[np.arange(R), rows.cols[:, c]] += rows.vals[:, c]
    num = _fd(lambda qq, tt: terms.arap_rows(qq, tt, g, wpair, 1.0, 20.0, 100.0)[0].r, q, t, N)
    err = np.abs(num - full).max() / np.abs(full).max()
    assert err < 1e-6, err


def test_icp_and_orb_jacobians_finite_differences(tiny):
    sc, tpl = tiny
    rng = np.random.default_rng(11)
    N = tpl.g.shape[0]
    q, t = random_state(rng, N, rot=0.02, trans=0.5)
    f = sc.frames[0]
    tgt = solver.prepare_target(f.depth, tpl.K)
    x, Jx = dqb.warp_points(q, t, tpl.g, tpl.p, tpl.nid, tpl.alpha, tpl.nid[:, 0])
    rows, _, _, pix, valid = terms.icp_rows(x, Jx, tpl.nid, tgt.X, tgt.n, tgt.ok, tpl.K, tpl.W,
                                            tpl.H, 10.0)
    v = np.flatnonzero(valid)[::37]
    qq_ = tgt.X.reshape(-1, 3)[pix[v]]
    nn_ = tgt.n.reshape(-1, 3)[pix[v]]

    def res(qa, ta):
        xx, _ = dqb.warp_points(qa, ta, tpl.g, tpl.p[v], tpl.nid[v], tpl.alpha[v], tpl.nid[v, 0], False)
        return (nn_ * (xx - qq_)).sum(1)

    num = _fd(res, q, t, N)
    sel = np.searchsorted(np.flatnonzero(valid), v)
    full = np.zeros((len(v), 6 * N))
    for c in range(24):
        full[np.arange(len(v)), rows.cols[sel, c]] += rows.vals[sel, c]
    err = np.abs(num - full).max() / np.abs(full).max()
    assert err < 1e-6, err


# ----------------------------------------------------------------------------- ARAP closed form


def test_arap_zero_for_common_rigid_motion():
    rng = np.random.default_rng(12)
    for _ in range(10):
        N = int(rng.integers(3, 12))
        g = rng.normal(scale=30, size=(N, 3)) + [0, 0, 100]
        qa = qexp_half(rng.normal(size=3))
        if qa[0] < 0:
            qa = -qa
        R = rotmat(qa)
        T = rng.normal(scale=10, size=3)
        q = np.tile(qa, (N, 1))
        t = g @ R.T + T - g
        wpair, _ = terms.arap_pair_weights(g, 0.25)
        rows, cost = terms.arap_rows(q, t, g, wpair, 3.0, 20.0, 100.0)
        assert cost < 1e-20
        A, b = solver.assemble([rows], 6 * N)
        assert np.abs(b).max() < 1e-9
        # ... and positive for a non-rigid state
        q2, t2 = random_state(rng, N)
        assert terms.arap_rows(q2, t2, g, wpair, 3.0, 20.0, 100.0)[1] > 1e-3


# ----------------------------------------------------------------------------- assembly / linear algebra


def test_normal_equations_equal_explicit_dense_triple_loop():
    cfg = Config("mini", 20, 15, 6, 20, 3, 0.3, 0.0, 0.0, 3.0, 0.0, 2.0, 1.0, 1, n_hyp=8)
    sc = make_scene(cfg, 5, f64=True)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes)
    f = sc.frames[0]
    tgt = solver.prepare_target(f.depth, tpl.K)
    rng = np.random.default_rng(13)
    q, t = random_state(rng, 6, rot=0.01, trans=0.3)
    mask = rng.random(20) < 0.5
    orb = (f.match_idx, f.match_xyz.astype(float), mask, mask.astype(float))
    rows, *_ = solver.data_terms(tpl, tgt, q, t, orb, solver.Params())
    ar, _ = terms.arap_rows(q, t, tpl.g, tpl.wpair, 2.0, 20.0, 100.0)
    rows.append(ar)
    n = 36
    Jd, Wd, rd = [], [], []
    for rw in rows:
        for i in range(rw.r.shape[0]):
            row = [0.0] * n
            for c, val in zip(rw.cols[i], rw.vals[i]):
                row[c] += val
            Jd.append(row)
            Wd.append(rw.W[i])
            rd.append(rw.r[i])
    A_ref = [[0.0] * n for _ in range(n)]
    b_ref = [0.0] * n
    for a in range(n):
        for c in range(n):
            s = 0.0
            for i in range(len(Jd)):
                s += Jd[i][a] * Wd[i] * Jd[i][c]
            A_ref[a][c] = s
        b_ref[a] = -sum(Jd[i][a] * Wd[i] * rd[i] for i in range(len(Jd)))
    A, b = solver.assemble(rows, n)
    A_ref = np.array(A_ref)
    assert np.abs(A - A_ref).max() <= 1e-12 * np.abs(A_ref).max()
    assert np.abs(b - np.array(b_ref)).max() <= 1e-12 * np.abs(b_ref).max()


def _gauss_partial_pivot(A, b):
    A = [list(r) for r in A]
    b = list(b)
    n = len(b)
    for k in range(n):
        p = max(range(k, n), key=lambda i: abs(A[i][k]))
        A[k], A[p] = A[p], A[k]
        b[k], b[p] = b[p], b[k]
        for i in range(k + 1, n):
            f = A[i][k] / A[k][k]
            for j in range(k, n):
                A[i][j] -= f * A[k][j]
            b[i] -= f * b[k]
    x = [0.0] * n
    for i in range(n - 1, -1, -1):
        x[i] = (b[i] - sum(A[i][j] * x[j] for j in range(i + 1, n))) / A[i][i]
    return np.array(x)


def test_cholesky_reconstruction_and_gaussian_elimination(tiny):
    sc, tpl = tiny
    f = sc.frames[0]
    res = solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, iters=1, keep_lins=True)
    A = solver.damp(res.lins[0].A, solver.Params())
    b = res.lins[0].b
    L = np.linalg.cholesky(A)
    assert np.linalg.norm(L @ L.T - A) / np.linalg.norm(A) < 1e-14
    x = solver.cholesky_solve(A, b)
    xg = _gauss_partial_pivot(A, b)
    assert np.abs(x - xg).max() <= 1e-9 * np.abs(xg).max()
    d0 = np.diag(res.lins[0].A)
    assert np.allclose(np.diag(A), d0 + 1e-4 * (d0 + 1e-9), rtol=1e-14, atol=0)


# ----------------------------------------------------------------------------- whole solve


def test_exact_recovery_of_a_rigid_motion_on_a_plane():
    cfg = Config("rigid_plane", 80, 60, 32, 200, 0, 0.0, 0.0, 0.0, 0.0, 0.0, 3.0, 2.0, 1,
                 planar=True)
    sc = make_scene(cfg, 31, f64=True)
    f = sc.frames[0]
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes)
    res = solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, iters=10)
    err = np.abs(res.pos - f.node_truth).max()
    assert err < 1e-9, err
    R = f.motion.Rc
    qe = res.q
    assert np.abs(rotmat(qe) - R).max() < 1e-9
    assert res.ransac["mask"].all()


def test_gauss_newton_cost_non_increasing(tiny):
    sc, tpl = tiny
    f = sc.frames[0]
    res = solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, iters=10)
    c = np.array(res.costs)
    assert (np.diff(c) <= 1e-9 * c[:-1]).all(), c
    assert c[-1] < 0.2 * c[0]


# ----------------------------------------------------------------------------- block-Jacobi step


def test_block_jacobi_step_equals_block_diagonal_gaussian_elimination(tiny):
    """The per-node step is the solution of the damped system with every coupling block between
    control points removed (checked against plain Gaussian elimination on that matrix)."""
    sc, tpl = tiny
    f = sc.frames[0]
    res = solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, iters=1, keep_lins=True)
    A = solver.damp(res.lins[0].A, solver.Params())
    b = res.lins[0].b
    n = A.shape[0]
    node = np.arange(n) // 6
    Ab = np.where(node[:, None] == node[None, :], A, 0.0)
    x = solver.block_jacobi_solve(A, b)
    xg = _gauss_partial_pivot(Ab, b)
    assert np.abs(x - xg).max() <= 1e-9 * np.abs(xg).max()
    # and it differs from the coupled step (the off-diagonal blocks are not zero here)
    assert np.abs(x - solver.cholesky_solve(A, b)).max() > 1e-3 * np.abs(xg).max()


def test_block_jacobi_keeps_an_exact_rigid_motion():
    """At the exact rigid motion of a plane every residual and gradient vanishes, so the
    block-Jacobi iteration stays there."""
    cfg = Config("rigid_plane", 80, 60, 32, 200, 0, 0.0, 0.0, 0.0, 0.0, 0.0, 3.0, 2.0, 1,
                 planar=True)
    sc = make_scene(cfg, 31, f64=True)
    f = sc.frames[0]
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes)
    exact = solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, iters=10)
    prm = solver.Params(solver="block_jacobi")
    res = solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, prm=prm, iters=3,
                             q0=exact.q, t0=exact.t)
    assert np.abs(res.pos - f.node_truth).max() < 1e-9


def test_block_jacobi_cost_non_increasing(tiny):
    sc, tpl = tiny
    f = sc.frames[0]
    prm = solver.Params(solver="block_jacobi")
    res = solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, prm=prm, iters=10)
    c = np.array(res.costs)
    assert (np.diff(c) <= 1e-9 * c[:-1]).all(), c


# ----------------------------------------------------------------------------- bilinear association


def _random_target(rng, W, H):
    X = rng.normal(size=(H, W, 3)) + np.array([0.0, 0.0, 50.0])
    n = rng.normal(size=(H, W, 3))
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    return X, n


def test_bilinear_association_equals_tent_sum_brute_force():
    """The blend is the tent-kernel sum over the image's usable pixels, weight of pixel (i, j)
    max(0, 1 - |u - i|) max(0, 1 - |v - j|), normalised by the sum of those weights; valid iff
    that sum is >= 1/2."""
    rng = np.random.default_rng(21)
    W, H = 9, 7
    K = (9.0, 9.0, 4.0, 3.0)
    X, n = _random_target(rng, W, H)
    ok = rng.uniform(size=(H, W)) > 0.15
    x = np.concatenate([rng.uniform(-6, 6, (300, 1)), rng.uniform(-5, 5, (300, 1)),
                        rng.uniform(8, 20, (300, 1))], 1)
    q, nn, valid, _, _ = terms.associate_bilinear(x, K, W, H, X, n, ok)
    fx, fy, cx, cy = K
    nvalid = 0
    for k in range(x.shape[0]):
        u = fx * x[k, 0] / x[k, 2] + cx
        v = fy * x[k, 1] / x[k, 2] + cy
        ws = 0.0
        qs = np.zeros(3)
        ns = np.zeros(3)
        for j in range(H):
            for i in range(W):
                w = max(0.0, 1 - abs(u - i)) * max(0.0, 1 - abs(v - j))
                if ok[j, i]:
                    ws += w
                    qs += w * X[j, i]
                    ns += w * n[j, i]
        assert valid[k] == (ws >= 0.5 and np.linalg.norm(ns) > 0), (k, u, v, ws)
        if not valid[k]:
            continue
        nvalid += 1
        assert np.abs(q[k] - qs / ws).max() < 1e-12
        assert np.abs(nn[k] - ns / np.linalg.norm(ns)).max() < 1e-12
    assert 50 < nvalid < 300


def test_bilinear_association_validity():
    rng = np.random.default_rng(22)
    W, H = 9, 7
    K = (9.0, 9.0, 4.0, 3.0)
    X, n = _random_target(rng, W, H)
    ok = np.ones((H, W), dtype=bool)
    ok[3, 5] = False
    # projections (u, v) chosen directly: z = 10, x = (u - cx) z / fx
    uv = np.array([[5.0, 3.0], [5.4, 3.0], [5.6, 3.0], [4.4, 3.0], [5.5, 3.5], [5.75, 3.75],
                   [8.0, 3.0], [8.4, 3.0], [8.6, 3.0], [-0.1, 2.0], [-0.6, 2.0], [2.0, 6.0],
                   [0.0, 0.0]])
    x = np.stack([(uv[:, 0] - 4.0) * 10 / 9.0, (uv[:, 1] - 3.0) * 10 / 9.0, np.full(len(uv), 10.0)], 1)
    _, _, valid, _, w = terms.associate_bilinear(x, K, W, H, X, n, ok)
    # usable weight: 0, 0.4, 0.6, 0.6, 0.75, 0.9375; right edge: 1, 0.6, 0.4; left edge: 0.9,
    # 0.4; bottom row 1; corner 1
    assert list(valid) == [False, False, True, True, True, True, True, True, False, True, False,
                           True, True]
    assert np.abs(w[valid].sum(1) - 1).max() < 1e-15
    # behind the camera
    _, _, v2, _, _ = terms.associate_bilinear(np.array([[0.0, 0.0, -5.0]]), K, W, H, X, n, ok)
    assert not v2[0]


def test_bilinear_association_on_a_plane_is_the_exact_distance():
    """On a planar target every blend of pixel points lies on the plane and every normal is the
    plane's, so r = n0 . x - c0 exactly (closed form), for any point projecting inside."""
    H, W = 12, 16
    K = (16.0, 16.0, 7.5, 5.5)
    n0 = np.array([0.2, -0.3, -1.0])
    n0 /= np.linalg.norm(n0)
    c0 = -100.0
    u, v = np.meshgrid(np.arange(W), np.arange(H))
    d = np.stack([(u - 7.5) / 16.0, (v - 5.5) / 16.0, np.ones_like(u, dtype=float)], -1)
    X, valid = frame.backproject(c0 / (d @ n0), K)
    nrm, ok = frame.target_normals(X, valid)
    rng = np.random.default_rng(23)
    uu = rng.uniform(0.5, W - 1.5, 300)
    vv = rng.uniform(0.5, H - 1.5, 300)
    z = rng.uniform(80, 120, 300)
    x = np.stack([(uu - 7.5) * z / 16.0, (vv - 5.5) * z / 16.0, z], 1)
    q, nn, vb, _, _ = terms.associate_bilinear(x, K, W, H, X, nrm, ok)
    inner = (uu >= 1) & (uu < W - 2) & (vv >= 1) & (vv < H - 2)   # all 4 corners off the border
    assert vb[inner].all() and vb.sum() > inner.sum()
    r = (nn * (x - q)).sum(1)
    assert np.abs(r[vb] - (x[vb] @ n0 - c0)).max() < 1e-9


def test_bilinear_association_is_continuous_where_rounding_jumps():
    """Along a line of points crossing many pixel boundaries the largest change of the bilinear
    residual between neighbouring samples shrinks with the sampling step (a continuous function);
    the nearest-pixel residual keeps jumps of fixed size at the half-pixel crossings."""
    sc = make_scene(CONFIGS["frame_80x60_n32"], 1000, f64=True)
    tgt = solver.prepare_target(sc.frames[0].depth, sc.K)
    Hh, Ww = tgt.ok.shape
    fx, fy, cx, cy = sc.K
    z = tgt.X[30, 40, 2] + 4.0     # off the surface, so that the normal matters

    def jumps(ns):
        us = np.linspace(30.2, 49.8, ns)
        x = np.stack([(us - cx) * z / fx, np.full_like(us, (30.3 - cy) * z / fy),
                      np.full_like(us, z)], 1)
        q, n, vb, _, _ = terms.associate_bilinear(x, sc.K, Ww, Hh, tgt.X, tgt.n, tgt.ok)
        assert vb.all()
        rb = (n * (x - q)).sum(1)
        pix, vn, _, _ = terms.associate(x, sc.K, Ww, Hh, tgt.ok)
        assert vn.all()
        rn = (tgt.n.reshape(-1, 3)[pix] * (x - tgt.X.reshape(-1, 3)[pix])).sum(1)
        return np.abs(np.diff(rb)).max(), np.abs(np.diff(rn)).max()

    b1, n1 = jumps(2001)
    b2, n2 = jumps(20001)
    assert b2 < 0.2 * b1, (b1, b2)
    assert n2 > 0.5 * n1, (n1, n2)
    assert n2 > 10 * b2


def test_bilinear_at_pixel_centres_equals_nearest():
    sc = make_scene(CONFIGS["frame_80x60_n32"], 1000, f64=True)
    tgt = solver.prepare_target(sc.frames[0].depth, sc.K)
    Hh, Ww = tgt.ok.shape
    fx, fy, cx, cy = sc.K
    rng = np.random.default_rng(24)
    pts = []
    for _ in range(200):
        i, j = rng.integers(2, Ww - 3), rng.integers(2, Hh - 3)
        z = rng.uniform(80, 120)
        pts.append([(i - cx) * z / fx, (j - cy) * z / fy, z])
    x = np.array(pts)
    qb, nb, vb, _, _ = terms.associate_bilinear(x, sc.K, Ww, Hh, tgt.X, tgt.n, tgt.ok)
    pix, vn, _, _ = terms.associate(x, sc.K, Ww, Hh, tgt.ok)
    assert np.array_equal(vb, vn)      # at a pixel centre the two validity rules agree
    both = vb & vn
    assert both.sum() > 100
    assert np.abs(qb[both] - tgt.X.reshape(-1, 3)[pix[both]]).max() < 1e-9
    assert np.abs(nb[both] - tgt.n.reshape(-1, 3)[pix[both]]).max() < 1e-9


def test_bilinear_exact_recovery_of_a_rigid_motion_on_a_plane():
    cfg = Config("rigid_plane", 80, 60, 32, 200, 0, 0.0, 0.0, 0.0, 0.0, 0.0, 3.0, 2.0, 1,
                 planar=True)
    sc = make_scene(cfg, 31, f64=True)
    f = sc.frames[0]
    prm = solver.Params(assoc="bilinear")
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    res = solver.solve_frame(tpl, f.depth, f.match_idx, f.match_xyz, f.hyp, prm, iters=10)
    assert np.abs(res.pos - f.node_truth).max() < 1e-9
    assert np.abs(rotmat(res.q) - f.motion.Rc).max() < 1e-9


# ----------------------------------------------------------------------------- warm-start RANSAC o1


def test_warm_o1_at_the_identity_is_the_template():
    sc, tpl = make_scene(CONFIGS["frame_80x60_n32"], 1000, f64=True), None
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes)
    f = sc.frames[0]
    N = tpl.g.shape[0]
    q = np.tile([1.0, 0, 0, 0], (N, 1))
    t = np.zeros((N, 3))
    o1w = solver.ransac_o1(tpl, f.match_idx, q, t, solver.Params(ransac_o1="warm"))
    o1t = solver.ransac_o1(tpl, f.match_idx, q, t, solver.Params())
    assert np.array_equal(o1t, tpl.X0[f.match_idx])
    assert np.abs(o1w - o1t).max() < 1e-12


def test_warm_o1_common_rigid_state_leaves_ransac_unchanged():
    """Every node on one rigid map x -> R x + T: the warped o1 is that map of the template
    points, and the rectified distances of Eq. 2-4 do not change (the fitted rotation absorbs R,
    the rectification removes T)."""
    sc = make_scene(CONFIGS["frame_80x60_n32"], 1000, f64=True)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes)
    f = sc.frames[0]
    rng = np.random.default_rng(25)
    N = tpl.g.shape[0]
    qr = qexp_half(rng.normal(size=3) * 0.2)
    R = rotmat(qr)
    T = rng.normal(size=3) * 5.0
    q = np.tile(qr, (N, 1))
    t = T + tpl.g @ R.T - tpl.g
    prm = solver.Params(ransac_o1="warm")
    o1w = solver.ransac_o1(tpl, f.match_idx, q, t, prm)
    p = tpl.X0[f.match_idx]
    assert np.abs(o1w - (p @ R.T + T)).max() < 1e-9
    a = ransac.ransac_1p(p, f.match_xyz, f.hyp, 2.0, 10, 0.5)
    b = ransac.ransac_1p(o1w, f.match_xyz, f.hyp, 2.0, 10, 0.5)
    assert np.abs(a["d"] - b["d"]).max() < 1e-8
    assert np.array_equal(a["kept"], b["kept"])
    near = np.zeros(len(f.match_idx), dtype=bool)
    for h in np.flatnonzero(a["kept"]):
        near |= np.abs(a["d"][h] - 2.0) <= 1e-6
    assert np.array_equal(a["mask"][~near], b["mask"][~near])


def test_warm_o1_recovers_planted_inliers_under_a_nonrigid_state():
    """Live matches made by a known non-rigid state (inliers exact, outliers >= 20 mm off): with
    o1 warped by that state the rigid model is exact for every inlier, so the preselection is
    the planted set; from the template points it is not."""
    sc = make_scene(CONFIGS["frame_80x60_n32"], 1000, f64=True)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes)
    rng = np.random.default_rng(26)
    N = tpl.g.shape[0]
    q, t = random_state(rng, N, rot=0.3, trans=3.0)
    M = 150
    midx = rng.choice(tpl.pidx, size=M, replace=False)
    prm = solver.Params(ransac_o1="warm")
    truth = solver.ransac_o1(tpl, midx, q, t, prm)
    inl = rng.uniform(size=M) >= 0.3
    off = rng.normal(size=(M, 3))
    off *= rng.uniform(20, 40, (M, 1)) / np.linalg.norm(off, axis=1, keepdims=True)
    o2 = np.where(inl[:, None], truth, truth + off)
    hyp = rng.choice(M, size=30, replace=False)
    rs = ransac.ransac_1p(truth, o2, hyp, 2.0, 10, 0.5)
    assert np.array_equal(rs["mask"], inl)
    rt = ransac.ransac_1p(tpl.X0[midx], o2, hyp, 2.0, 10, 0.5)
    assert not np.array_equal(rt["mask"], inl)


def test_warm_o1_is_invariant_to_quaternion_signs():
    """q and -q are the same rotation: flipping the sign of any nodes' quaternions leaves the
    warped o1 points unchanged (the blend aligns signs to the nearest node)."""
    sc = make_scene(CONFIGS["frame_80x60_n32"], 1000, f64=True)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes)
    f = sc.frames[0]
    rng = np.random.default_rng(27)
    N = tpl.g.shape[0]
    q, t = random_state(rng, N, rot=0.3, trans=3.0)
    prm = solver.Params(ransac_o1="warm")
    a = solver.ransac_o1(tpl, f.match_idx, q, t, prm)
    flip = rng.uniform(size=N) < 0.5
    b = solver.ransac_o1(tpl, f.match_idx, np.where(flip[:, None], -q, q), t, prm)
    assert flip.any() and np.abs(a - b).max() < 1e-9


def test_dynamic_arap_weight_counts_the_data_weights(tiny):
    """Section 2 (after Eq. 1): w_ARAP scales with the summed ICP and ORB weights per control
    point.  Live depth = template depth at the identity: every ICP association has residual 0
    (Tukey weight 1) on exactly the usable target pixels, and matches to the template's own
    points are all preselected with weight 1, so w_ARAP = w_arap0 (usable pixels + w_ORB M) / N."""
    sc, tpl = tiny
    prm = solver.Params()
    N = tpl.g.shape[0]
    rng = np.random.default_rng(5)
    midx = rng.choice(tpl.pidx, size=40, replace=False)
    o2 = tpl.X0[midx]
    rs = ransac.ransac_1p(o2, o2, np.arange(30), prm.H, prm.n_reweight, prm.keep_frac)
    assert rs["mask"].all()
    tgt = solver.prepare_target(sc.template_depth, sc.K)
    usable = int(np.asarray(tgt.ok).reshape(-1)[tpl.pidx].sum())
    q = np.tile([1.0, 0.0, 0.0, 0.0], (N, 1))
    lin, w = solver.linearize(tpl, tgt, q, np.zeros((N, 3)), (midx, o2, rs["mask"], rs["what"]),
                              None, prm)
    assert lin.n_icp == usable and lin.wsum_icp == pytest.approx(usable, rel=1e-12)
    assert lin.wsum_orb == pytest.approx(40.0, rel=1e-12)
    assert w == pytest.approx(prm.w_arap0 * (usable + prm.w_orb * 40) / N, rel=1e-12)
    # the ICP and ORB costs vanish with the residuals; the ARAP term is zero at the identity
    assert lin.cost_icp < 1e-20 and lin.cost_orb < 1e-20 and lin.cost_arap < 1e-20


def test_arap_cost_closed_form_two_nodes():
    """Eq. 5-6 on two control points 10 mm apart (pair weight w, both ordered pairs), against
    costs written out by hand: node 1 turned by theta about an axis across the pair (length kept;
    pair (1, 2) sees the angle theta, both pairs the quaternion difference of a theta / 2 turn),
    then node 2 moved sideways by d (no rotation; both pairs see the length change and the angle
    atan(d / 10))."""
    g = np.array([[0.0, 0.0, 100.0], [10.0, 0.0, 100.0]])
    w, w_arap, w_angle, w_rot = 0.7, 1.3, 20.0, 100.0
    wpair = np.array([[0.0, w], [w, 0.0]])
    th = 0.3
    q = np.array([[math.cos(th / 2), 0.0, 0.0, math.sin(th / 2)], [1.0, 0.0, 0.0, 0.0]])
    _, c = terms.arap_rows(q, np.zeros((2, 3)), g, wpair, w_arap, w_angle, w_rot)
    want = 0.5 * w_arap * w * (w_angle * (2 - 2 * math.cos(th))
                               + w_rot * 2 * (2 - 2 * math.cos(th / 2)))
    assert c == pytest.approx(want, rel=1e-12)
    dd = 4.0
    ell = math.hypot(10.0, dd)
    t = np.array([[0.0, 0.0, 0.0], [0.0, dd, 0.0]])
    _, c = terms.arap_rows(np.tile([1.0, 0, 0, 0], (2, 1)), t, g, wpair, w_arap, w_angle, w_rot)
    want = 0.5 * w_arap * w * (2 * (ell - 10.0) ** 2 + w_angle * 2 * (2 - 2 * 10.0 / ell))
    assert c == pytest.approx(want, rel=1e-12)


def test_point_to_plane_ignores_tangential_offsets():
    """Section 2, ICP paragraph: only the distance along the live surface's normal counts.  On a
    fronto-parallel plane at 100 mm (normal (0, 0, -1), towards the camera), points moved off
    the plane by delta along the normal and anywhere within it have residual exactly delta,
    whichever pixel they land on, and the cost is the Tukey penalty of those deltas."""
    W, H = 80, 60
    K = (80.0, 80.0, 39.5, 29.5)
    tgt = solver.prepare_target(np.full((H, W), 100.0), K)
    rng = np.random.default_rng(11)
    P = 300
    u = rng.uniform(6, W - 7, P)
    v = rng.uniform(6, H - 7, P)
    delta = rng.uniform(-3.0, 3.0, P)
    x = np.stack([(u - K[2]) * 100.0 / K[0], (v - K[3]) * 100.0 / K[1], np.full(P, 100.0)], 1)
    x[:, 2] -= delta                       # + delta along n = (0, 0, -1)
    rows, cost, wsum, pix, valid = terms.icp_rows(x, np.zeros((P, 3, 4, 6)),
                                                  np.zeros((P, 4), dtype=np.int64), tgt.X,
                                                  tgt.n, tgt.ok, K, W, H, 10.0)
    assert valid.all()
    assert np.abs(rows.r - delta).max() < 1e-12
    assert cost == pytest.approx(terms.tukey_rho(delta, 10.0).sum(), rel=1e-12)
    assert wsum == pytest.approx(terms.tukey_weight(delta, 10.0).sum(), rel=1e-12)


def test_no_data_keeps_the_identity(tiny):
    """Degenerate frame: a live depth map with no surface and no matches.  Only the ARAP term
    remains; it is zero with zero gradient at the identity (a common rigid state), so every
    damped Gauss-Newton step is exactly zero and the cost stays 0."""
    sc, tpl = tiny
    res = solver.solve_frame(tpl, np.zeros_like(sc.template_depth), np.zeros(0, np.int32),
                             np.zeros((0, 3)), np.zeros(0, np.int32), iters=3)
    N = tpl.g.shape[0]
    assert np.array_equal(res.q, np.tile([1.0, 0.0, 0.0, 0.0], (N, 1)))
    assert np.array_equal(res.t, np.zeros((N, 3)))
    assert res.costs == [0.0, 0.0, 0.0]


def test_association_validity_with_holes_and_points_behind_the_camera():
    """Section 2's projective association is valid only in front of the camera, inside the
    image and on a usable target pixel: brute force over every pixel with a random hole mask."""
    rng = np.random.default_rng(21)
    W, H = 9, 7
    K = (9.0, 9.0, 4.0, 3.0)
    x = np.concatenate([rng.uniform(-6, 6, (400, 2)), rng.uniform(-4, 12, (400, 1))], 1)
    x[:5, 2] = 0.0                                # on the camera plane: never valid
    tgt_ok = rng.random((H, W)) < 0.7
    pix, valid, _, _ = terms.associate(x, K, W, H, tgt_ok)
    for i in range(x.shape[0]):
        want = False
        if x[i, 2] > 0:
            u = K[0] * x[i, 0] / x[i, 2] + K[2]
            v = K[1] * x[i, 1] / x[i, 2] + K[3]
            for pv in range(H):
                for pu in range(W):
                    if -0.5 <= u - pu < 0.5 and -0.5 <= v - pv < 0.5:
                        want = bool(tgt_ok[pv, pu])
                        assert not want or pix[i] == pv * W + pu
        assert valid[i] == want, i
    assert valid.any() and not valid.all()


def test_quaternion_algebra_textbook_identities():
    """The quaternion helpers behind Section 2's warp against textbook facts: the product is
    norm-multiplicative and matches its left / right matrices, rotation matrices compose like
    the product and are proper rotations, and exp(theta / 2) is Rodrigues' rotation by |theta|
    about theta / |theta|."""
    from oracle.quat import qL, qmul, qR, rotmat, skew
    rng = np.random.default_rng(17)
    a, b = rng.normal(size=(50, 4)), rng.normal(size=(50, 4))
    ab = qmul(a, b)
    assert np.allclose(np.linalg.norm(ab, axis=1),
                       np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1), rtol=1e-13)
    assert np.allclose(np.einsum("pij,pj->pi", qL(a), b), ab, atol=1e-13)
    assert np.allclose(np.einsum("pij,pj->pi", qR(b), a), ab, atol=1e-13)
    ua = a / np.linalg.norm(a, axis=1, keepdims=True)
    ub = b / np.linalg.norm(b, axis=1, keepdims=True)
    Ra, Rb, Rab = rotmat(ua), rotmat(ub), rotmat(qmul(ua, ub))
    assert np.allclose(Rab, Ra @ Rb, atol=1e-13)
    assert np.allclose(Ra @ np.swapaxes(Ra, 1, 2), np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(Ra), 1.0, atol=1e-13)
    th = rng.normal(size=(50, 3))
    ang = np.linalg.norm(th, axis=1)
    k = th / ang[:, None]
    Kx = skew(k)
    rod = (np.eye(3) + np.sin(ang)[:, None, None] * Kx
           + (1 - np.cos(ang))[:, None, None] * (Kx @ Kx))
    assert np.allclose(rotmat(qexp_half(th)), rod, atol=1e-13)
    v = rng.normal(size=(50, 3))
    assert np.allclose(np.einsum("pij,pj->pi", skew(k), v), np.cross(k, v), atol=1e-14)


def test_ransac_preselects_the_rigid_majority_over_a_shifted_minority():
    """Section 2.1 on structured outliers: 60 matches of one exact rigid motion, 25 of the same
    rotation with a translation 100 mm off (after the rectification of Eq. 2, 100 mm off every
    fit of the first group) and 15 matches 30-60 mm off the first group's prediction.  Every
    reference on the majority settles on it (score 59 plus less than 2 from the far matches),
    every reference on the minority scores below half of that, and the preselection is exactly
    the majority, each with weight 1."""
    rng = np.random.default_rng(66)
    nA, nB, nO = 60, 25, 15
    o1 = rng.uniform(-50, 50, (nA + nB + nO, 3))
    R = axis_angle(np.array([0.3, -0.2, 1.0]), 0.4)
    o2 = o1 @ R.T + np.array([5.0, -3.0, 2.0])
    o2[nA:nA + nB] += np.array([0.0, 100.0, 0.0])
    e = rng.normal(size=(nO, 3))
    o2[nA + nB:] += e / np.linalg.norm(e, axis=1, keepdims=True) * rng.uniform(30, 60, (nO, 1))
    hyp = np.concatenate([rng.choice(nA, 8, replace=False), nA + rng.choice(nB, 6, replace=False)])
    rs = ransac.ransac_1p(o1, o2, hyp, 2.0, 10, 0.5)
    sA = rs["score"][:8]
    assert np.all((sA >= nA - 1) & (sA < nA + 1))
    assert np.all(rs["score"][8:] < 0.5 * sA.min())
    assert rs["kept"][:8].all() and not rs["kept"][8:].any()
    for h in range(8):
        assert np.array_equal(rs["d"][h] <= 2.0, np.arange(len(o1)) < nA)
    assert np.array_equal(rs["mask"], np.arange(len(o1)) < nA)
    assert np.all(rs["what"][:nA] == 1.0) and np.all(rs["what"][nA:] < 1.0)


# ----------------------------------------------------------------------------- set-up weights


def _plane_template(nodes_uv, W=12, H=12):
    """A fronto-parallel plane at z = 100 mm seen with f = 100 and the principal point at pixel
    (0, 0), so the template point of pixel (u, v) is exactly (u, v, 100) mm."""
    depth = np.full((H, W), 100.0)
    K = (100.0, 100.0, 0.0, 0.0)
    nodes = np.array([v * W + u for u, v in nodes_uv], dtype=np.int64)
    return solver.setup_template(depth, K, nodes), W


def test_blend_weights_closed_form_on_an_uneven_row_of_nodes():
    """Section 2 blending under the Gaussian-over-4-nearest reading.  Four control points on a
    row at x = 0, 1, 3, 7 mm: their nearest-neighbour spacings are 1, 1, 2 and 4 mm, so
    sigma_b = their mean = 2 mm (the minimum, 1, the maximum, 4, the median, 1.5, and the mean
    over all pairs, 3.5, all differ).  Every template point's 4 weights are then
    exp(-d^2 / 8) over the 4 nodes, normalised to sum 1, ordered nearest first with ties to the
    lower node id; the values below are those exponentials written out for three points."""
    tpl, W = _plane_template([(0, 0), (1, 0), (3, 0), (7, 0)])
    assert tpl.sigma_b == pytest.approx(2.0, rel=1e-15)

    def weights_of(u, v):
        j = int(np.flatnonzero(tpl.pidx == v * W + u)[0])
        return tpl.nid[j], tpl.alpha[j]

    e = math.exp
    cases = {
        # (pixel) -> (node ids nearest first, squared distances over 2 sigma_b^2 = 8)
        (0, 0): ([0, 1, 2, 3], [0.0, 1 / 8, 9 / 8, 49 / 8]),
        (5, 0): ([2, 3, 1, 0], [4 / 8, 4 / 8, 16 / 8, 25 / 8]),    # tie 2 / 3 -> lower id first
        (3, 2): ([2, 1, 0, 3], [4 / 8, 8 / 8, 13 / 8, 20 / 8]),
    }
    for (u, v), (ids, ex) in cases.items():
        nid, alpha = weights_of(u, v)
        a = np.array([e(-x) for x in ex])
        assert list(nid) == ids, (u, v)
        assert np.abs(alpha - a / a.sum()).max() < 1e-15, (u, v)
        assert alpha.sum() == pytest.approx(1.0, abs=1e-15)


def test_blend_weights_on_a_square_lattice():
    """Control points on a square lattice of 4 mm: sigma_b = 4 mm exactly.  A point at the
    centre of a lattice cell is equidistant from its 4 corners and gets 1/4 from each; a point
    on a lattice corner node gets 1 : e^-1/2 : e^-1/2 : e^-1 from itself, its two lattice
    neighbours and the diagonal one, i.e. the outer product of (1, e^-1/2) / (1 + e^-1/2)."""
    tpl, W = _plane_template([(u, v) for v in (2, 6, 10) for u in (2, 6, 10)])
    assert tpl.sigma_b == pytest.approx(4.0, rel=1e-15)
    j = int(np.flatnonzero(tpl.pidx == 4 * W + 4)[0])      # centre of the cell (2..6) x (2..6)
    assert sorted(tpl.nid[j]) == [0, 1, 3, 4]
    assert np.abs(tpl.alpha[j] - 0.25).max() < 1e-15
    j = int(np.flatnonzero(tpl.pidx == 2 * W + 2)[0])      # on the corner node 0
    r = math.exp(-0.5)
    want = np.array([1.0, r, r, r * r]) / (1.0 + r) ** 2
    assert list(tpl.nid[j]) == [0, 1, 3, 4]
    assert np.abs(tpl.alpha[j] - want).max() < 1e-15


def test_arap_pair_weights_closed_form():
    """Section 2.2 pair weights under the reading w = exp(-|g_i1 - g_i2|^2 / (2 sigma_A^2)),
    sigma_A = 0.25 x the diagonal of the control points' 3D bounding box, zero on the diagonal.
    Nodes (0, 0, 0), (2, 3, 6), (2, 0, 0): box 2 x 3 x 6, diagonal 7, sigma_A = 1.75,
    2 sigma_A^2 = 6.125; the squared distances are 49, 4 and 45."""
    g = np.array([[0.0, 0.0, 0.0], [2.0, 3.0, 6.0], [2.0, 0.0, 0.0]])
    w, sig = terms.arap_pair_weights(g, 0.25)
    assert sig == pytest.approx(1.75, rel=1e-15)
    want = np.zeros((3, 3))
    want[0, 1] = want[1, 0] = math.exp(-49 / 6.125)
    want[0, 2] = want[2, 0] = math.exp(-4 / 6.125)
    want[1, 2] = want[2, 1] = math.exp(-45 / 6.125)
    assert np.abs(w - want).max() < 1e-16
    # the template set-up uses the same rule on its control points: on the plane, nodes at
    # (0, 0), (3, 0), (0, 4) mm and one inside the box at (1, 1) span a 3 x 4 box, diagonal 5,
    # sigma_A = 1.25; squared distances 9, 16, 25 between the corners, 2, 5, 10 to (1, 1)
    tpl, _ = _plane_template([(0, 0), (3, 0), (0, 4), (1, 1)])
    assert tpl.sigma_A == pytest.approx(1.25, rel=1e-15)
    s2 = 2 * 1.25 ** 2
    d2 = np.array([[0, 9, 16, 2], [9, 0, 25, 5], [16, 25, 0, 10], [2, 5, 10, 0]], dtype=float)
    want = np.exp(-d2 / s2) * (1 - np.eye(4))
    assert np.abs(tpl.wpair - want).max() < 1e-16


# ----------------------------------------------------------------------------- cost vs its normal equations


def test_right_hand_side_is_the_negative_cost_gradient(tiny):
    """Eq. 1 and its normal equations (A17: every term r^2 / 2 near zero, the Tukey rho for ICP):
    with w_ARAP fixed, the preselected ORB weights constant and the association unchanged by
    the step, b = -sum W J^T r is exactly minus the gradient of the reported cost in the
    (dtheta, dt) step coordinates. Central differences of the cost through the state update on
    random coordinates; a weight applied to the rows but not to the cost (or squared in one of
    them), a dropped 1/2 or a flipped residual sign breaks the equality."""
    sc, tpl = tiny
    prm = solver.Params()
    rng = np.random.default_rng(21)
    N = tpl.g.shape[0]
    q, t = random_state(rng, N, rot=0.02, trans=0.5)
    f = sc.frames[0]
    tgt = solver.prepare_target(f.depth, tpl.K)
    midx = np.asarray(f.match_idx[:60], dtype=np.int64)
    o2 = np.asarray(f.match_xyz[:60], dtype=np.float64)
    what = rng.uniform(0.5, 1.0, len(midx))
    orb = (midx, o2, np.ones(len(midx), dtype=bool), what)
    lin, w_arap = solver.linearize(tpl, tgt, q, t, orb, None, prm)
    assert lin.cost_icp > 0 and lin.cost_orb > 0 and lin.cost_arap > 0

    def cost_at(delta):
        qa, ta = dqb.apply_step(q, t, delta)
        la, _ = solver.linearize(tpl, tgt, qa, ta, orb, w_arap, prm)
        return la.cost, la

    h = 1e-6
    coords = rng.choice(6 * N, size=24, replace=False)
    g_fd = np.zeros(len(coords))
    for k, j in enumerate(coords):
        e = np.zeros(6 * N)
        e[j] = h
        cp, lp = cost_at(e)
        cm, lm = cost_at(-e)
        # the step must not move any point to another pixel, nor across a Tukey cut
        assert np.array_equal(lp.pix, lin.pix) and np.array_equal(lm.pix, lin.pix)
        assert np.array_equal(lp.icp_valid, lin.icp_valid)
        g_fd[k] = (cp - cm) / (2 * h)
    err = np.abs(g_fd + lin.b[coords]).max() / np.abs(lin.b).max()
    assert err < 1e-6, err


def test_orb_rows_hand_computed():
    """Section 2.1, last paragraph, and Eq. 1's ORB term: r_k = x'(j_k) - o2_k, row weight
    w_ORB omega_k with omega_k = the RANSAC weight for a preselected match and the ramp
    1 - d / (5H) clamped to [0, 1] otherwise; cost 1/2 sum w_ORB omega_k |r_k|^2."""
    H, w_orb = 2.0, 10.0
    xk = np.array([[0.0, 0.0, 100.0], [5.0, 5.0, 100.0], [1.0, 0.0, 90.0], [3.0, 3.0, 95.0]])
    o2 = xk + np.array([[1.0, 2.0, 2.0],      # d = 3, preselected, RANSAC weight 0.7
                        [0.0, 0.0, 4.0],      # d = 4, not preselected: 1 - 4/10 = 0.6
                        [0.0, 12.0, 0.0],     # d = 12 > 5H: weight 0
                        [0.0, 0.0, 0.0]])     # d = 0, not preselected: weight 1
    mask = np.array([True, False, False, False])
    what = np.array([0.7, 0.9, 0.9, 0.9])
    rng = np.random.default_rng(3)
    Jk = rng.normal(size=(4, 3, 4, 6))
    nidk = np.array([[0, 1, 2, 3], [4, 5, 6, 7], [1, 3, 5, 7], [2, 4, 6, 0]])
    rows, cost, om_sum = terms.orb_rows(xk, Jk, nidk, o2, mask, what, H, w_orb)
    om = np.array([0.7, 0.6, 0.0, 1.0])
    assert np.allclose(rows.r, -(o2 - xk).reshape(-1), rtol=0, atol=1e-15)
    assert np.allclose(rows.W, np.repeat(w_orb * om, 3), rtol=0, atol=1e-15)
    assert cost == pytest.approx(0.5 * w_orb * (0.7 * 9 + 0.6 * 16 + 0.0 * 144 + 1.0 * 0), rel=1e-14)
    assert om_sum == pytest.approx(2.3, rel=1e-14)
    # row 3 k + a holds component a of match k's warp Jacobian, on its 4 nodes' 6 columns
    for k in range(4):
        for a in range(3):
            assert np.array_equal(rows.cols[3 * k + a],
                                  (6 * nidk[k][:, None] + np.arange(6)).reshape(-1))
            assert np.array_equal(rows.vals[3 * k + a], Jk[k, a].reshape(-1))


# ----------------------------------------------------------------------------- damping and the update


def test_damping_touches_only_the_diagonal():
    """Reading A1: A + lambda (diag(A) + eps) with lambda = 1e-4, eps = 1e-9; the off-diagonal
    entries are left as they are."""
    prm = solver.Params()
    A = np.array([[4.0, 1.0, -2.0], [1.0, 9.0, 0.5], [-2.0, 0.5, 0.0]])
    Ad = solver.damp(A, prm)
    assert prm.lam == 1e-4 and prm.eps == 1e-9
    want = A.copy()
    for i, a in enumerate([4.0, 9.0, 0.0]):
        want[i, i] = a + 1e-4 * (a + 1e-9)
    assert np.array_equal(Ad, want)
    assert np.array_equal(A, [[4.0, 1.0, -2.0], [1.0, 9.0, 0.5], [-2.0, 0.5, 0.0]])  # not in place


def test_state_update_is_left_multiplicative_in_the_global_frame():
    """Reading A3: the step's rotation acts in the global frame, R <- exp([dtheta]x) R (the
    quaternion exp(dtheta / 2) multiplied on the left), normalised onto q_w >= 0, and the
    translation adds. A node turned 90 degrees about x, then stepped 90 degrees about z, has
    R = Rz(90) Rx(90), not Rx(90) Rz(90); a step that takes q_w below zero comes back with the
    opposite sign (the same rotation)."""
    s = math.sqrt(0.5)
    q = np.array([[s, s, 0.0, 0.0]])                       # Rx(90 deg)
    t = np.array([[1.0, 2.0, 3.0]])
    qn, tn = dqb.apply_step(q, t, np.array([0.0, 0.0, math.pi / 2, 0.5, -1.0, 2.0]))
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])
    assert np.allclose(rotmat(qn[0]), Rz @ Rx, atol=1e-14)
    assert not np.allclose(rotmat(qn[0]), Rx @ Rz, atol=1e-3)
    assert np.allclose(qn[0], [0.5, 0.5, 0.5, 0.5], atol=1e-15)
    assert np.array_equal(tn, [[1.5, 1.0, 5.0]])
    # 270 degrees about z from the identity: exp gives q_w = cos(135 deg) < 0, flipped back
    qf, _ = dqb.apply_step(np.array([[1.0, 0.0, 0.0, 0.0]]), np.zeros((1, 3)),
                           np.array([0.0, 0.0, 1.5 * math.pi, 0.0, 0.0, 0.0]))
    assert qf[0, 0] > 0 and np.allclose(qf[0], [s, 0.0, 0.0, -s], atol=1e-15)
