"""Template set-up, normal-equation assembly and the damped Gauss-Newton frame solve (oracle).

Section 2: the deformation is estimated by minimising Eq. 1 with Levenberg-Marquardt; the
Jacobian rows of each term are assembled into normal equations and solved by a Cholesky
decomposition; w_ORB = 10 and w_ARAP is rescaled by the summed ICP and ORB weights.

Readings used here (the CUDA path implements the same ones):
* the normal equations couple all 6N unknowns (one dense system) and are damped with a fixed
  lambda: A + lambda (diag(A) + eps), lambda = 1e-4, eps = 1e-9, with no accept/reject test, so
  both sides run the same number of iterations; the per-control-point update Section 2
  describes is the alternative block-Jacobi step (each control point's 6 x 6 diagonal block
  alone);
* w_ARAP = w_arap0 * (sum of ICP Tukey weights + w_ORB * sum of ORB weights) / N, evaluated once
  per frame at the warm-start state and then held for the frame;
* each template point is blended by its 4 nearest control points (3D distance at time 0, ties
  to the lower node id) with weights exp(-d^2 / (2 sigma_b^2)) normalised to 1, sigma_b =
  sigma_blend_scale x the mean nearest-neighbour spacing of the control points;
* the ORB match points of the template side (o1 of Eq. 2) are the template's back-projected
  points at the matched pixels (ransac_o1 = "template"), or, in the warm-start variant
  (ransac_o1 = "warm"), those template points warped by the frame's warm-start state, so that the
  rigid model of the 1-point RANSAC only has to explain the motion since the previous frame;
* the ICP association rounds the projection to the nearest pixel (assoc = "nearest") or blends
  the 4 surrounding pixels bilinearly (assoc = "bilinear", terms.associate_bilinear).
"""
import dataclasses

import numpy as np
import scipy.linalg
import scipy.sparse

from . import dqb, frame, ransac, terms


@dataclasses.dataclass
class Params:
    w_orb: float = 10.0          # Section 2
    w_angle: float = 20.0        # Section 2.2
    w_rot: float = 100.0         # Section 2.2
    w_arap0: float = 1.0
    H: float = 2.0               # threshold of Eq. 4 (mm)
    tukey_c: float = 10.0        # mm
    sigma_blend_scale: float = 1.0
    sigma_arap_scale: float = 0.25
    lam: float = 1e-4
    eps: float = 1e-9
    keep_frac: float = 0.5
    n_hyp: int = 30              # Section 2.1
    n_reweight: int = 10         # Section 2.1
    solver: str = "dense"        # "dense" Cholesky of the 6N system, or "block_jacobi" (per node)
    assoc: str = "nearest"       # ICP association: "nearest" pixel or "bilinear" blend
    ransac_o1: str = "template"  # RANSAC o1: "template" points or "warm" (warped by the warm start)


@dataclasses.dataclass
class Template:
    W: int
    H: int
    K: tuple
    X0: np.ndarray        # (H*W, 3) back-projected template
    valid0: np.ndarray    # (H*W,)
    nodes: np.ndarray     # (N,) pixel ids
    g: np.ndarray         # (N, 3)
    pidx: np.ndarray      # (P,) pixel ids of the valid template points
    p: np.ndarray         # (P, 3)
    nid: np.ndarray       # (P, 4) node ids, nearest first
    alpha: np.ndarray     # (P, 4)
    sigma_b: float
    wpair: np.ndarray     # (N, N)
    sigma_A: float


def nearest_nodes(p, g, k=4, chunk=8192):
    """k nearest nodes of every point by squared distance (dx^2 + dy^2) + dz^2, ties to the lower
    node id.  Returns (ids (P, k), squared distances (P, k)).
    Section 2: a template point's neighbouring control points."""
    P = p.shape[0]
    ids = np.zeros((P, k), dtype=np.int64)
    d2k = np.zeros((P, k))
    for a in range(0, P, chunk):
        pp = p[a:a + chunk]
        dx = pp[:, None, 0] - g[None, :, 0]
        dy = pp[:, None, 1] - g[None, :, 1]
        dz = pp[:, None, 2] - g[None, :, 2]
        d2 = dx * dx + dy * dy + dz * dz
        o = np.argsort(d2, axis=1, kind="stable")[:, :k]
        ids[a:a + chunk] = o
        d2k[a:a + chunk] = np.take_along_axis(d2, o, axis=1)
    return ids, d2k


def setup_template(depth, K, nodes, prm: Params = Params()):
    """Back-project the template, place the control points and build the blend tables.
    Section 2: template, control points and blending."""
    H, W = depth.shape
    X0, valid0 = frame.backproject(depth, K)
    X0 = X0.reshape(-1, 3)
    valid0 = valid0.reshape(-1)
    nodes = np.asarray(nodes, dtype=np.int64)
    if not valid0[nodes].all():
        raise ValueError("control point on an invalid template pixel")
    g = X0[nodes]
    N = g.shape[0]
    d2n = ((g[:, None, :] - g[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2n, np.inf)
    sigma_b = prm.sigma_blend_scale * np.sqrt(d2n.min(1)).mean()
    pidx = np.flatnonzero(valid0)
    p = X0[pidx]
    nid, d2 = nearest_nodes(p, g, 4)
    a = np.exp(-d2 / (2.0 * sigma_b * sigma_b))
    alpha = a / a.sum(1, keepdims=True)
    wpair, sigma_A = terms.arap_pair_weights(g, prm.sigma_arap_scale)
    return Template(W, H, tuple(float(k) for k in K), X0, valid0, nodes, g, pidx, p, nid, alpha,
                    sigma_b, wpair, sigma_A)


@dataclasses.dataclass
class Target:
    X: np.ndarray      # (H, W, 3)
    n: np.ndarray      # (H, W, 3)
    ok: np.ndarray     # (H, W)


def prepare_target(depth, K):
    """Section 2: the live point map and normals the ICP term associates with."""
    X, valid = frame.backproject(depth, K)
    n, ok = frame.target_normals(X, valid)
    return Target(X, n, ok)


def assemble(rows_list, n):
    """A = sum W J^T J (dense n x n), b = -sum W J^T r.
    Section 2: the normal equations of Eq. 1 for the Cholesky solve."""
    A = np.zeros((n, n))
    b = np.zeros(n)
    for rw in rows_list:
        R, k = rw.cols.shape
        if R == 0:
            continue
        J = scipy.sparse.csr_matrix((rw.vals.reshape(-1), (np.repeat(np.arange(R), k),
                                                            rw.cols.reshape(-1))), shape=(R, n))
        JW = J.T.multiply(rw.W[None, :]).tocsr()
        A += (JW @ J).toarray()
        b -= JW @ rw.r
    return A, b


@dataclasses.dataclass
class Linearization:
    A: np.ndarray
    b: np.ndarray
    cost: float
    cost_icp: float
    cost_orb: float
    cost_arap: float
    wsum_icp: float
    wsum_orb: float
    n_icp: int
    pix: np.ndarray
    icp_valid: np.ndarray


def data_terms(tpl: Template, tgt: Target, q, t, orb, prm: Params):
    """ICP and ORB rows at state (q, t).  orb = (match_idx, o2, mask, what) or None."""
    x, Jx = dqb.warp_points(q, t, tpl.g, tpl.p, tpl.nid, tpl.alpha, tpl.nid[:, 0])
    icp, c_icp, ws_icp, pix, valid = terms.icp_rows(x, Jx, tpl.nid, tgt.X, tgt.n, tgt.ok, tpl.K,
                                                    tpl.W, tpl.H, prm.tukey_c, prm.assoc)
    rows = [icp]
    c_orb, ws_orb = 0.0, 0.0
    if orb is not None and len(orb[0]) > 0:
        midx, o2, mask, what = orb
        jr = template_rank(tpl, midx)
        xk, Jk = x[jr], Jx[jr]
        orb_r, c_orb, ws_orb = terms.orb_rows(xk, Jk, tpl.nid[jr], o2, mask, what, prm.H, prm.w_orb)
        rows.append(orb_r)
    return rows, c_icp, c_orb, ws_icp, ws_orb, pix, valid


def template_rank(tpl: Template, pix):
    """Position of each template pixel in the list of valid template points.
    Section 2.1: the template point o1 of a match (Eq. 2)."""
    rank = np.full(tpl.W * tpl.H, -1, dtype=np.int64)
    rank[tpl.pidx] = np.arange(tpl.pidx.shape[0])
    return rank[np.asarray(pix, dtype=np.int64)]


def ransac_o1(tpl: Template, midx, q, t, prm: Params):
    """o1 of Eq. 2 for the matched template pixels: the template points, or (warm-start
    variant) the same points warped by the state (q, t) the frame starts from."""
    if prm.ransac_o1 == "warm":
        jr = template_rank(tpl, midx)
        x, _ = dqb.warp_points(q, t, tpl.g, tpl.p[jr], tpl.nid[jr], tpl.alpha[jr], tpl.nid[jr, 0],
                               with_jac=False)
        return x
    return tpl.X0[np.asarray(midx, dtype=np.int64)]


def linearize(tpl: Template, tgt: Target, q, t, orb, w_arap, prm: Params):
    """Normal equations (undamped) and cost at state (q, t).  If w_arap is None it is set from
    the data-term weights at this state (the per-frame rule) and returned in the result.
    Eq. 1: f_ICP + w_ORB f_ORB + w_ARAP f_ARAP and its normal equations."""
    rows, c_icp, c_orb, ws_icp, ws_orb, pix, valid = data_terms(tpl, tgt, q, t, orb, prm)
    N = tpl.g.shape[0]
    if w_arap is None:
        w_arap = prm.w_arap0 * (ws_icp + prm.w_orb * ws_orb) / N
    ar, c_arap = terms.arap_rows(q, t, tpl.g, tpl.wpair, w_arap, prm.w_angle, prm.w_rot)
    rows.append(ar)
    A, b = assemble(rows, 6 * N)
    lin = Linearization(A, b, c_icp + c_orb + c_arap, c_icp, c_orb, c_arap, ws_icp, ws_orb,
                        int(valid.sum()), pix, valid)
    return lin, w_arap


def damp(A, prm: Params):
    """A + lambda (diag(A) + eps) on the diagonal.
    Section 2 (Levenberg-Marquardt): the damping of the normal equations."""
    Ad = A.copy()
    idx = np.arange(A.shape[0])
    Ad[idx, idx] += prm.lam * (np.diag(A) + prm.eps)
    return Ad


def cholesky_solve(A, b):
    """x = L^-T L^-1 b with A = L L^T (Section 2: Cholesky decomposition)."""
    L = np.linalg.cholesky(A)
    y = scipy.linalg.solve_triangular(L, b, lower=True)
    return scipy.linalg.solve_triangular(L.T, y, lower=False)


def block_jacobi_solve(A, b):
    """Section 2 takes the LM step one control point at a time: every control point's
    6 unknowns from its own 6 x 6 diagonal block of the (damped) normal matrix, the coupling
    blocks between control points left out. x_i = A_ii^-1 b_i, each by a Cholesky
    factorisation."""
    n = A.shape[0]
    x = np.empty(n)
    for i in range(0, n, 6):
        x[i:i + 6] = cholesky_solve(A[i:i + 6, i:i + 6], b[i:i + 6])
    return x


@dataclasses.dataclass
class FrameResult:
    q: np.ndarray
    t: np.ndarray
    pos: np.ndarray                 # control points p_i = g_i + t_i
    costs: list                     # cost at each linearisation point
    w_arap: float
    ransac: dict
    states: list                    # (q, t) after every iteration
    lins: list


def solve_frame(tpl: Template, depth, match_idx, match_xyz, hyp, prm: Params = Params(), iters=10,
                q0=None, t0=None, keep_lins=False):
    """One frame: target prep, 1-point RANSAC, then `iters` damped Gauss-Newton iterations.
    Sections 2 and 2.1: one frame's whole deformation solve."""
    N = tpl.g.shape[0]
    q = np.tile([1.0, 0.0, 0.0, 0.0], (N, 1)) if q0 is None else np.asarray(q0, np.float64).copy()
    t = np.zeros((N, 3)) if t0 is None else np.asarray(t0, np.float64).copy()
    tgt = prepare_target(depth, tpl.K)
    midx = np.asarray(match_idx, dtype=np.int64)
    o1 = ransac_o1(tpl, midx, q, t, prm) if len(midx) > 0 else np.zeros((0, 3))
    o2 = np.asarray(match_xyz, dtype=np.float64).reshape(-1, 3)
    if len(midx) > 0:
        rs = ransac.ransac_1p(o1, o2, np.asarray(hyp), prm.H, prm.n_reweight, prm.keep_frac)
        orb = (midx, o2, rs["mask"], rs["what"])
    else:
        rs = None
        orb = None
    w_arap = None
    costs, states, lins = [], [], []
    for _ in range(iters):
        lin, w_arap = linearize(tpl, tgt, q, t, orb, w_arap, prm)
        costs.append(lin.cost)
        Ad = damp(lin.A, prm)
        if prm.solver == "block_jacobi":
            delta = block_jacobi_solve(Ad, lin.b)
        else:
            delta = cholesky_solve(Ad, lin.b)
        q, t = dqb.apply_step(q, t, delta)
        states.append((q.copy(), t.copy()))
        if keep_lins:
            lins.append(lin)
    return FrameResult(q, t, tpl.g + t, costs, w_arap, rs, states, lins)


def frame_cost(tpl: Template, depth, q, t, orb, w_arap, prm: Params = Params()):
    """Cost of Eq. 1 at state (q, t) for a frame, with a fixed w_ARAP."""
    tgt = prepare_target(depth, tpl.K)
    lin, _ = linearize(tpl, tgt, q, t, orb, w_arap, prm)
    return lin.cost
