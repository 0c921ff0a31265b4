"""Dual-quaternion warp of template points by their neighbouring control points (oracle).

Section 2: every control point i carries a dual quaternion W_i (a 6-DoF rigid transform) and a
template point moves with a blend of the control points near it, as in DynamicFusion.  Readings used here:

* node state: unit quaternion q_i and translation t_i with the node-centred transform
  W_i(x) = R_i (x - g_i) + g_i + t_i, g_i the node's template position; as a dual quaternion
  dq_i = (q_i, 1/2 (0, T_i) (x) q_i) with T_i = g_i + t_i - R_i g_i;
* a point j blends the dual quaternions of its 4 nearest nodes with weights alpha_jk, each sign
  aligned to the point's nearest node (s_k = +1 if q_k . q_near >= 0 else -1):
  b = sum_k alpha_jk s_k dq_k, and x' = vec(b_r (x) (0, p) (x) b_r*) / |b_r|^2
  + 2 vec(b_d (x) b_r*) / |b_r|^2 (the unit-normalised dual quaternion applied to p);
* a Gauss-Newton step moves node i by q_i <- exp(dtheta_i / 2) (x) q_i and t_i <- t_i + dt_i,
  so the 6 unknowns per node are (dtheta_i, dt_i), dtheta in the camera frame.
"""
import numpy as np

from .quat import CONJ, pure, qconj, qexp_half, qL, qmul, qR, rotmat, skew


def node_dq(q, t, g):
    """Dual quaternions (N, 8) of the node transforms.
    Section 2: each control point's warp W_i as a dual quaternion."""
    R = rotmat(q)
    T = g + t - np.einsum("nij,nj->ni", R, g)
    d = 0.5 * qmul(pure(T), q)
    return np.concatenate([q, d], axis=-1)


def node_dq_jac(q, t, g):
    """d dq_i / d(dtheta_i, dt_i) at zero step: (N, 8, 6).

    Real part:  d q / d dtheta = 1/2 qR(q)[:, 1:4]     (from (0, dtheta/2) (x) q)
    Dual part:  d = 1/2 (0, T) (x) q, with dT/d dtheta = [R g]x and dT/d dt = I, so by the
                product rule d d / d dtheta = 1/2 qL((0,T)) (d q / d dtheta)
                + 1/2 qR(q)[:, 1:4] [R g]x  and  d d / d dt = 1/2 qR(q)[:, 1:4].
    Derivative of Section 2's node dual quaternion for the Gauss-Newton step."""
    N = q.shape[0]
    R = rotmat(q)
    Rg = np.einsum("nij,nj->ni", R, g)
    T = g + t - Rg
    Rq = qR(q)[:, :, 1:4]                       # (N, 4, 3)
    dq_dth = 0.5 * Rq
    J = np.zeros((N, 8, 6))
    J[:, 0:4, 0:3] = dq_dth
    J[:, 4:8, 0:3] = 0.5 * qL(pure(T)) @ dq_dth + 0.5 * Rq @ skew(Rg)
    J[:, 4:8, 3:6] = 0.5 * Rq
    return J


def blend(dq, nid, alpha, near):
    """b_j = sum_k alpha_jk s_jk dq[nid_jk] with s_jk = sign(q_nid_jk . q_near_j) (+1 on 0).

    dq: (N, 8); nid, alpha: (P, 4); near: (P,) node id of each point's nearest node.
    Returns b (P, 8) and the signs s (P, 4).
    Section 2: a template point moves with a blend of the control points near it."""
    qk = dq[nid, 0:4]                           # (P, 4, 4)
    qn = dq[near, 0:4]                          # (P, 4)
    s = np.where(np.einsum("pki,pi->pk", qk, qn) >= 0, 1.0, -1.0)
    b = np.einsum("pk,pki->pi", alpha * s, dq[nid])
    return b, s


def apply_dq(b, p):
    """x' = (vec(b_r (x) (0,p) (x) b_r*) + 2 vec(b_d (x) b_r*)) / |b_r|^2.  b (P,8), p (P,3).
    Section 2: the blended dual quaternion applied to a template point."""
    br, bd = b[:, 0:4], b[:, 4:8]
    y = qmul(qmul(br, pure(p)), qconj(br))[:, 1:4] + 2.0 * qmul(bd, qconj(br))[:, 1:4]
    s = (br * br).sum(1)
    return y / s[:, None]


def apply_dq_jac(b, p):
    """d x' / d b: (P, 3, 8), from x' = y / s with s = |b_r|^2 and
       dy/db_r = Pv [qR((0,p) (x) b_r*) + qL(b_r (x) (0,p)) CONJ + 2 qL(b_d) CONJ],
       dy/db_d = 2 Pv qR(b_r*),  ds/db_r = 2 b_r.
    Derivative of Section 2's warp of a point for the Gauss-Newton step."""
    br, bd = b[:, 0:4], b[:, 4:8]
    pp = pure(p)
    brc = qconj(br)
    y = qmul(qmul(br, pp), brc)[:, 1:4] + 2.0 * qmul(bd, brc)[:, 1:4]
    s = (br * br).sum(1)
    x = y / s[:, None]
    dy_dbr = (qR(qmul(pp, brc)) + qL(qmul(br, pp)) @ CONJ + 2.0 * qL(bd) @ CONJ)[:, 1:4, :]
    dy_dbd = 2.0 * qR(brc)[:, 1:4, :]
    dy = np.concatenate([dy_dbr, dy_dbd], axis=2)            # (P, 3, 8)
    ds = np.concatenate([2.0 * br, np.zeros_like(bd)], axis=1)  # (P, 8)
    return (dy - x[:, :, None] * ds[:, None, :]) / s[:, None, None]


def warp_points(q, t, g, p, nid, alpha, near, with_jac=True):
    """Warped points x' (P, 3) and, if asked, d x' / d(dtheta, dt) of the 4 nodes: (P, 3, 4, 6).
    Section 2: the deformed template."""
    dq = node_dq(q, t, g)
    b, s = blend(dq, nid, alpha, near)
    x = apply_dq(b, p)
    if not with_jac:
        return x, None
    Gn = node_dq_jac(q, t, g)                    # (N, 8, 6)
    Dx = apply_dq_jac(b, p)                      # (P, 3, 8)
    J = np.einsum("pab,pkbc->pkac", Dx, (alpha * s)[:, :, None, None] * Gn[nid])
    return x, np.transpose(J, (0, 2, 1, 3))      # (P, 3, 4, 6)


def apply_step(q, t, delta):
    """Node update of the Gauss-Newton step delta (N*6,): q <- normalize(exp(dtheta/2) (x) q),
    flipped to q_w >= 0; t <- t + dt.
    Section 2: the Levenberg-Marquardt update of every W_i, taken as a damped Gauss-Newton step."""
    d = np.asarray(delta, dtype=np.float64).reshape(-1, 6)
    qn = qmul(qexp_half(d[:, 0:3]), q)
    qn = qn / np.linalg.norm(qn, axis=1, keepdims=True)
    qn = np.where((qn[:, 0] < 0)[:, None], -qn, qn)
    return qn, t + d[:, 3:6]
