"""The three terms of the total cost, Eq. 1: f_ICP + w_ORB f_ORB + w_ARAP f_ARAP (oracle).

Each term returns residual rows in a sparse form: r (R,), row weight W (R,), column ids (R, k)
and Jacobian values (R, k) over the 6N unknowns (node-major, (dtheta, dt) per node).  The
Gauss-Newton normal equations are A = sum W J^T J and b = -sum W J^T r; the reported cost is
sum rho(r) for ICP and 1/2 sum W r^2 for the two squared terms (so that every term is r^2 / 2
near zero, matching the Tukey penalty's small-residual behaviour).
"""
import dataclasses

import numpy as np

from .quat import qR, rotmat, skew


@dataclasses.dataclass
class Rows:
    r: np.ndarray
    W: np.ndarray
    cols: np.ndarray
    vals: np.ndarray


# ----------------------------------------------------------------------------- ICP


def tukey_weight(r, c):
    """IRLS weight of Tukey's biweight: (1 - (r/c)^2)^2 for |r| < c, else 0.
    Section 2, ICP paragraph: Tukey's penalty on the point-to-plane residual."""
    u = r / c
    return np.where(np.abs(r) < c, (1.0 - u * u) ** 2, 0.0)


def tukey_rho(r, c):
    """Tukey's penalty c^2/6 (1 - (1 - (r/c)^2)^3), capped at c^2/6 for |r| >= c.
    Section 2, ICP paragraph: Tukey's penalty on the point-to-plane residual."""
    u = r / c
    return np.where(np.abs(r) < c, c * c / 6.0 * (1.0 - (1.0 - u * u) ** 3), c * c / 6.0)


def associate(x, K, W, H, tgt_ok):
    """Projective association (Section 2, the "rasterization" that replaces a kd-tree search):
    project the warped point and take the nearest pixel, pu = floor(fx x/z + cx + 1/2) and the
    same for v.  No z-buffer.  Returns (pixel index (P,), valid (P,) bool, (u, v) float)."""
    fx, fy, cx, cy = K
    z = x[:, 2]
    zs = np.where(z > 0, z, 1.0)
    u = fx * x[:, 0] / zs + cx
    v = fy * x[:, 1] / zs + cy
    pu = np.floor(u + 0.5)
    pv = np.floor(v + 0.5)
    inside = (z > 0) & (pu >= 0) & (pu < W) & (pv >= 0) & (pv < H)
    pix = np.where(inside, pv * W + pu, 0).astype(np.int64)
    valid = inside & tgt_ok.reshape(-1)[pix]
    return pix, valid, u, v


def associate_bilinear(x, K, W, H, tgtX, tgtN, tgt_ok):
    """Continuous variant of the projective association (Section 2 "rasterization"; an
    interpolated lookup replaces the pixel rounding): with (u, v) the projection of the warped
    point, u0 = floor(u), a = u - u0 (v0, b likewise), the 4 pixels (u0 + i, v0 + j),
    i, j in {0, 1}, carry the bilinear weights (1 - a)(1 - b), a (1 - b), (1 - a) b, a b.  Pixels
    outside the image or not usable are dropped and the weights of the others renormalised:
    q = sum_c w_c X_c / sum_c w_c over usable corners, n = the same blend of normals, normalised.
    Valid iff z > 0, the usable weight sum is >= 1/2 and the normal blend is nonzero.  (Along
    one axis next to an unusable pixel the point stays valid exactly while the nearest-pixel
    rule would pick the usable pixel; the result is continuous in (u, v) inside the valid set,
    including at integer coordinates, where the template points fall at the identity state.)

    Returns (q (P, 3), n (P, 3), valid (P,) bool, corner pixels (P, 4), weights (P, 4)); the
    weights are the renormalised ones (0 for dropped corners)."""
    fx, fy, cx, cy = K
    z = x[:, 2]
    zs = np.where(z > 0, z, 1.0)
    u = fx * x[:, 0] / zs + cx
    v = fy * x[:, 1] / zs + cy
    u0 = np.floor(u)
    v0 = np.floor(v)
    a = u - u0
    b = v - v0
    cu = np.stack([u0, u0 + 1, u0, u0 + 1], 1)
    cv = np.stack([v0, v0, v0 + 1, v0 + 1], 1)
    inimg = (z[:, None] > 0) & (cu >= 0) & (cu <= W - 1) & (cv >= 0) & (cv <= H - 1)
    pix = np.where(inimg, cv * W + cu, 0).astype(np.int64)
    usable = inimg & tgt_ok.reshape(-1)[pix]
    wts = np.stack([(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b], 1) * usable
    ws = wts.sum(1)
    X = tgtX.reshape(-1, 3)[pix]                       # (P, 4, 3)
    Nn = tgtN.reshape(-1, 3)[pix]
    wn = wts / np.where(ws > 0, ws, 1.0)[:, None]
    q = (wn[:, :, None] * X).sum(1)
    nb = (wn[:, :, None] * Nn).sum(1)
    ln = np.linalg.norm(nb, axis=1)
    valid = (z > 0) & (ws >= 0.5) & (ln > 0)
    n = nb / np.where(ln > 0, ln, 1.0)[:, None]
    return q, n, valid, pix, wn


def icp_rows(x, Jx, nid, tgtX, tgtN, tgt_ok, K, W, H, c, assoc="nearest"):
    """Point-to-plane ICP with Tukey weights: r_j = n_q . (x'_j - q) at the associated target
    pixel q (Section 2, ICP paragraph).  x: (P, 3) warped template points, Jx: (P, 3, 4, 6).
    assoc = "nearest" (pixel rounding) or "bilinear" (associate_bilinear); in both the target
    point and normal are held fixed in the Jacobian, J = n^T dx'/d(dtheta, dt).

    Returns (Rows over the valid associations, cost, sum of Tukey weights, pixel, valid); the
    pixel of a bilinear association is its (u0, v0) corner."""
    if assoc == "bilinear":
        q, n, valid, pix4, _ = associate_bilinear(x, K, W, H, tgtX, tgtN, tgt_ok)
        pix = pix4[:, 0]
    else:
        pix, valid, _, _ = associate(x, K, W, H, tgt_ok)
        q = tgtX.reshape(-1, 3)[pix]
        n = tgtN.reshape(-1, 3)[pix]
    r = (n * (x - q)).sum(1)
    w = tukey_weight(r, c)
    rho = tukey_rho(r, c)
    cost = rho[valid].sum()
    wsum = w[valid].sum()
    J = np.einsum("pa,pakc->pkc", n, Jx).reshape(-1, 24)
    cols = (6 * nid[:, :, None] + np.arange(6)).reshape(-1, 24)
    v = np.flatnonzero(valid)
    return Rows(r[v], w[v], cols[v], J[v]), cost, wsum, pix, valid


# ----------------------------------------------------------------------------- ORB


def orb_weight(d, mask, what, H):
    """Section 2.1, last paragraph: preselected matches keep their RANSAC weight; the others get
    w = -d / (5H) + 1 clamped to [0, 1], d the current distance of the match."""
    ramp = np.clip(1.0 - d / (5.0 * H), 0.0, 1.0)
    return np.where(mask, what, ramp)


def orb_rows(xk, Jk, nidk, o2, mask, what, H, w_orb):
    """r_k = x'(j_k) - o2_k (3 rows per match), row weight w_ORB * omega_k.
    xk: (M, 3), Jk: (M, 3, 4, 6).  Returns (Rows, cost, sum omega)."""
    r = xk - o2
    d = np.linalg.norm(r, axis=1)
    om = orb_weight(d, mask, what, H)
    M = xk.shape[0]
    cols = (6 * nidk[:, :, None] + np.arange(6)).reshape(M, 1, 24)
    cols = np.broadcast_to(cols, (M, 3, 24)).reshape(-1, 24)
    vals = Jk.reshape(M, 3, 24).reshape(-1, 24)
    Wr = np.repeat(w_orb * om, 3)
    cost = 0.5 * (w_orb * om * (r * r).sum(1)).sum()
    return Rows(r.reshape(-1), Wr, cols, vals), cost, om.sum()


# ----------------------------------------------------------------------------- ARAP


def arap_pair_weights(g, sigma_scale):
    """w_{i1 i2} = exp(-|g_i1 - g_i2|^2 / (2 sigma_A^2)), sigma_A = sigma_scale x the diagonal of
    the control points' bounding box (Section 2.2: nearer at time 0 -> larger weight); zero on
    the diagonal.  Returns (w (N, N), sigma_A)."""
    sig = sigma_scale * np.linalg.norm(g.max(0) - g.min(0))
    d2 = ((g[:, None, :] - g[None, :, :]) ** 2).sum(-1)
    w = np.exp(-d2 / (2.0 * sig * sig))
    np.fill_diagonal(w, 0.0)
    return w, sig


def arap_rows(q, t, g, wpair, w_arap, w_angle, w_rot, chunk=64):
    """Dense ARAP over all ordered pairs i1 != i2 (Eq. 5-6), with p_i = W_i(g_i) = g_i + t_i.

      r_len = |p_i2 - p_i1| - |g_i2 - g_i1|                                   (1 row)
      r_ang = u - v, u = unit(W_i1(g_i2) - p_i1) = unit(R_i1 (g_i2 - g_i1)),
              v = unit(p_i2 - p_i1)                                           (3 rows)
      r_rot = q_i1 - s q_i2, s = sign(q_i1 . q_i2)                            (4 rows)

    |r_ang|^2 = 2 - 2 cos(angle), a smooth stand-in for the angle of Eq. 6; r_rot compares the
    rotation quaternions (the dual quaternions' real parts) up to the q ~ -q sign.
    Row weights: w_ARAP w_i1i2 x (1, w_angle, w_rot).  Columns: (dtheta, dt) of i1 then i2."""
    N = g.shape[0]
    R = rotmat(q)
    p = g + t
    Rq = qR(q)[:, :, 1:4]                              # d q / d dtheta = 1/2 Rq
    out_r, out_W, out_c, out_v = [], [], [], []
    cost = 0.0
    I3 = np.eye(3)
    for a0 in range(0, N, chunk):
        i1, i2 = np.meshgrid(np.arange(a0, min(N, a0 + chunk)), np.arange(N), indexing="ij")
        i1 = i1.reshape(-1)
        i2 = i2.reshape(-1)
        keep = i1 != i2
        i1, i2 = i1[keep], i2[keep]
        P = i1.shape[0]
        e = p[i2] - p[i1]
        ell = np.linalg.norm(e, axis=1)
        L0 = np.linalg.norm(g[i2] - g[i1], axis=1)
        vhat = e / ell[:, None]
        a = np.einsum("pij,pj->pi", R[i1], g[i2] - g[i1])
        an = np.linalg.norm(a, axis=1)
        uhat = a / an[:, None]
        s = np.where((q[i1] * q[i2]).sum(1) >= 0, 1.0, -1.0)
        r_len = ell - L0
        r_ang = uhat - vhat
        r_rot = q[i1] - s[:, None] * q[i2]
        J = np.zeros((P, 8, 12))
        # length: d|e| / d dt_i2 = vhat^T, d / d dt_i1 = -vhat^T
        J[:, 0, 3:6] = -vhat
        J[:, 0, 9:12] = vhat
        # angle: du/d dtheta_i1 = (I - u u^T)/|a| (-[a]x); dv/d dt_i2 = (I - v v^T)/|e|
        Pu = (I3 - uhat[:, :, None] * uhat[:, None, :]) / an[:, None, None]
        Pv = (I3 - vhat[:, :, None] * vhat[:, None, :]) / ell[:, None, None]
        J[:, 1:4, 0:3] = Pu @ (-skew(a))
        J[:, 1:4, 3:6] = Pv
        J[:, 1:4, 9:12] = -Pv
        # rotation: d q_i1 / d dtheta_i1 = 1/2 Rq(q_i1); d(-s q_i2) / d dtheta_i2 = -s/2 Rq(q_i2)
        J[:, 4:8, 0:3] = 0.5 * Rq[i1]
        J[:, 4:8, 6:9] = -0.5 * s[:, None, None] * Rq[i2]
        r = np.concatenate([r_len[:, None], r_ang, r_rot], axis=1)          # (P, 8)
        wp = w_arap * wpair[i1, i2]
        W = wp[:, None] * np.array([1.0, w_angle, w_angle, w_angle, w_rot, w_rot, w_rot, w_rot])
        cols = np.concatenate([6 * i1[:, None] + np.arange(6), 6 * i2[:, None] + np.arange(6)], 1)
        cost += 0.5 * (W * r * r).sum()
        out_r.append(r.reshape(-1))
        out_W.append(W.reshape(-1))
        out_c.append(np.broadcast_to(cols[:, None, :], (P, 8, 12)).reshape(-1, 12))
        out_v.append(J.reshape(-1, 12))
    return (Rows(np.concatenate(out_r), np.concatenate(out_W), np.concatenate(out_c),
                 np.concatenate(out_v)), cost)
