"""1-point RANSAC + reweighting inlier preselection (oracle, float64).

Section 2.1, Eq. 2-4: for a reference match k0 the coordinates of both 3D match sets are
rectified to that match (Eq. 2); a rotation R with S2(k) ~ R S1(k) (Eq. 3) is fitted from the
weighted columns, the weights are reset to w_k = min(H / d_k, 1) with d_k = |S2(k) - R S1(k)|
(Eq. 4), and the two steps alternate for a fixed number of iterations (10 in the paper).  A
reference whose weight sum is small is dropped; 30 random references are tried.

Readings where the paper is silent:
* the rotation is the weighted orthogonal Procrustes (Kabsch) solution with a reflection guard,
  R = U diag(1, 1, det(U V^T)) V^T for C = sum_k w_k S2(k) S1(k)^T = U Sigma V^T; no centroid,
  because the rectification already puts the reference at the origin.  If sum w < 1e-12, or the
  fit is degenerate (sigma2 + det-sign * sigma3 <= 1e-12 |C|_F, i.e. the two largest eigenvalues
  of Horn's matrix coincide), R = I;
* d_k = 0 gives w_k = 1;
* a reference is kept iff sum_{k != k0} w_k >= keep_frac * max over references (keep_frac 0.5);
* a match is preselected iff some kept reference has d_k <= H; its weight is the largest w_k
  over kept references.
"""
import numpy as np


def kabsch(S1, S2, w):
    """Weighted rotation R maximising sum_k w_k S2(k)^T R S1(k).  S1, S2: (M, 3); w: (M,).
    Eq. 3: the rotation of the 1-point RANSAC fit."""
    C = (S2 * w[:, None]).T @ S1
    if w.sum() < 1e-12:
        return np.eye(3)
    U, sig, Vt = np.linalg.svd(C)
    d = 1.0 if np.linalg.det(U @ Vt) >= 0 else -1.0
    fro = np.sqrt((C * C).sum())
    if sig[1] + d * sig[2] <= 1e-12 * fro:
        return np.eye(3)
    return U @ np.diag([1.0, 1.0, d]) @ Vt


def horn(S1, S2, w):
    """The same rotation by Horn's method: the eigenvector of the largest eigenvalue of the 4x4
    symmetric matrix built from M = sum_k w_k S1(k) S2(k)^T is the unit quaternion of R.
    Used only as an independent check of kabsch()."""
    M = (S1 * w[:, None]).T @ S2
    Sxx, Sxy, Sxz = M[0]
    Syx, Syy, Syz = M[1]
    Szx, Szy, Szz = M[2]
    N = np.array([[Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx],
                  [Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz],
                  [Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy],
                  [Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz]])
    evals, evecs = np.linalg.eigh(N)
    q = evecs[:, -1]
    w0, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w0 * z), 2 * (x * z + w0 * y)],
                     [2 * (x * y + w0 * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w0 * x)],
                     [2 * (x * z - w0 * y), 2 * (y * z + w0 * x), 1 - 2 * (x * x + y * y)]])


def reweight(S1, S2, H, n_iter):
    """Alternate Kabsch and Eq. 4 for one reference.  Returns (d, w) after the last update."""
    M = S1.shape[0]
    w = np.ones(M)
    d = np.zeros(M)
    for _ in range(n_iter):
        R = kabsch(S1, S2, w)
        d = np.linalg.norm(S2 - S1 @ R.T, axis=1)
        w = np.ones(M)
        pos = d > 0
        w[pos] = np.minimum(H / d[pos], 1.0)
    return d, w


def ransac_1p(o1, o2, hyp, H, n_reweight=10, keep_frac=0.5):
    """o1: (M, 3) template feature points, o2: (M, 3) live feature points, hyp: reference ids.

    Returns a dict with
      mask  (M,) bool   preselected inliers
      what  (M,)        weight of each match (max over kept references)
      kept  (NH,) bool  kept references
      score (NH,)       sum_{k != k0} w_k per reference
      d, w  (NH, M)     final distances and weights per reference.
    Section 2.1, Eq. 2-4: 1-point RANSAC with reweighting and the preselection it gives."""
    o1 = np.asarray(o1, dtype=np.float64)
    o2 = np.asarray(o2, dtype=np.float64)
    NH = len(hyp)
    M = o1.shape[0]
    D = np.zeros((NH, M))
    Wt = np.zeros((NH, M))
    score = np.zeros(NH)
    for h, k0 in enumerate(hyp):
        S1 = o1 - o1[k0]          # Eq. 2, l = 1
        S2 = o2 - o2[k0]          # Eq. 2, l = 2
        d, w = reweight(S1, S2, H, n_reweight)
        D[h], Wt[h] = d, w
        score[h] = w.sum() - w[k0]
    kept = score >= keep_frac * score.max()
    mask = np.zeros(M, dtype=bool)
    what = np.zeros(M)
    for h in np.flatnonzero(kept):
        mask |= D[h] <= H
        what = np.maximum(what, Wt[h])
    return dict(mask=mask, what=what, kept=kept, score=score, d=D, w=Wt)
