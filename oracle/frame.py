"""Depth map -> 3D points and normals (oracle, float64).

The ICP term keeps only the distance along the normal direction of the live surface (Section 2,
the point-to-plane remark of the ICP paragraph); the normals are central finite differences of
the back-projected point map.
"""
import numpy as np


def backproject(depth, K):
    """X(u, v) = ((u - cx) z / fx, (v - cy) z / fy, z); valid where z > 0 and finite.

    depth: (H, W) array (any float dtype, widened to float64).  K = (fx, fy, cx, cy).
    Returns X (H, W, 3) float64 and valid (H, W) bool.
    Section 2: the point maps of the template and of the live depth."""
    fx, fy, cx, cy = (float(k) for k in K)
    z = np.asarray(depth, dtype=np.float64)
    H, W = z.shape
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    x = (u - cx) * z / fx
    y = (v - cy) * z / fy
    X = np.stack([x, y, z], axis=-1)
    valid = np.isfinite(z) & (z > 0)
    return X, valid


def target_normals(X, valid):
    """Central-difference normals n = c / |c|, c = (X(u+1,v) - X(u-1,v)) x (X(u,v+1) - X(u,v-1)),
    flipped so that n_z <= 0 (toward the camera).  A pixel is usable when it and its four
    neighbours are valid, it is not on the image border and |c| > 0.

    Returns n (H, W, 3) and usable (H, W) bool.
    Section 2, ICP paragraph: the normals of the point-to-plane distance."""
    H, W, _ = X.shape
    n = np.zeros_like(X)
    ok = np.zeros((H, W), dtype=bool)
    du = X[1:-1, 2:] - X[1:-1, :-2]
    dv = X[2:, 1:-1] - X[:-2, 1:-1]
    c = np.cross(du, dv)
    cn = np.linalg.norm(c, axis=-1)
    inner = (valid[1:-1, 1:-1] & valid[1:-1, 2:] & valid[1:-1, :-2] & valid[2:, 1:-1]
             & valid[:-2, 1:-1] & (cn > 0))
    safe = np.where(cn > 0, cn, 1.0)
    nn = c / safe[..., None]
    nn = np.where((nn[..., 2] > 0)[..., None], -nn, nn)
    n[1:-1, 1:-1] = np.where(inner[..., None], nn, 0.0)
    ok[1:-1, 1:-1] = inner
    return n, ok
