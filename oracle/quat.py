"""Quaternion algebra in (w, x, y, z) order, float64.

Product: (a0, a) (x) (b0, b) = (a0 b0 - a.b, a0 b + b0 a + a x b).
"""
import numpy as np


def qmul(a, b):
    """Hamilton product, broadcasting over leading axes.
    Quaternion algebra of Section 2's dual-quaternion warp."""
    a0, a1, a2, a3 = np.moveaxis(np.asarray(a, dtype=np.float64), -1, 0)
    b0, b1, b2, b3 = np.moveaxis(np.asarray(b, dtype=np.float64), -1, 0)
    return np.stack([a0 * b0 - a1 * b1 - a2 * b2 - a3 * b3,
                     a0 * b1 + a1 * b0 + a2 * b3 - a3 * b2,
                     a0 * b2 - a1 * b3 + a2 * b0 + a3 * b1,
                     a0 * b3 + a1 * b2 - a2 * b1 + a3 * b0], axis=-1)


def qconj(q):
    """Quaternion conjugate (algebra of Section 2's dual-quaternion warp)."""
    q = np.asarray(q, dtype=np.float64)
    return q * np.array([1.0, -1.0, -1.0, -1.0])


CONJ = np.diag([1.0, -1.0, -1.0, -1.0])


def qL(a):
    """Left-product matrix: a (x) b = qL(a) @ b.  Shape (..., 4, 4).
    Quaternion algebra of Section 2's dual-quaternion warp."""
    a0, a1, a2, a3 = np.moveaxis(np.asarray(a, dtype=np.float64), -1, 0)
    return np.stack([np.stack([a0, -a1, -a2, -a3], -1),
                     np.stack([a1, a0, -a3, a2], -1),
                     np.stack([a2, a3, a0, -a1], -1),
                     np.stack([a3, -a2, a1, a0], -1)], axis=-2)


def qR(b):
    """Right-product matrix: a (x) b = qR(b) @ a.  Shape (..., 4, 4).
    Quaternion algebra of Section 2's dual-quaternion warp."""
    b0, b1, b2, b3 = np.moveaxis(np.asarray(b, dtype=np.float64), -1, 0)
    return np.stack([np.stack([b0, -b1, -b2, -b3], -1),
                     np.stack([b1, b0, b3, -b2], -1),
                     np.stack([b2, -b3, b0, b1], -1),
                     np.stack([b3, b2, -b1, b0], -1)], axis=-2)


def pure(v):
    """Embed 3-vectors as pure quaternions (0, v).
    Quaternion algebra of Section 2's dual-quaternion warp."""
    v = np.asarray(v, dtype=np.float64)
    return np.concatenate([np.zeros(v.shape[:-1] + (1,)), v], axis=-1)


def rotmat(q):
    """Rotation matrix of a unit quaternion: R v = vec(q (x) (0, v) (x) q*).
    Quaternion algebra of Section 2's dual-quaternion warp."""
    q = np.asarray(q, dtype=np.float64)
    w, x, y, z = np.moveaxis(q, -1, 0)
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)],
                    axis=-2)


def qexp_half(theta):
    """Unit quaternion of the rotation vector theta: (cos(|theta|/2), sin(|theta|/2) theta/|theta|).
    The rotation increment of Section 2's Gauss-Newton step."""
    theta = np.asarray(theta, dtype=np.float64)
    a = np.linalg.norm(theta, axis=-1)
    safe = np.where(a > 0, a, 1.0)
    s = np.where(a > 0, np.sin(a / 2) / safe, 0.5)
    return np.concatenate([np.cos(a / 2)[..., None], s[..., None] * theta], axis=-1)


def skew(v):
    """[v]x with [v]x u = v x u.  Shape (..., 3, 3).
    Cross-product matrix (algebra of Section 2's warp Jacobians)."""
    v = np.asarray(v, dtype=np.float64)
    z = np.zeros(v.shape[:-1])
    x, y, w = np.moveaxis(v, -1, 0)
    return np.stack([np.stack([z, -w, y], -1),
                     np.stack([w, z, -x], -1),
                     np.stack([-y, x, z], -1)], axis=-2)
