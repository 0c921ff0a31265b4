"""Seeded synthetic scenes: depth templates, deformed target frames and ORB-like matches.

These arrays stand in for the stereo-derived templates and live frames of the paper's
experiments (Section 3), whose videos are not available. The module only builds inputs: a
smooth heightfield seen by a pinhole camera, a smooth non-rigid deformation plus a rigid camera
motion, ray-cast depth maps, noisy and outlier feature matches, the random reference list of the
1-point RANSAC (Section 2.1) and the control-point pixels. It contains none of the solve's
arithmetic (no back-projection of the method, no normals, no residuals, no Jacobians): both the
oracle and the CUDA path receive its arrays unchanged.

All geometry is in millimetres, in the camera frame (x right, y down, z forward).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


# ----------------------------------------------------------------------------- camera


def intrinsics_for(W: int, H: int) -> tuple[float, float, float, float]:
    """Pinhole intrinsics used for every workload: fx = fy = W (about 53 deg horizontal field
    of view) and the principal point at the image centre, pixel centres at integer (u, v)."""
    return float(W), float(W), (W - 1) / 2.0, (H - 1) / 2.0


# ----------------------------------------------------------------------------- surface


@dataclasses.dataclass
class Heightfield:
    """z = clip(base + tilt . (x, y) + sum_b a_b exp(-|(x,y) - mu_b|^2 / (2 s_b^2)), zmin, zmax)."""

    base: float
    tilt: np.ndarray          # (2,)
    amp: np.ndarray           # (B,)
    mu: np.ndarray            # (B, 2)
    sig: np.ndarray           # (B,)
    zmin: float = 50.0
    zmax: float = 150.0

    def eval(self, x: np.ndarray, y: np.ndarray):
        """Height and its two partial derivatives at lateral positions (x, y)."""
        z = self.base + self.tilt[0] * x + self.tilt[1] * y
        zx = np.full_like(x, self.tilt[0], dtype=np.float64)
        zy = np.full_like(x, self.tilt[1], dtype=np.float64)
        for a, (mx, my), s in zip(self.amp, self.mu, self.sig):
            dx = x - mx
            dy = y - my
            e = a * np.exp(-(dx * dx + dy * dy) / (2.0 * s * s))
            z = z + e
            zx = zx - e * dx / (s * s)
            zy = zy - e * dy / (s * s)
        clipped = (z < self.zmin) | (z > self.zmax)
        z = np.clip(z, self.zmin, self.zmax)
        zx = np.where(clipped, 0.0, zx)
        zy = np.where(clipped, 0.0, zy)
        return z, zx, zy


def random_heightfield(rng: np.random.Generator, n_bumps: int, width_mm: float = 100.0,
                       aspect: float = 0.75) -> Heightfield:
    """Sum of Gaussian bumps over the footprint seen at 100 mm depth (width 100 mm)."""
    half_w = width_mm / 2.0
    half_h = half_w * aspect
    amp = rng.uniform(-20.0, 20.0, n_bumps)
    mu = np.stack([rng.uniform(-half_w, half_w, n_bumps),
                   rng.uniform(-half_h, half_h, n_bumps)], axis=1)
    sig = rng.uniform(0.12, 0.25, n_bumps) * width_mm
    return Heightfield(100.0, np.zeros(2), amp, mu, sig)


def planar_heightfield(tilt=(0.15, -0.1), base: float = 100.0) -> Heightfield:
    return Heightfield(base, np.asarray(tilt, dtype=np.float64), np.zeros(0), np.zeros((0, 2)),
                       np.zeros(0), zmin=-1e30, zmax=1e30)


# ----------------------------------------------------------------------------- deformation


@dataclasses.dataclass
class Motion:
    """Target surface point = Rc (S + a * phi(S_xy) e_z) + Tc, where S = (x, y, h(x, y)) and
    phi is a unit Gaussian bump centred at mu with width s."""

    Rc: np.ndarray            # (3, 3)
    Tc: np.ndarray            # (3,)
    a: float                  # bump amplitude along the camera axis (mm)
    mu: np.ndarray            # (2,)
    s: float

    def surface(self, hf: Heightfield, x: np.ndarray, y: np.ndarray):
        """Deformed point Y(x, y) (..., 3) and its partial derivatives dY/dx, dY/dy."""
        z, zx, zy = hf.eval(x, y)
        dx = x - self.mu[0]
        dy = y - self.mu[1]
        ph = np.exp(-(dx * dx + dy * dy) / (2.0 * self.s * self.s))
        zz = z + self.a * ph
        zzx = zx - self.a * ph * dx / (self.s * self.s)
        zzy = zy - self.a * ph * dy / (self.s * self.s)
        P = np.stack([x, y, zz], axis=-1)
        Px = np.stack([np.ones_like(x), np.zeros_like(x), zzx], axis=-1)
        Py = np.stack([np.zeros_like(x), np.ones_like(x), zzy], axis=-1)
        Y = P @ self.Rc.T + self.Tc
        return Y, Px @ self.Rc.T, Py @ self.Rc.T


def axis_angle(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rotation matrix from a unit axis and an angle (Rodrigues)."""
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


# ----------------------------------------------------------------------------- rendering


def raycast_template(hf: Heightfield, W: int, H: int, iters: int = 40):
    """Depth map of the undeformed heightfield: per pixel, Newton on lambda = h(lambda d)
    along the ray d = ((u-cx)/fx, (v-cy)/fy, 1).  Returns (depth f64 (H, W), X0 f64 (H, W, 3));
    pixels where the iteration does not settle get depth 0."""
    fx, fy, cx, cy = intrinsics_for(W, H)
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    dx = (u - cx) / fx
    dy = (v - cy) / fy
    lam = np.full(u.shape, hf.base if np.isfinite(hf.base) else 100.0)
    # Newton per pixel; a pixel stops once |lambda - h| < 1e-12 (only the others are iterated)
    act = np.arange(lam.size)
    lf, dxf, dyf = lam.reshape(-1), dx.reshape(-1), dy.reshape(-1)
    for _ in range(iters):
        la, ax, ay = lf[act], dxf[act], dyf[act]
        z, zx, zy = hf.eval(la * ax, la * ay)
        f = la - z
        going = np.abs(f) >= 1e-12
        if not going.any():
            break
        act, la, f, ax, ay = act[going], la[going], f[going], ax[going], ay[going]
        df = 1.0 - (zx[going] * ax + zy[going] * ay)
        df = np.where(np.abs(df) < 0.2, np.sign(df + 1e-300) * 0.2, df)
        lf[act] = la - f / df
    lam = lf.reshape(u.shape)
    z, _, _ = hf.eval(lam * dx, lam * dy)
    ok = np.abs(lam - z) < 1e-9
    depth = np.where(ok, lam, 0.0)
    X0 = np.stack([lam * dx, lam * dy, lam], axis=-1)
    return depth, X0


def render_target(hf: Heightfield, mo: Motion, W: int, H: int, iters: int = 12,
                  return_xy: bool = False):
    """Depth map of the deformed, moved surface: per target pixel, 2D Newton over the surface
    parameters (x, y) until the projected point hits the pixel centre.  Pixels whose iteration
    does not settle to 1e-7 px, or whose point is behind the camera, get depth 0.  With
    return_xy, also the surface parameters (x, y) seen at each pixel."""
    fx, fy, cx, cy = intrinsics_for(W, H)
    up, vp = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    x = (up - cx) / fx * 100.0
    y = (vp - cy) / fy * 100.0
    # 2D Newton per pixel; a pixel stops once its projection is within 1e-10 px of its centre
    # (only the others are iterated)
    act = np.arange(x.size)
    xf, yf, uf, vf = x.reshape(-1), y.reshape(-1), up.reshape(-1), vp.reshape(-1)
    for _ in range(iters):
        xa, ya = xf[act], yf[act]
        Y, Yx, Yy = mo.surface(hf, xa, ya)
        iz = 1.0 / Y[..., 2]
        pu = fx * Y[..., 0] * iz + cx
        pv = fy * Y[..., 1] * iz + cy
        ru = pu - uf[act]
        rv = pv - vf[act]
        going = np.maximum(np.abs(ru), np.abs(rv)) >= 1e-10
        if not going.any():
            break
        act, xa, ya, ru, rv = act[going], xa[going], ya[going], ru[going], rv[going]
        Y, Yx, Yy, iz = Y[going], Yx[going], Yy[going], iz[going]
        # d(pu, pv)/dY
        du = np.stack([fx * iz, np.zeros_like(iz), -fx * Y[..., 0] * iz * iz], axis=-1)
        dv = np.stack([np.zeros_like(iz), fy * iz, -fy * Y[..., 1] * iz * iz], axis=-1)
        a11 = (du * Yx).sum(-1)
        a12 = (du * Yy).sum(-1)
        a21 = (dv * Yx).sum(-1)
        a22 = (dv * Yy).sum(-1)
        det = a11 * a22 - a12 * a21
        det = np.where(np.abs(det) < 1e-12, 1e-12, det)
        xf[act] = xa - (a22 * ru - a12 * rv) / det
        yf[act] = ya - (-a21 * ru + a11 * rv) / det
    x, y = xf.reshape(up.shape), yf.reshape(up.shape)
    Y, _, _ = mo.surface(hf, x, y)
    pu = fx * Y[..., 0] / Y[..., 2] + cx
    pv = fy * Y[..., 1] / Y[..., 2] + cy
    ok = (np.abs(pu - up) < 1e-7) & (np.abs(pv - vp) < 1e-7) & (Y[..., 2] > 1.0)
    if return_xy:
        return np.where(ok, Y[..., 2], 0.0), x, y
    return np.where(ok, Y[..., 2], 0.0)


def occlude(rng: np.random.Generator, depth: np.ndarray, frac: float) -> np.ndarray:
    """Zero the depth inside random discs until at least `frac` of the pixels are covered
    (instrument or smoke occlusion)."""
    H, W = depth.shape
    out = depth.copy()
    if frac <= 0:
        return out
    u, v = np.meshgrid(np.arange(W), np.arange(H))
    mask = np.zeros((H, W), dtype=bool)
    while mask.mean() < frac:
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        r = rng.uniform(0.03, 0.08) * W
        mask |= (u - cx) ** 2 + (v - cy) ** 2 <= r * r
    out[mask] = 0.0
    return out


# ----------------------------------------------------------------------------- control points


def control_point_pixels(depth: np.ndarray, N: int) -> np.ndarray:
    """N control-point pixel indices on a regular lattice over the image.

    The lattice is gx x gy with gx * gy = N and gx / gy closest to W / H in log ratio (tie:
    gx >= gy).  If no factor pair is within a factor 2 of the aspect (e.g. a prime N), the
    lattice is gy = round(sqrt(N H / W)) rows of gx = ceil(N / gy), filled row-major and cut
    to N.  Each node sits at the centre of its lattice cell; an invalid pixel moves to the
    nearest valid one (tie: lower pixel index)."""
    H, W = depth.shape
    best = None
    for gy in range(1, N + 1):
        if N % gy:
            continue
        gx = N // gy
        score = abs(math.log(gx / gy) - math.log(W / H))
        key = (score, -gx)
        if best is None or key < best[0]:
            best = (key, gx, gy)
    _, gx, gy = best
    if best[0][0] > math.log(2.0):
        gy = max(1, int(round(math.sqrt(N * H / W))))
        gx = -(-N // gy)
    cells = []
    for j in range(gy):
        for i in range(gx):
            if len(cells) < N:
                cells.append(((i + 0.5) * W / gx - 0.5, (j + 0.5) * H / gy - 0.5))
    valid = depth.reshape(-1) > 0
    vidx = np.flatnonzero(valid)
    vu = (vidx % W).astype(np.float64)
    vv = (vidx // W).astype(np.float64)
    out = []
    for (cu, cv) in cells:
        pu, pv = int(round(cu)), int(round(cv))
        pu = min(max(pu, 0), W - 1)
        pv = min(max(pv, 0), H - 1)
        p = pv * W + pu
        if not valid[p] or p in out:
            d2 = (vu - pu) ** 2 + (vv - pv) ** 2
            taken = np.isin(vidx, np.asarray(out, dtype=np.int64))
            d2 = np.where(taken, np.inf, d2)
            p = int(vidx[int(np.argmin(d2))])     # argmin: first (lowest index) on ties
        out.append(p)
    return np.asarray(out, dtype=np.int32)


# ----------------------------------------------------------------------------- workloads


@dataclasses.dataclass
class Frame:
    depth: np.ndarray          # (H, W) float32 (float64 when requested)
    match_idx: np.ndarray      # (M,) int32 template pixel index
    match_xyz: np.ndarray      # (M, 3) float32 target point
    hyp: np.ndarray            # (n_hyp,) int32 reference match ids
    inlier: np.ndarray         # (M,) bool, planted inliers (ground truth, not an input)
    node_truth: np.ndarray     # (N, 3) float64 true deformed control-point positions
    motion: Motion


@dataclasses.dataclass
class Scene:
    W: int
    H: int
    K: tuple
    template_depth: np.ndarray   # (H, W) float32 (float64 when requested)
    nodes: np.ndarray            # (N,) int32 control-point pixel indices
    hf: Heightfield
    X0: np.ndarray               # (H, W, 3) float64 generator-side surface points
    frames: list


@dataclasses.dataclass
class Config:
    name: str
    W: int
    H: int
    N: int
    M: int
    n_bumps: int
    outlier: float            # fraction of outlier matches
    noise: float              # inlier noise sigma (mm)
    occlusion: float          # fraction of occluded target pixels
    amp: float                # deformation amplitude (mm)
    freq_hz: float            # deformation frequency; 0 = a single static bump
    rot_deg: float            # rigid rotation (single frame) or random-walk step (sequence)
    trans_mm: float
    n_frames: int
    iters: int = 10
    n_hyp: int = 30
    planar: bool = False
    outlier_min_dist: float = 0.0


# The five workloads; names carry their sizes.
CONFIGS = {
    # single frame, template 80x60, 32 nodes, 200 matches (30% outliers), one 5 mm bump + 3 deg / 2 mm
    "frame_80x60_n32": Config("frame_80x60_n32", 80, 60, 32, 200, 5, 0.30, 0.0, 0.0, 5.0, 0.0,
                              3.0, 2.0, 1),
    # 300-frame sequence, 320x240, 256 nodes, 2000 matches (40% outliers, 0.5 mm noise), 10% occluded
    "seq_320x240_n256": Config("seq_320x240_n256", 320, 240, 256, 2000, 20, 0.40, 0.5, 0.10, 10.0,
                               1.0, 0.2, 0.5, 300),
    # 100-frame fast-deformation sequence, 640x480, 1024 nodes, 4000 matches (50% outliers)
    "seq_640x480_n1024": Config("seq_640x480_n1024", 640, 480, 1024, 4000, 20, 0.50, 0.5, 0.10, 15.0,
                                1.0, 0.2, 0.5, 100),
}


def _seq_motion(cfg: Config, rng: np.random.Generator, t: int, state: dict, mu: np.ndarray,
                s: float) -> Motion:
    if cfg.freq_hz == 0.0:
        R = axis_angle(random_unit(rng), math.radians(cfg.rot_deg))
        T = random_unit(rng) * cfg.trans_mm
        return Motion(R, T, cfg.amp, mu, s)
    # random-walk camera: rot_deg / trans_mm per frame, deformation a sin(2 pi f t / 15 fps)
    dR = axis_angle(random_unit(rng), math.radians(cfg.rot_deg))
    state["R"] = dR @ state["R"]
    state["T"] = state["T"] + random_unit(rng) * cfg.trans_mm
    a = cfg.amp * math.sin(2.0 * math.pi * cfg.freq_hz * t / 15.0)
    return Motion(state["R"].copy(), state["T"].copy(), a, mu, s)


def make_scene(cfg: Config, seed: int, n_frames: int | None = None, f64: bool = False,
               M: int | None = None, N: int | None = None) -> Scene:
    """Build the template and `n_frames` target frames of a workload from a seed."""
    rng = np.random.default_rng(seed)
    W, H = cfg.W, cfg.H
    N = cfg.N if N is None else N
    M = cfg.M if M is None else M
    hf = planar_heightfield() if cfg.planar else random_heightfield(rng, cfg.n_bumps)
    tdepth, X0 = raycast_template(hf, W, H)
    nodes = control_point_pixels(tdepth, N)
    valid_t = np.flatnonzero(tdepth.reshape(-1) > 0)
    mu = rng.uniform(-15.0, 15.0, 2)
    s = 25.0 if cfg.freq_hz > 0 else 20.0
    state = {"R": np.eye(3), "T": np.zeros(3)}
    frames = []
    nf = cfg.n_frames if n_frames is None else n_frames
    X0f = X0.reshape(-1, 3)
    for t in range(1, nf + 1):
        mo = _seq_motion(cfg, rng, t, state, mu, s)
        dep = render_target(hf, mo, W, H)
        dep = occlude(rng, dep, cfg.occlusion)
        # matches: distinct template pixels; planted inliers at the true target point + noise
        j = rng.choice(valid_t, size=M, replace=False).astype(np.int32)
        Yj, _, _ = mo.surface(hf, X0f[j, 0], X0f[j, 1])
        n_out = int(round(cfg.outlier * M))
        inl = np.ones(M, dtype=bool)
        inl[rng.choice(M, size=n_out, replace=False)] = False
        xyz = Yj + rng.normal(0.0, cfg.noise, (M, 3)) * (cfg.noise > 0)
        tv = dep.reshape(-1) > 0
        if tv.any():
            fx, fy, cx, cy = intrinsics_for(W, H)
            uu = np.arange(W * H) % W
            vv = np.arange(W * H) // W
            zz = dep.reshape(-1)
            P = np.stack([(uu - cx) * zz / fx, (vv - cy) * zz / fy, zz], axis=1)[tv]
            lo, hi = P.min(0), P.max(0)
        else:
            lo, hi = Yj.min(0), Yj.max(0)
        for k in np.flatnonzero(~inl):
            while True:
                o = rng.uniform(lo, hi)
                if np.linalg.norm(o - Yj[k]) >= cfg.outlier_min_dist:
                    break
            xyz[k] = o
        hyp = rng.choice(M, size=cfg.n_hyp, replace=False).astype(np.int32)
        gn = X0f[nodes]
        node_truth, _, _ = mo.surface(hf, gn[:, 0], gn[:, 1])
        dt = np.float64 if f64 else np.float32
        frames.append(Frame(dep.astype(dt), j, xyz.astype(dt), hyp, inl, node_truth, mo))
    dt = np.float64 if f64 else np.float32
    return Scene(W, H, intrinsics_for(W, H), tdepth.astype(dt), nodes, hf, X0, frames)


def seed_for(config_index: int, stream: int = 0) -> int:
    """Seed convention: config index x 1000 + stream id."""
    return config_index * 1000 + stream
