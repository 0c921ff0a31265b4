"""Uniform ORB features and template-to-live matching (Section 2.1, first paragraph) — oracle.

Test infrastructure only (like the rest of oracle/): a plain numpy restatement the CUDA path
is compared against.

The paper names the parts and the one change it makes: FAST corners are detected on the GPU
and a corner is suppressed when a neighbouring pixel has a larger corner response, so that
features spread over the low-texture areas instead of gathering in the textured ones; the
template's ORB features are then matched to each live image, giving the two 3D point sets of
Eq. 2.  Readings where the paper is silent (the CUDA path implements the same):

* images are 8-bit grey levels;
* FAST-9 (Rosten & Drummond): the 16 pixels of the digital circle of radius 3 (the lattice
  points whose distance from the centre rounds to 3), in angular order; p is a corner iff 9
  cyclically contiguous circle pixels are all brighter than I_p + t or all darker than I_p - t;
* corner response, the score of the same authors: V = max(sum over brighter pixels of
  (I_c - I_p - t), sum over darker pixels of (I_p - I_c - t)), 0 for a non-corner;
* suppression: a corner is dropped iff one of its 8 neighbours has a strictly larger response
  (equal responses both survive); keypoints lie at least `border` pixels from every image edge
  and, when a depth map is given, on pixels of positive depth (a feature needs a 3D point);
  keypoints are listed in ascending pixel order, the first `max_kp` kept;
* orientation (ORB's intensity centroid): m10 = sum x I, m01 = sum y I over the disc of radius
  15 around the keypoint, theta = atan2(m01, m10), quantised to `nbins` = 32 directions:
  bin = rint(theta / (2 pi / 32)) mod 32 (32 rather than ORB's customary 30 makes a quarter
  turn a whole number of bins);
* descriptor (steered BRIEF): 256 binary tests; test i compares the 5 x 5 box sums S at the two
  points of pair i of the test pattern (an input), rotated by the bin's angle and rounded to
  the nearest integer offset (ties to even): bit i = S(p + a_i) < S(p + b_i).  Bit i is bit
  i mod 32 of 32-bit word i / 32;
* matching: Hamming distances; template keypoint t and live keypoint l match iff l is t's
  nearest live descriptor, t is l's nearest template descriptor (ties to the lower index) and
  the distance is <= max_dist; matches are listed in ascending t;
* the 3D points: the template pixel of the match (its template point, o1 of Eq. 2) and the
  live keypoint back-projected by the live depth, ((u - cx) z / fx, (v - cy) z / fy, z) (o2).
"""
import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class OrbParams:
    fast_t: int = 20
    border: int = 16
    nbins: int = 32
    max_dist: int = 64
    max_kp: int = 1 << 30


def fast_circle():
    """The 16 offsets (dx, dy) of the radius-3 digital circle in increasing angle.
    Section 2.1: FAST corners."""
    pts = [(dx, dy) for dy in range(-3, 4) for dx in range(-3, 4)
           if round(math.hypot(dx, dy)) == 3]
    pts.sort(key=lambda p: math.atan2(p[1], p[0]))
    return pts


def fast_scores(img, t):
    """FAST-9 response of every pixel (int64 (H, W)); 0 for non-corners and for pixels whose
    circle leaves the image.
    Section 2.1: FAST corners and their responses."""
    I = np.asarray(img, dtype=np.int64)
    H, W = I.shape
    out = np.zeros((H, W), dtype=np.int64)
    if H < 7 or W < 7:
        return out
    c = I[3:H - 3, 3:W - 3]
    ring = [I[3 + dy:H - 3 + dy, 3 + dx:W - 3 + dx] for dx, dy in fast_circle()]
    bright = [r > c + t for r in ring]
    dark = [r < c - t for r in ring]
    corner = np.zeros_like(c, dtype=bool)
    for s in range(16):
        run_b = np.ones_like(corner)
        run_d = np.ones_like(corner)
        for k in range(9):
            run_b &= bright[(s + k) % 16]
            run_d &= dark[(s + k) % 16]
        corner |= run_b | run_d
    sb = sum(np.where(b, r - c - t, 0) for b, r in zip(bright, ring))
    sd = sum(np.where(d, c - r - t, 0) for d, r in zip(dark, ring))
    out[3:H - 3, 3:W - 3] = np.where(corner, np.maximum(sb, sd), 0)
    return out


def suppress(score, border, depth=None):
    """Keep mask of the uniform detection (see the module notes).
    Section 2.1: a corner is dropped when a neighbour has a larger response."""
    H, W = score.shape
    keep = score > 0
    inner = np.zeros_like(keep)
    if H > 2 * border and W > 2 * border:
        inner[border:H - border, border:W - border] = True
    keep &= inner
    pad = np.pad(score, 1)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dx or dy:
                keep &= pad[1 + dy:1 + dy + H, 1 + dx:1 + dx + W] <= score
    if depth is not None:
        keep &= np.asarray(depth) > 0
    return keep


def disc_offsets(radius=15):
    """The patch of ORB's intensity-centroid orientation (Section 2.1 uses ORB features)."""
    return [(dx, dy) for dy in range(-radius, radius + 1) for dx in range(-radius, radius + 1)
            if dx * dx + dy * dy <= radius * radius]


def orientation(img, pix, nbins=32):
    """(theta, bin) of each keypoint pixel.
    Section 2.1 (ORB features): intensity-centroid orientation."""
    I = np.asarray(img, dtype=np.int64)
    H, W = I.shape
    u = np.asarray(pix) % W
    v = np.asarray(pix) // W
    m10 = np.zeros(len(u), dtype=np.int64)
    m01 = np.zeros(len(u), dtype=np.int64)
    for dx, dy in disc_offsets():
        val = I[v + dy, u + dx]
        m10 += dx * val
        m01 += dy * val
    theta = np.arctan2(m01.astype(np.float64), m10.astype(np.float64))
    step = 2.0 * np.pi / nbins
    b = np.rint(theta / step).astype(np.int64) % nbins
    return theta, b


def rotated_pattern(pattern, nbins=32):
    """Integer test offsets (nbins, 256, 4): the pattern rotated by 2 pi k / nbins, rounded.
    Section 2.1 (ORB features): the steered test pattern."""
    pattern = np.asarray(pattern, dtype=np.float64)
    out = np.zeros((nbins, pattern.shape[0], 4), dtype=np.int64)
    for k in range(nbins):
        phi = 2.0 * np.pi * k / nbins
        c, s = np.cos(phi), np.sin(phi)
        for j in (0, 2):
            x, y = pattern[:, j], pattern[:, j + 1]
            out[k, :, j] = np.rint(x * c - y * s)
            out[k, :, j + 1] = np.rint(x * s + y * c)
    return out


def box5(img):
    """5 x 5 box sums (int64 (H, W)), 0 within 2 pixels of the edge.
    Section 2.1 (ORB features): the smoothed intensities the binary tests compare."""
    I = np.asarray(img, dtype=np.int64)
    H, W = I.shape
    out = np.zeros((H, W), dtype=np.int64)
    acc = np.zeros((H - 4, W - 4), dtype=np.int64)
    for dy in range(5):
        for dx in range(5):
            acc += I[dy:H - 4 + dy, dx:W - 4 + dx]
    out[2:H - 2, 2:W - 2] = acc
    return out


def descriptors(img, pix, bins, pattern, nbins=32):
    """(K, 8) uint32 steered binary descriptors.
    Section 2.1 (ORB features): steered binary descriptors."""
    W = img.shape[1]
    S = box5(img)
    tab = rotated_pattern(pattern, nbins)[np.asarray(bins)]       # (K, 256, 4)
    u = (np.asarray(pix) % W)[:, None]
    v = (np.asarray(pix) // W)[:, None]
    sa = S[v + tab[:, :, 1], u + tab[:, :, 0]]
    sb = S[v + tab[:, :, 3], u + tab[:, :, 2]]
    bits = (sa < sb).astype(np.uint64)                            # (K, 256)
    words = np.zeros((len(pix), 8), dtype=np.uint64)
    for i in range(256):
        words[:, i // 32] |= bits[:, i] << np.uint64(i % 32)
    return words.astype(np.uint32)


def detect(img, depth, pattern, prm: OrbParams = OrbParams()):
    """Keypoints of one image: dict with pix (ascending), score, theta, bin, desc.
    Section 2.1: uniform ORB detection and description of one image."""
    sc = fast_scores(img, prm.fast_t)
    keep = suppress(sc, prm.border, depth)
    pix = np.flatnonzero(keep)[:prm.max_kp]
    n_total = int(keep.sum())
    theta, b = orientation(img, pix, prm.nbins)
    desc = descriptors(img, pix, b, pattern, prm.nbins)
    return dict(pix=pix, score=sc.reshape(-1)[pix], theta=theta, bin=b, desc=desc,
                n_total=n_total)


_POP8 = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint16)


def hamming(D1, D2, rows=128):
    """(n1, n2) Hamming distances between two sets of 256-bit descriptors (popcount of the XOR;
    evaluated `rows` descriptors of D1 at a time to bound memory).
    Section 2.1: the distance the template and live features are matched by."""
    D1 = np.ascontiguousarray(D1, np.uint32)
    D2 = np.ascontiguousarray(D2, np.uint32)
    out = np.empty((len(D1), len(D2)), dtype=np.int64)
    for a in range(0, len(D1), rows):
        x = np.bitwise_xor(D1[a:a + rows, None, :], D2[None, :, :])
        out[a:a + rows] = _POP8[x.view(np.uint8)].sum(-1)
    return out


def match(Dt, Dl, max_dist):
    """Mutual nearest neighbours within max_dist: (t index, l index, distance), ascending t.
    Section 2.1: template features matched to a live frame."""
    if len(Dt) == 0 or len(Dl) == 0:
        e = np.zeros(0, dtype=np.int64)
        return e, e.copy(), e.copy()
    d = hamming(Dt, Dl)
    bt = np.argmin(d, axis=1)          # first minimum: the lower index on ties
    bl = np.argmin(d, axis=0)
    t = np.arange(len(Dt))
    ok = (bl[bt] == t) & (d[t, bt] <= max_dist)
    ti = t[ok]
    return ti, bt[ok], d[ti, bt[ok]]


def match_points(tmpl, live, live_depth, K, max_dist):
    """The matches as the solve's inputs: template pixel per match and the live 3D point.
    Eq. 2: the matched 3D points o1 (template) and o2 (live)."""
    ti, li, dist = match(tmpl["desc"], live["desc"], max_dist)
    fx, fy, cx, cy = (float(k) for k in K)
    W = np.asarray(live_depth).shape[1]
    lp = live["pix"][li]
    z = np.asarray(live_depth, dtype=np.float64).reshape(-1)[lp]
    xyz = np.stack([((lp % W) - cx) * z / fx, ((lp // W) - cy) * z / fy, z], axis=1)
    return dict(t=ti, l=li, dist=dist, tmpl_pix=tmpl["pix"][ti], xyz=xyz)
