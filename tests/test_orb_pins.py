"""Pins of the ORB oracle (uniform FAST detection, steered binary descriptors, mutual-nearest
matching) to facts outside itself: brute-force definitions on small inputs, closed forms,
exact symmetries of the image grid and planted structure.  CPU only."""
import math

import numpy as np
import pytest

from oracle import orb
from synth import CONFIGS, make_textured_scene, orb_pattern


def _blocks(rng, H, W, cell=4, levels=(40, 90, 140, 200)):
    """Piecewise-constant image of random cells (corners at cell junctions)."""
    g = rng.choice(levels, size=(H // cell + 1, W // cell + 1))
    return np.kron(g, np.ones((cell, cell), dtype=np.int64))[:H, :W].astype(np.uint8)


def test_fast_circle_is_the_radius_3_digital_circle():
    c = orb.fast_circle()
    assert len(c) == 16 and len(set(c)) == 16
    for dx, dy in c:
        assert round(math.hypot(dx, dy)) == 3
    # the standard Bresenham circle of radius 3, and consecutive pixels touch (8-neighbours)
    assert set(c) == {(0, 3), (1, 3), (2, 2), (3, 1), (3, 0), (3, -1), (2, -2), (1, -3), (0, -3),
                      (-1, -3), (-2, -2), (-3, -1), (-3, 0), (-3, 1), (-2, 2), (-1, 3)}
    for k in range(16):
        (a, b), (p, q) = c[k], c[(k + 1) % 16]
        assert max(abs(a - p), abs(b - q)) == 1


def _fast_bruteforce(I, t):
    I = I.astype(np.int64)
    H, W = I.shape
    circ = orb.fast_circle()
    out = np.zeros((H, W), dtype=np.int64)
    for v in range(3, H - 3):
        for u in range(3, W - 3):
            p = I[v, u]
            vals = [I[v + dy, u + dx] for dx, dy in circ]
            corner = False
            for s in range(16):
                seg = [vals[(s + k) % 16] for k in range(9)]
                if all(x > p + t for x in seg) or all(x < p - t for x in seg):
                    corner = True
            if corner:
                sb = sum(x - p - t for x in vals if x > p + t)
                sd = sum(p - x - t for x in vals if x < p - t)
                out[v, u] = max(sb, sd)
    return out


def test_fast_scores_equal_the_segment_test_brute_force():
    rng = np.random.default_rng(41)
    img = _blocks(rng, 30, 34)
    img[rng.integers(0, 30, 20), rng.integers(0, 34, 20)] = rng.integers(0, 256, 20)
    for t in (10, 20, 45):
        s = orb.fast_scores(img, t)
        assert np.array_equal(s, _fast_bruteforce(img, t))
        assert (s > 0).sum() > 20


def test_fast_fires_at_the_corners_of_a_square_only():
    img = np.full((40, 40), 50, dtype=np.uint8)
    img[15:25, 15:25] = 200
    s = orb.fast_scores(img, 20)
    corners = [(15, 15), (24, 15), (15, 24), (24, 24)]       # (u, v) of the square's corner pixels
    hit = np.argwhere(s > 0)                                   # (v, u)
    assert len(hit) > 0
    for v, u in hit:
        assert min(max(abs(u - cu), abs(v - cv)) for cu, cv in corners) <= 2
    for cu, cv in corners:
        assert s[cv, cu] > 0
    for (u, v) in [(20, 15), (15, 20), (20, 24), (24, 20), (20, 20)]:   # edges, interior
        assert s[v, u] == 0
    # the response peaks at the corner pixel itself: suppression leaves exactly the 4 corners
    keep = orb.suppress(s, 3)
    assert sorted((int(u), int(v)) for v, u in np.argwhere(keep)) == sorted(corners)


def test_suppression_brute_force():
    rng = np.random.default_rng(42)
    H, W, B = 24, 30, 4
    sc = rng.integers(0, 4, (H, W)) * rng.integers(0, 2, (H, W))     # many ties and zeros
    depth = rng.uniform(size=(H, W)) > 0.1
    keep = orb.suppress(sc, B, depth)
    for v in range(H):
        for u in range(W):
            exp = sc[v, u] > 0 and B <= u < W - B and B <= v < H - B and depth[v, u]
            if exp:
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        if (dx or dy) and sc[v + dy, u + dx] > sc[v, u]:
                            exp = False
            assert keep[v, u] == exp


@pytest.mark.parametrize("bx,by", [(3, 0), (0, 2), (-2, 1), (1, -4), (-3, -3), (4, 1), (2, 3)])
def test_orientation_of_a_linear_ramp_is_its_gradient_direction(bx, by):
    """Over the symmetric disc sum x = sum xy = 0, so for I = a + bx x + by y the centroid
    moments are (bx, by) times sum x^2: theta = atan2(by, bx) exactly."""
    H = W = 41
    y, x = np.mgrid[0:H, 0:W]
    img = (128 + bx * (x - 20) + by * (y - 20)).astype(np.uint8)
    theta, b = orb.orientation(img, np.array([20 * W + 20]))
    phi = math.atan2(by, bx)
    assert abs(theta[0] - phi) < 1e-12
    assert b[0] == round(phi / (2 * math.pi / 32)) % 32


def _textured_crop(seed=1000, size=(100, 120)):
    ts = make_textured_scene(CONFIGS["seq_320x240_n256"], seed, n_frames=1)
    img = ts.template_image[60:60 + size[0], 90:90 + size[1]]
    return np.ascontiguousarray(img)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_descriptors_are_invariant_under_quarter_turns(k):
    """Rotating the image by k quarter turns moves every keypoint to the rotated pixel, adds
    8 k bins (mod 32, up to the direction convention) and leaves every descriptor unchanged."""
    img = _textured_crop()
    pat = orb_pattern(7)
    prm = orb.OrbParams(fast_t=20)
    a = orb.detect(img, None, pat, prm)
    rimg = np.ascontiguousarray(np.rot90(img, k))
    b = orb.detect(rimg, None, pat, prm)
    H, W = img.shape
    Wr = rimg.shape[1]
    # where np.rot90 sends pixel (u, v): rotate an index image the same way
    idx = np.rot90(np.arange(H * W).reshape(H, W), k).reshape(-1)
    where = np.empty(H * W, dtype=np.int64)
    where[idx] = np.arange(H * W)
    mapped = np.sort(where[a["pix"]])
    assert np.array_equal(mapped, b["pix"])
    assert len(a["pix"]) > 30
    order = np.argsort(where[a["pix"]])
    shift = (b["bin"] - a["bin"][order]) % 32
    assert np.all(shift == shift[0]) and shift[0] in ((8 * k) % 32, (-8 * k) % 32)
    assert np.array_equal(b["desc"], a["desc"][order])
    assert Wr == (W if k % 2 == 0 else H)


def test_descriptor_bits_brute_force():
    img = _textured_crop()
    pat = orb_pattern(7)
    d = orb.detect(img, None, pat)
    W = img.shape[1]
    I = img.astype(np.int64)
    for j in range(0, len(d["pix"]), max(1, len(d["pix"]) // 12)):
        p = d["pix"][j]
        u, v = p % W, p // W
        phi = 2 * math.pi * d["bin"][j] / 32
        for i in range(256):
            ax, ay, bx, by = pat[i]
            pa = (round_half_even(ax * math.cos(phi) - ay * math.sin(phi)),
                  round_half_even(ax * math.sin(phi) + ay * math.cos(phi)))
            pb = (round_half_even(bx * math.cos(phi) - by * math.sin(phi)),
                  round_half_even(bx * math.sin(phi) + by * math.cos(phi)))
            sa = I[v + pa[1] - 2:v + pa[1] + 3, u + pa[0] - 2:u + pa[0] + 3].sum()
            sb = I[v + pb[1] - 2:v + pb[1] + 3, u + pb[0] - 2:u + pb[0] + 3].sum()
            bit = (int(d["desc"][j, i // 32]) >> (i % 32)) & 1
            assert bit == int(sa < sb)


def round_half_even(x):
    return int(round(x))       # Python's round is half-to-even


def test_matching_brute_force_with_ties():
    rng = np.random.default_rng(43)
    Dt = rng.integers(0, 2**32, (40, 8), dtype=np.uint64).astype(np.uint32)
    Dl = rng.integers(0, 2**32, (35, 8), dtype=np.uint64).astype(np.uint32)
    Dl[3] = Dl[9] = Dt[5]                    # a tie on the live side
    Dt[7] = Dt[12] = Dl[20]                  # and on the template side
    Dl[30] = Dt[1]                           # a near copy: 3 bits flipped
    Dl[30, 0] ^= np.uint32(0b1011)
    ti, li, dist = orb.match(Dt, Dl, 100)
    def ham(a, b):
        return sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b))
    D = np.array([[ham(a, b) for b in Dl] for a in Dt])
    exp = []
    for t in range(len(Dt)):
        l = min(range(len(Dl)), key=lambda j: (D[t, j], j))
        t2 = min(range(len(Dt)), key=lambda i: (D[i, l], i))
        if t2 == t and D[t, l] <= 100:
            exp.append((t, l, D[t, l]))
    assert [tuple(x) for x in zip(ti, li, dist)] == exp
    assert (5, 3, 0) in exp and (7, 20, 0) in exp and (1, 30, 3) in exp
    assert not any(t == 12 for t, _, _ in exp)


def test_a_shifted_image_matches_every_keypoint_to_its_shifted_pixel():
    ts = make_textured_scene(CONFIGS["seq_320x240_n256"], 1000, n_frames=1)
    big = ts.template_image
    dx, dy = 7, -5
    a = np.ascontiguousarray(big[40:200, 60:260])
    b = np.ascontiguousarray(big[40 + dy:200 + dy, 60 + dx:260 + dx])   # b(u, v) = a(u + dx, v + dy)
    pat = orb_pattern(7)
    A = orb.detect(a, None, pat)
    Bk = orb.detect(b, None, pat)
    ti, li, dist = orb.match(A["desc"], Bk["desc"], 64)
    W = a.shape[1]
    ua, va = A["pix"][ti] % W, A["pix"][ti] // W
    ub, vb = Bk["pix"][li] % W, Bk["pix"][li] // W
    exact = (ub == ua - dx) & (vb == va - dy) & (dist == 0)
    # keypoints of a whose shifted position is a keypoint of b
    inside = set(zip(Bk["pix"] % W + dx, Bk["pix"] // W + dy))
    common = sum((u, v) in inside for u, v in zip(A["pix"] % W, A["pix"] // W))
    assert common > 200
    assert exact.sum() >= 0.95 * common


def test_matches_of_a_deformed_frame_land_on_the_true_points():
    """End to end on a synthetic frame: most mutual matches put the live 3D point within 2 mm of
    where the generator moved the matched template point."""
    ts = make_textured_scene(CONFIGS["seq_320x240_n256"], 1000, n_frames=1)
    sc, fr = ts.scene, ts.scene.frames[0]
    pat = orb_pattern(7)
    T = orb.detect(ts.template_image, sc.template_depth, pat)
    L = orb.detect(ts.images[0], fr.depth, pat)
    m = orb.match_points(T, L, fr.depth, sc.K, 64)
    X0 = sc.X0.reshape(-1, 3)
    Y, _, _ = fr.motion.surface(sc.hf, X0[m["tmpl_pix"], 0], X0[m["tmpl_pix"], 1])
    err = np.linalg.norm(Y - m["xyz"], axis=1)
    assert len(err) > 400
    assert (err < 2.0).mean() > 0.8
    assert np.all(np.asarray(sc.template_depth).reshape(-1)[m["tmpl_pix"]] > 0)


def test_detection_is_invariant_to_an_intensity_offset():
    """FAST compares differences, the centroid's moments of a constant vanish over the symmetric
    disc and both box sums of a test gain the same amount: adding a constant to an image (with
    no clipping) changes no keypoint, response, bin or descriptor bit."""
    img = _textured_crop().astype(np.int64)
    img = np.clip(img, 0, 200).astype(np.uint8)
    pat = orb_pattern(7)
    a = orb.detect(img, None, pat)
    b = orb.detect((img.astype(np.int64) + 37).astype(np.uint8), None, pat)
    assert len(a["pix"]) > 30
    assert np.array_equal(a["pix"], b["pix"]) and np.array_equal(a["score"], b["score"])
    assert np.array_equal(a["bin"], b["bin"]) and np.array_equal(a["desc"], b["desc"])


def test_box_sums_and_hamming_distances_brute_force():
    """The descriptor's 5 x 5 box sums and the matcher's Hamming distance against their plain
    definitions: explicit 25-pixel sums (0 where the box leaves the image) and bit counts of the
    XOR of every word pair."""
    rng = np.random.default_rng(33)
    img = rng.integers(0, 256, (11, 13), dtype=np.uint8)
    S = orb.box5(img)
    H, W = img.shape
    for v in range(H):
        for u in range(W):
            if 2 <= v < H - 2 and 2 <= u < W - 2:
                want = sum(int(img[v + dy, u + dx]) for dy in range(-2, 3) for dx in range(-2, 3))
            else:
                want = 0
            assert S[v, u] == want, (v, u)
    D1 = rng.integers(0, 2**32, (7, 8), dtype=np.uint64).astype(np.uint32)
    D2 = rng.integers(0, 2**32, (5, 8), dtype=np.uint64).astype(np.uint32)
    Hd = orb.hamming(D1, D2, rows=3)
    for i in range(7):
        for j in range(5):
            assert Hd[i, j] == sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(D1[i], D2[j]))
