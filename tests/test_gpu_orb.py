"""GPU parity of the uniform ORB features (Section 2.1) through the C ABI against the oracle:
keypoint lists, responses and descriptors bit-exact (integer work), orientation bins exact
outside a 1e-9 band around a bin edge (both sides decide the bin in FP64), matches exact, live
3D points within FP32 rounding, and the matches driving a whole frame solve."""
import ctypes

import numpy as np
import pytest

from gpu_common import COST_RTOL, POS_TOL_MM, lib, oracle_params
from oracle import orb, solver
from synth import CONFIGS, make_textured_scene, orb_pattern
from synth.scene import Config

pytestmark = pytest.mark.gpu

SMALL = Config("orb_160x120_n48", 160, 120, 48, 300, 8, 0.3, 0.5, 0.1, 8.0, 1.0, 0.5, 1.0, 1)


@pytest.fixture(scope="module")
def d():
    return lib()


@pytest.fixture(scope="module")
def pat():
    return orb_pattern(7)


@pytest.fixture(scope="module")
def full():
    return make_textured_scene(CONFIGS["seq_320x240_n256"], 1000, n_frames=1)


@pytest.fixture(scope="module")
def small():
    return make_textured_scene(SMALL, 55, n_frames=1)


def _near_edge(theta, nbins=32):
    x = np.asarray(theta) / (2 * np.pi / nbins)
    return np.abs(np.abs(x - np.floor(x)) - 0.5) < 1e-9


def _check_kp(g, o):
    assert np.array_equal(g["pix"], o["pix"])
    assert g["n_total"] == o["n_total"]
    assert np.array_equal(g["score"], o["score"])
    ok = ~_near_edge(o["theta"])
    assert np.array_equal(g["bin"][ok], o["bin"][ok])
    same = g["bin"] == o["bin"]
    assert np.array_equal(g["desc"][same], o["desc"][same])
    return bool(same.all())


def _detect(d, sc, pat, img, dep, prm=None):
    g = d.Orb(sc.W, sc.H, sc.K, pat, prm)
    g.detect(img, dep)
    return g, g.keypoints()


@pytest.mark.parametrize("which", ["small", "full", "large"])
def test_keypoints_and_descriptors_bit_exact(d, pat, which, small, full):
    if which == "large":
        ts = make_textured_scene(CONFIGS["seq_640x480_n1024"], 2000, n_frames=1)
    else:
        ts = small if which == "small" else full
    sc = ts.scene
    for img, dep in [(ts.template_image, sc.template_depth), (ts.images[0], sc.frames[0].depth)]:
        g, gk = _detect(d, sc, pat, img, dep)
        o = orb.detect(img, dep, pat)
        assert len(o["pix"]) > 100
        _check_kp(gk, o)
        g.close()


def test_without_depth_other_parameters_and_capacity(d, pat, full):
    sc = full.scene
    img = full.template_image
    g, gk = _detect(d, sc, pat, img, None)
    _check_kp(gk, orb.detect(img, None, pat))
    g.close()
    for kw in [dict(fast_t=5), dict(fast_t=60, border=24), dict(max_kp=100)]:
        g, gk = _detect(d, sc, pat, img, sc.template_depth, d.orb_default_params(**kw))
        o = orb.detect(img, sc.template_depth, pat, orb.OrbParams(**kw))
        _check_kp(gk, o)
        if "max_kp" in kw:
            assert len(gk["pix"]) == 100 and gk["n_total"] > 100
        g.close()


def test_flat_image_and_no_depth_give_no_keypoints(d, pat, small):
    sc = small.scene
    flat = np.full((sc.H, sc.W), 128, np.uint8)
    g, gk = _detect(d, sc, pat, flat, sc.template_depth)
    assert len(gk["pix"]) == 0 and gk["n_total"] == 0
    L, lk = _detect(d, sc, pat, small.images[0], np.zeros((sc.H, sc.W), np.float32))
    assert len(lk["pix"]) == 0
    m = L.match_from(g)
    assert len(m["t"]) == 0
    g.close()
    L.close()


@pytest.mark.parametrize("which", ["small", "full"])
def test_matches_bit_exact(d, pat, which, small, full):
    ts = small if which == "small" else full
    sc, fr = ts.scene, ts.scene.frames[0]
    T, tk = _detect(d, sc, pat, ts.template_image, sc.template_depth)
    L, lk = _detect(d, sc, pat, ts.images[0], fr.depth)
    oT = orb.detect(ts.template_image, sc.template_depth, pat)
    oL = orb.detect(ts.images[0], fr.depth, pat)
    if not (_check_kp(tk, oT) and _check_kp(lk, oL)):
        pytest.skip("an orientation exactly at a bin edge (listed): descriptors differ there")
    gm = L.match_from(T)
    om = orb.match_points(oT, oL, fr.depth, sc.K, 64)
    assert len(om["t"]) > 50
    assert np.array_equal(gm["t"], om["t"])
    assert np.array_equal(gm["l"], om["l"])
    assert np.array_equal(gm["dist"], om["dist"])
    assert np.array_equal(gm["tmpl_pix"], om["tmpl_pix"])
    assert np.abs(gm["xyz"] - om["xyz"]).max() <= 2e-5 * np.abs(om["xyz"]).max()
    # the same template object matched to itself: every keypoint is its own mutual nearest
    # at distance 0 unless an identical descriptor exists elsewhere (then the lower index wins)
    T2, _ = _detect(d, sc, pat, ts.template_image, sc.template_depth)
    self_m = T2.match_from(T2)
    assert np.all(self_m["dist"] == 0)
    assert len(self_m["t"]) >= 0.95 * len(tk["pix"])
    for o in (T, L, T2):
        o.close()


def test_errors(d, pat, small):
    sc = small.scene
    with pytest.raises(d.DsError) as e:
        d.Orb(30, 30, sc.K, pat)
    assert e.value.status == d.DS_ERR_ARG
    with pytest.raises(d.DsError):
        d.Orb(sc.W, sc.H, sc.K, pat, d.orb_default_params(border=10))
    bad = pat.copy()
    bad[5, 0] = 14.0
    with pytest.raises(d.DsError):
        d.Orb(sc.W, sc.H, sc.K, bad)
    T, _ = _detect(d, sc, pat, small.template_image, sc.template_depth)
    L = d.Orb(sc.W, sc.H, sc.K, pat)
    with pytest.raises(d.DsError) as e:
        d.ds_orb_match(T.o, L.o)               # nothing detected on the live side
    assert e.value.status == d.DS_ERR_STATE
    L.detect(small.images[0])                  # no live depth: no 3D points to return
    with pytest.raises(d.DsError) as e:
        d.ds_orb_match(T.o, L.o)
    assert e.value.status == d.DS_ERR_STATE
    other = d.Orb(sc.W + 8, sc.H, sc.K, pat)
    other.detect(np.zeros((sc.H, sc.W + 8), np.uint8), np.ones((sc.H, sc.W + 8), np.float32))
    with pytest.raises(d.DsError) as e:
        d.ds_orb_match(T.o, other.o)
    assert e.value.status == d.DS_ERR_ARG
    for o in (T, L, other):
        o.close()


def test_orb_matches_drive_a_frame_solve(d, pat, full):
    """Template and live features matched on the GPU, handed to ds_submit_frame as device
    pointers, solved; the oracle solves the same frame from the same matches."""
    sc, fr = full.scene, full.scene.frames[0]
    T, _ = _detect(d, sc, pat, full.template_image, sc.template_depth)
    L, _ = _detect(d, sc, pat, full.images[0], fr.depth)
    d.ds_orb_match(T.o, L.o)
    M = d.ds_orb_num_matches(L.o)
    assert M > 300
    pix_dev, xyz_dev = d.ds_orb_match_device(L.o)
    host = dict(pix=np.zeros(M, np.int32), xyz=np.zeros((M, 3), np.float32))
    d.ds_orb_get_matches(L.o, None, None, None, host["pix"], host["xyz"])
    hyp = np.random.default_rng(9).choice(M, size=30, replace=False).astype(np.int32)
    p = d.default_params(precision=2)
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    depth = np.ascontiguousarray(fr.depth, np.float32)
    rc = d.lib().ds_submit_frame(s.h, depth.ctypes.data, ctypes.c_void_p(pix_dev),
                                 ctypes.c_void_p(xyz_dev), M, hyp.ctypes.data)
    assert rc == d.DS_OK
    st = s.solve(10, stats=True)
    _, t = s.deformation64()
    prm = oracle_params(p)
    tpl = solver.setup_template(sc.template_depth, sc.K, sc.nodes, prm)
    res = solver.solve_frame(tpl, fr.depth, host["pix"], host["xyz"], hyp, prm, 10)
    assert np.abs(tpl.g + t - res.pos).max() <= POS_TOL_MM
    rel = np.abs(np.array(st.cost[:10]) - np.array(res.costs)) / np.array(res.costs)
    assert rel.max() <= COST_RTOL, rel
    # and the recovered control points are close to the generator's truth
    assert np.median(np.linalg.norm(res.pos - fr.node_truth, axis=1)) < 1.5
    s.close()
    T.close()
    L.close()
