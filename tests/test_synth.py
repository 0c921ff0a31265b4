"""The seeded input generator (CPU): what the parity tests and the benchmark feed both sides must
be what it claims to be, independently of the solve.  Template rays land on the analytic
surface, planted inliers sit on the moved surface, outliers keep their stated distance,
references and match pixels are distinct, occlusion covers the stated fraction, and a seed
reproduces its scene exactly."""
import numpy as np

from synth import CONFIGS, make_scene
from synth.scene import Config, intrinsics_for


def test_template_rays_land_on_the_heightfield():
    sc = make_scene(CONFIGS["frame_80x60_n32"], 1000, f64=True)
    fx, fy, cx, cy = intrinsics_for(sc.W, sc.H)
    z = sc.template_depth
    ok = z > 0
    assert ok.mean() > 0.99
    v, u = np.nonzero(ok)
    x = (u - cx) * z[ok] / fx
    y = (v - cy) * z[ok] / fy
    h, _, _ = sc.hf.eval(x, y)
    assert np.abs(h - z[ok]).max() < 1e-9
    assert np.abs(sc.X0[ok][:, 2] - z[ok]).max() == 0.0


def test_matches_inliers_outliers_and_references():
    cfg = Config("noise_free", 80, 60, 32, 300, 5, 0.4, 0.0, 0.1, 5.0, 0.0, 3.0, 2.0, 1,
                 outlier_min_dist=20.0)
    sc = make_scene(cfg, 5, f64=True)
    f = sc.frames[0]
    assert len(np.unique(f.match_idx)) == len(f.match_idx)
    assert np.all(sc.template_depth.reshape(-1)[f.match_idx] > 0)
    assert len(np.unique(f.hyp)) == len(f.hyp) == cfg.n_hyp
    assert np.all((f.hyp >= 0) & (f.hyp < cfg.M))
    assert (~f.inlier).sum() == round(cfg.outlier * cfg.M)
    X0 = sc.X0.reshape(-1, 3)[f.match_idx]
    Y, _, _ = f.motion.surface(sc.hf, X0[:, 0], X0[:, 1])
    d = np.linalg.norm(f.match_xyz - Y, axis=1)
    assert d[f.inlier].max() == 0.0
    assert d[~f.inlier].min() >= cfg.outlier_min_dist


def test_occlusion_fraction_and_reproducibility():
    cfg = CONFIGS["seq_320x240_n256"]
    a = make_scene(cfg, 1000, n_frames=2)
    b = make_scene(cfg, 1000, n_frames=2)
    c = make_scene(cfg, 1001, n_frames=1)
    assert np.array_equal(a.template_depth, b.template_depth)
    for fa, fb in zip(a.frames, b.frames):
        assert np.array_equal(fa.depth, fb.depth)
        assert np.array_equal(fa.match_idx, fb.match_idx)
        assert np.array_equal(fa.match_xyz, fb.match_xyz)
        assert np.array_equal(fa.hyp, fb.hyp)
    assert not np.array_equal(a.frames[0].match_idx, c.frames[0].match_idx)
    empty = (a.frames[0].depth == 0).mean()
    assert cfg.occlusion * 0.8 <= empty <= cfg.occlusion * 1.5 + 0.05


def test_live_pixels_see_the_moved_surface_and_its_texture():
    """Each live pixel with depth sees the moved surface point whose lateral coordinates it
    reports: that point projects back onto the pixel, its depth is the pixel's, and the pixel's
    grey level is the texture there."""
    from synth import make_textured_scene
    from synth.texture import to_u8
    ts = make_textured_scene(CONFIGS["frame_80x60_n32"], 1000, n_frames=1, f64=True)
    sc, fr = ts.scene, ts.scene.frames[0]
    fx, fy, cx, cy = sc.K
    dep = np.asarray(fr.depth)
    ok = dep > 0
    xy = ts.live_xy[0]
    Y, _, _ = fr.motion.surface(sc.hf, xy[..., 0][ok], xy[..., 1][ok])
    v, u = np.nonzero(ok)
    assert np.abs(fx * Y[:, 0] / Y[:, 2] + cx - u).max() < 1e-6
    assert np.abs(fy * Y[:, 1] / Y[:, 2] + cy - v).max() < 1e-6
    assert np.abs(Y[:, 2] - dep[ok]).max() < 1e-6
    assert np.array_equal(ts.images[0], to_u8(ts.texture.eval(xy[..., 0], xy[..., 1]), ok))
