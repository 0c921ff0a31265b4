"""The allocation-free RANSAC entry point (ds_ransac_noalloc) gives the same preselection as the
handle path (ds_submit_frame + ds_get_inlier_mask / ds_get_ransac) on two calls in a row.

It exists for callers that cannot allocate device memory (a host process confined to a
pre-sized memory pool, or a real-time loop that must not block on an allocation); its working
memory is one fixed array inside the library. This file is collected last on purpose."""
import numpy as np
import pytest

from gpu_common import MID, lib, unpack_bits
from synth import CONFIGS, make_scene

pytestmark = pytest.mark.gpu


def _handle_path(d, sc, fr, p):
    s = d.Solver(sc.template_depth, sc.K, sc.nodes, p)
    s.submit(fr.depth, fr.match_idx, fr.match_xyz, fr.hyp)
    M = len(fr.match_idx)
    bits = np.zeros((M + 31) // 32, np.uint32)
    d.ds_get_inlier_mask(s.h, bits)
    w = np.zeros(M, np.float32)
    kept = np.zeros(2, np.uint32)
    score = np.zeros(p.n_hyp, np.float64)
    d.ds_get_ransac(s.h, w, kept, score)
    s.close()
    return bits, w, kept, score


def test_noalloc_ransac_matches_handle_path_twice():
    torch = pytest.importorskip("torch")
    d = lib()
    p = d.default_params()
    dev = torch.device("cuda", 0)
    for sc in (make_scene(CONFIGS["frame_80x60_n32"], 1000), make_scene(MID, 4242)):
        fr = sc.frames[0]
        M = len(fr.match_idx)
        ref_bits, ref_w, ref_kept, ref_score = _handle_path(d, sc, fr, p)
        depth0 = torch.from_numpy(np.ascontiguousarray(sc.template_depth, np.float32)).to(dev)
        midx = torch.from_numpy(fr.match_idx).to(dev)
        mxyz = torch.from_numpy(np.ascontiguousarray(fr.match_xyz, np.float32)).to(dev)
        hyp = torch.from_numpy(fr.hyp).to(dev)
        bits = torch.zeros((M + 31) // 32, dtype=torch.int32, device=dev)
        w = torch.zeros(M, dtype=torch.float32, device=dev)
        kept = torch.zeros(2, dtype=torch.int32, device=dev)
        score = torch.zeros(p.n_hyp, dtype=torch.float64, device=dev)
        d.ds_ransac_noalloc(depth0, sc.W, sc.H, sc.K, midx, mxyz, M, hyp, p.n_hyp, p.n_reweight,
                            p.H_mm, p.keep_frac, bits, w, kept, score)
        got_bits = bits.cpu().numpy().view(np.uint32)
        assert np.array_equal(unpack_bits(got_bits, M), unpack_bits(ref_bits, M))
        assert np.array_equal(kept.cpu().numpy().view(np.uint32), ref_kept)
        assert np.abs(w.cpu().numpy() - ref_w).max() <= 1e-6
        assert np.abs(score.cpu().numpy() - ref_score).max() <= 1e-9 * np.abs(ref_score).max()


def test_noalloc_ransac_rejects_oversize():
    torch = pytest.importorskip("torch")
    d = lib()
    p = d.default_params()
    dev = torch.device("cuda", 0)
    M = 5000                                        # beyond DS_NOALLOC_MAX_MATCHES
    z = lambda *s, dt=torch.float32: torch.zeros(*s, dtype=dt, device=dev)
    with pytest.raises(d.DsError) as e:
        d.ds_ransac_noalloc(z(60, 80), 80, 60, (80, 80, 39.5, 29.5), z(M, dt=torch.int32),
                            z(M, 3), M, z(30, dt=torch.int32), 30, 10, 2.0, 0.5,
                            z(157, dt=torch.int32), z(M), z(2, dt=torch.int32),
                            z(30, dt=torch.float64))
    assert e.value.status == d.DS_ERR_ARG


def _noalloc(d, torch, dev, sc, midx_np, hyp_np, fr, p):
    M = len(midx_np)
    t = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a, dt)).to(dev)
    bits = torch.zeros((M + 31) // 32, dtype=torch.int32, device=dev)
    w = torch.zeros(M, dtype=torch.float32, device=dev)
    kept = torch.zeros(2, dtype=torch.int32, device=dev)
    score = torch.zeros(p.n_hyp, dtype=torch.float64, device=dev)
    d.ds_ransac_noalloc(t(sc.template_depth, np.float32), sc.W, sc.H, sc.K, t(midx_np),
                        t(fr.match_xyz, np.float32), M, t(hyp_np), p.n_hyp, p.n_reweight, p.H_mm,
                        p.keep_frac, bits, w, kept, score)
    return (bits.cpu().numpy().view(np.uint32), w.cpu().numpy(), kept.cpu().numpy().view(np.uint32),
            score.cpu().numpy())


def test_noalloc_ransac_at_its_limits_matches_handle_path():
    """M = DS_NOALLOC_MAX_MATCHES = 4000 matches and 64 references (DS_MAX_HYP): the largest
    case, whose per-match staging takes 224,000 B of the kernel's dynamic shared memory."""
    torch = pytest.importorskip("torch")
    from synth.scene import Config
    d = lib()
    p = d.default_params(n_hyp=64)
    dev = torch.device("cuda", 0)
    cfg = Config("na_200x150_m4000", 200, 150, 40, 4000, 8, 0.45, 0.5, 0.05, 6.0, 0.0, 2.0, 1.5,
                 1, n_hyp=64)
    sc = make_scene(cfg, 777)
    fr = sc.frames[0]
    M = len(fr.match_idx)
    assert M == 4000 and len(fr.hyp) == 64
    ref_bits, ref_w, ref_kept, ref_score = _handle_path(d, sc, fr, p)
    for _ in range(2):
        bits, w, kept, score = _noalloc(d, torch, dev, sc, fr.match_idx, fr.hyp, fr, p)
        assert np.array_equal(unpack_bits(bits, M), unpack_bits(ref_bits, M))
        assert np.array_equal(kept, ref_kept)
        assert np.abs(w - ref_w).max() <= 1e-6
        assert np.abs(score - ref_score).max() <= 1e-9 * np.abs(ref_score).max()


def test_noalloc_ransac_reports_bad_indices_and_recovers():
    """An out-of-range match pixel and an out-of-range reference id are replaced on the device
    (no read outside the caller's buffers) and reported as DS_ERR_ARG after the run; the next
    call with good indices is clean and equals the handle path."""
    torch = pytest.importorskip("torch")
    d = lib()
    p = d.default_params()
    dev = torch.device("cuda", 0)
    sc = make_scene(MID, 4242)
    fr = sc.frames[0]
    M = len(fr.match_idx)
    bad_idx = fr.match_idx.copy()
    bad_idx[5] = sc.W * sc.H + 17          # past the image
    bad_hyp = fr.hyp.copy()
    bad_hyp[3] = M + 2                     # past the matches
    with pytest.raises(d.DsError) as e:
        _noalloc(d, torch, dev, sc, bad_idx, fr.hyp, fr, p)
    assert e.value.status == d.DS_ERR_ARG
    with pytest.raises(d.DsError) as e:
        _noalloc(d, torch, dev, sc, fr.match_idx, bad_hyp, fr, p)
    assert e.value.status == d.DS_ERR_ARG
    ref_bits, ref_w, ref_kept, ref_score = _handle_path(d, sc, fr, p)
    bits, w, kept, score = _noalloc(d, torch, dev, sc, fr.match_idx, fr.hyp, fr, p)
    assert np.array_equal(unpack_bits(bits, M), unpack_bits(ref_bits, M))
    assert np.array_equal(kept, ref_kept)
    assert np.abs(w - ref_w).max() <= 1e-6
