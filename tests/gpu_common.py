"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and the FP64
oracle on the same seeded inputs, and compare."""
import numpy as np

from oracle import solver
from synth import make_scene
from synth.scene import Config

# Parity tolerances: control points within 1e-3 mm, cost within 1e-5 relative,
# RANSAC masks bit-exact outside the 1e-6 mm band around H.
POS_TOL_MM = 1e-3
COST_RTOL = 1e-5
BAND_MM = 1e-6

MID = Config("mid_150x110_n50", 150, 110, 50, 333, 8, 0.35, 0.5, 0.05, 6.0, 0.0, 2.0, 1.5, 1)


def lib():
    from paper_2007_08576_gb300 import build
    build.build()
    from paper_2007_08576_gb300 import defsolve
    defsolve.lib()
    return defsolve


def oracle_params(p):
    """oracle.Params mirroring a DsParams."""
    return solver.Params(w_orb=p.w_orb, w_angle=p.w_angle, w_rot=p.w_rot, w_arap0=p.w_arap0,
                         H=p.H_mm, tukey_c=p.tukey_c_mm, sigma_blend_scale=p.sigma_blend_scale,
                         sigma_arap_scale=p.sigma_arap_scale, lam=p.lambda_, eps=p.eps_damp,
                         keep_frac=p.keep_frac, n_hyp=p.n_hyp, n_reweight=p.n_reweight,
                         solver="block_jacobi" if getattr(p, "solver", 0) == 1 else "dense",
                         assoc="bilinear" if getattr(p, "assoc", 0) == 1 else "nearest",
                         ransac_o1="warm" if getattr(p, "ransac_o1", 0) == 1 else "template")


def gpu_frame(d, sc, frame, params, iters=10, solver_obj=None):
    s = solver_obj or d.Solver(sc.template_depth, sc.K, sc.nodes, params)
    s.submit(frame.depth, frame.match_idx, frame.match_xyz, frame.hyp)
    st = s.solve(iters, stats=True)
    q, t = s.deformation64()
    return s, st, q, t


def ransac_listed(rs, H, band=BAND_MM, cut_rel=1e-6):
    """Matches whose mask bit is not graded: within `band` of H for some kept reference, or
    decided by a reference whose score is within cut_rel of the keep cut."""
    kept = rs["kept"]
    listed = np.zeros(rs["d"].shape[1], dtype=bool)
    for h in np.flatnonzero(kept):
        listed |= np.abs(rs["d"][h] - H) <= band
    cut = 0.5 * rs["score"].max()
    amb = np.abs(rs["score"] - cut) <= cut_rel * abs(cut)
    for h in np.flatnonzero(amb):
        listed |= rs["d"][h] <= H + band
    return listed, amb


def unpack_bits(bits, M):
    k = np.arange(M)
    return ((bits[k // 32] >> (k % 32).astype(np.uint32)) & 1).astype(bool)


def scene(cfg, seed, n_frames=1):
    return make_scene(cfg, seed, n_frames=n_frames)
