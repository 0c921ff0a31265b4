"""Python binding of libdefsolve (the C ABI in include/defsolve.h and include/defsolve_orb.h).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels. Arrays
may be numpy arrays (host memory) or torch CUDA tensors (device memory); both are passed to the
library as plain pointers. The library must be built first (paper_2007_08576_gb300.build); a
missing library raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdefsolve.so")

DS_OK, DS_ERR_ARG, DS_ERR_OOM, DS_ERR_BAD_INPUT, DS_ERR_NOT_SPD, DS_ERR_STATE, DS_ERR_TIMEOUT, \
    DS_ERR_CUDA = range(8)
DS_PREC_FP64, DS_PREC_FP32, DS_PREC_FP32_REFINE = 0, 1, 2
DS_MAX_ITERS = 64
DS_MAX_HYP = 64
DS_FACTOR_AUTO = -1

# every exported symbol of include/defsolve.h and include/defsolve_orb.h
EXPORTS = [
    "ds_default_params", "ds_create_template", "ds_set_control_points", "ds_submit_frame",
    "ds_solve", "ds_solve_batch", "ds_batch_create", "ds_batch_solve", "ds_batch_solve_masked",
    "ds_batch_status",
    "ds_batch_destroy", "ds_batch_set_tracing", "ds_batch_phase_times", "ds_batch_set_graph",
    "ds_batch_tune", "ds_batch_factor_kernel", "ds_get_deformation", "ds_get_deformation64",
    "ds_set_deformation", "ds_get_inlier_mask", "ds_get_ransac", "ds_get_cost",
    "ds_get_blend_table", "ds_get_frame_points", "ds_linearize", "ds_set_tracing",
    "ds_get_phase_times", "ds_get_counters", "ds_get_device_bytes", "ds_factor_tasks",
    "ds_ransac_noalloc",
    "ds_selftest_bounded_wait",
    "ds_destroy", "ds_status_str", "ds_version",
    "ds_orb_default_params", "ds_orb_create", "ds_orb_detect", "ds_orb_num_keypoints",
    "ds_orb_get_keypoints", "ds_orb_match", "ds_orb_num_matches", "ds_orb_get_matches",
    "ds_orb_match_device", "ds_orb_destroy",
]


class DsIntrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float)]


class DsParams(ctypes.Structure):
    _fields_ = [("w_orb", ctypes.c_double), ("w_angle", ctypes.c_double),
                ("w_rot", ctypes.c_double), ("w_arap0", ctypes.c_double),
                ("H_mm", ctypes.c_double), ("tukey_c_mm", ctypes.c_double),
                ("sigma_blend_scale", ctypes.c_double), ("sigma_arap_scale", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("eps_damp", ctypes.c_double),
                ("keep_frac", ctypes.c_double), ("n_hyp", ctypes.c_int32),
                ("n_reweight", ctypes.c_int32), ("n_nearest", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("factor_tc", ctypes.c_int32),
                ("solver", ctypes.c_int32), ("assoc", ctypes.c_int32), ("jtj", ctypes.c_int32),
                ("ransac_o1", ctypes.c_int32)]


class DsOrbParams(ctypes.Structure):
    _fields_ = [("fast_t", ctypes.c_int32), ("border", ctypes.c_int32),
                ("max_dist", ctypes.c_int32), ("max_kp", ctypes.c_int32)]


class DsSolveStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("n_inliers", ctypes.c_int32),
                ("n_kept", ctypes.c_int32), ("n_icp_valid_last", ctypes.c_int32),
                ("w_arap", ctypes.c_double), ("cost", ctypes.c_double * DS_MAX_ITERS),
                ("cost_icp", ctypes.c_double * DS_MAX_ITERS),
                ("cost_orb", ctypes.c_double * DS_MAX_ITERS),
                ("cost_arap", ctypes.c_double * DS_MAX_ITERS)]


class DsError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn}: {status_str(status)} ({status})")


_lib = None


def lib(path: str | None = None):
    """Load libdefsolve.so once; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libdefsolve.so not built ({p}); run paper_2007_08576_gb300.build.build()")
    L = ctypes.CDLL(p)
    vp, i32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    sig = {
        "ds_default_params": (None, [ctypes.POINTER(DsParams)]),
        "ds_create_template": (i32, [vp, i32, i32, DsIntrinsics, ctypes.POINTER(DsParams), vp,
                                     ctypes.POINTER(vp)]),
        "ds_set_control_points": (i32, [vp, vp, i32]),
        "ds_submit_frame": (i32, [vp, vp, vp, vp, i32, vp]),
        "ds_solve": (i32, [vp, i32, ctypes.POINTER(DsSolveStats)]),
        "ds_solve_batch": (i32, [ctypes.POINTER(vp), i32, i32]),
        "ds_batch_create": (i32, [ctypes.POINTER(vp), i32, vp, ctypes.POINTER(vp)]),
        "ds_batch_solve": (i32, [vp, i32]),
        "ds_batch_solve_masked": (i32, [vp, vp, i32]),
        "ds_batch_status": (i32, [vp]),
        "ds_batch_destroy": (i32, [vp]),
        "ds_batch_set_tracing": (i32, [vp, i32]),
        "ds_batch_set_graph": (i32, [vp, i32]),
        "ds_batch_tune": (i32, [vp, i32, ctypes.POINTER(i32), vp]),
        "ds_batch_factor_kernel": (i32, [vp, ctypes.POINTER(i32), vp]),
        "ds_batch_phase_times": (i32, [vp, vp]),
        "ds_get_deformation": (i32, [vp, vp, vp, vp]),
        "ds_get_deformation64": (i32, [vp, vp, vp]),
        "ds_set_deformation": (i32, [vp, vp, vp]),
        "ds_get_inlier_mask": (i32, [vp, vp]),
        "ds_get_ransac": (i32, [vp, vp, vp, vp]),
        "ds_get_cost": (i32, [vp, ctypes.POINTER(f64)]),
        "ds_get_blend_table": (i32, [vp, ctypes.POINTER(i32), vp, vp, vp]),
        "ds_get_frame_points": (i32, [vp, vp, vp]),
        "ds_linearize": (i32, [vp, f64, vp, vp, vp, ctypes.POINTER(f64)]),
        "ds_set_tracing": (i32, [vp, i32]),
        "ds_get_phase_times": (i32, [vp, vp]),
        "ds_get_counters": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "ds_get_device_bytes": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "ds_factor_tasks": (i32, [i32, i32, vp, i32, ctypes.POINTER(ctypes.c_int32)]),
        "ds_ransac_noalloc": (i32, [vp, i32, i32, DsIntrinsics, vp, vp, i32, vp, i32, i32, f64,
                                    f64, vp, vp, vp, vp, vp]),
        "ds_selftest_bounded_wait": (i32, [i32, ctypes.c_int64, i32, ctypes.POINTER(f64)]),
        "ds_destroy": (i32, [vp]),
        "ds_status_str": (ctypes.c_char_p, [i32]),
        "ds_version": (ctypes.c_char_p, []),
        "ds_orb_default_params": (None, [ctypes.POINTER(DsOrbParams)]),
        "ds_orb_create": (i32, [i32, i32, DsIntrinsics, ctypes.POINTER(DsOrbParams), vp, vp,
                                ctypes.POINTER(vp)]),
        "ds_orb_detect": (i32, [vp, vp, vp]),
        "ds_orb_num_keypoints": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "ds_orb_get_keypoints": (i32, [vp, vp, vp, vp, vp]),
        "ds_orb_match": (i32, [vp, vp]),
        "ds_orb_num_matches": (i32, [vp, ctypes.POINTER(i32)]),
        "ds_orb_get_matches": (i32, [vp, vp, vp, vp, vp, vp]),
        "ds_orb_match_device": (i32, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "ds_orb_destroy": (i32, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def status_str(status: int) -> str:
    return lib().ds_status_str(int(status)).decode()


def _check(fn, rc):
    if rc != DS_OK:
        raise DsError(fn, rc)


def _ptr(x, dtype):
    """Plain pointer of a contiguous numpy array or torch tensor of the given numpy dtype."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        tmap = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
                np.uint8: torch.uint8,
                np.uint32: torch.uint32 if hasattr(torch, "uint32") else torch.int32}
        if x.dtype != tmap[np.dtype(dtype).type] or not x.is_contiguous():
            raise TypeError(f"expected a contiguous tensor of {np.dtype(dtype)}")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def default_params(**kw) -> DsParams:
    p = DsParams()
    lib().ds_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, "lambda_" if k == "lambda" else k, v)
    return p


# ----------------------------------------------------------------------------- the C ABI


def ds_create_template(depth_hw, W, H, K, params: DsParams | None = None, stream=None):
    h = ctypes.c_void_p()
    Kc = DsIntrinsics(*[float(k) for k in K])
    rc = lib().ds_create_template(_ptr(depth_hw, np.float32), int(W), int(H), Kc,
                                  ctypes.byref(params) if params is not None else None,
                                  stream, ctypes.byref(h))
    _check("ds_create_template", rc)
    return h


def ds_set_control_points(h, pixel_index, N=None):
    N = len(pixel_index) if N is None else N
    _check("ds_set_control_points", lib().ds_set_control_points(h, _ptr(pixel_index, np.int32), int(N)))


def ds_submit_frame(h, depth_hw, match_tmpl_idx, match_xyz, M=None, hyp_list=None):
    M = (len(match_tmpl_idx) if match_tmpl_idx is not None else 0) if M is None else M
    rc = lib().ds_submit_frame(h, _ptr(depth_hw, np.float32), _ptr(match_tmpl_idx, np.int32),
                               _ptr(match_xyz, np.float32), int(M), _ptr(hyp_list, np.int32))
    _check("ds_submit_frame", rc)


def ds_solve(h, iters, stats: bool = False):
    st = DsSolveStats() if stats else None
    rc = lib().ds_solve(h, int(iters), ctypes.byref(st) if st is not None else None)
    _check("ds_solve", rc)
    return st


def ds_solve_batch(handles, iters):
    _check("ds_solve_batch", lib().ds_solve_batch(_handle_array(handles), len(handles), int(iters)))


def _handle_array(handles):
    return (ctypes.c_void_p * len(handles))(*[hh.value if isinstance(hh, ctypes.c_void_p) else hh
                                              for hh in handles])


def ds_batch_create(handles, stream=None):
    b = ctypes.c_void_p()
    _check("ds_batch_create", lib().ds_batch_create(_handle_array(handles), len(handles), stream,
                                                    ctypes.byref(b)))
    return b


def ds_batch_solve(b, iters):
    _check("ds_batch_solve", lib().ds_batch_solve(b, int(iters)))


def ds_batch_solve_masked(b, active, iters):
    """Solves the handles with active[p] != 0 (a length-n sequence of 0 / 1 in batch order)."""
    m = np.ascontiguousarray(np.asarray(active, dtype=np.uint8))
    _check("ds_batch_solve_masked", lib().ds_batch_solve_masked(b, m.ctypes.data, int(iters)))


def ds_batch_status(b):
    _check("ds_batch_status", lib().ds_batch_status(b))


def ds_batch_set_tracing(b, on=True):
    _check("ds_batch_set_tracing", lib().ds_batch_set_tracing(b, 1 if on else 0))


FACTOR_KERNELS = ["simt64", "tc64", "tc128_stage64k", "tc128_quads", "tc128_stage64k_pairs",
                  "tc128_pipelined"]


def ds_batch_tune(b, reps=3):
    """(chosen factor kernel index, [ms of kernels 0..5]) after timing them on the batch's sizes
    (kernel names in FACTOR_KERNELS)."""
    c = ctypes.c_int32()
    ms = np.zeros(6, np.float64)
    _check("ds_batch_tune", lib().ds_batch_tune(b, int(reps), ctypes.byref(c), _ptr(ms, np.float64)))
    return c.value, ms


def ds_batch_factor_kernel(b):
    c = ctypes.c_int32()
    ms = np.zeros(6, np.float64)
    _check("ds_batch_factor_kernel",
           lib().ds_batch_factor_kernel(b, ctypes.byref(c), _ptr(ms, np.float64)))
    return c.value, ms


def ds_batch_set_graph(b, on=True):
    _check("ds_batch_set_graph", lib().ds_batch_set_graph(b, 1 if on else 0))


def ds_batch_phase_times(b):
    ms = np.zeros(4, np.float64)
    _check("ds_batch_phase_times", lib().ds_batch_phase_times(b, ms.ctypes.data))
    return ms


def ds_batch_destroy(b):
    _check("ds_batch_destroy", lib().ds_batch_destroy(b))


def ds_get_deformation(h, q_N4=None, t_N3=None, pos_N3=None):
    rc = lib().ds_get_deformation(h, _ptr(q_N4, np.float32), _ptr(t_N3, np.float32),
                                  _ptr(pos_N3, np.float32))
    _check("ds_get_deformation", rc)


def ds_get_deformation64(h, q_N4=None, t_N3=None):
    _check("ds_get_deformation64",
           lib().ds_get_deformation64(h, _ptr(q_N4, np.float64), _ptr(t_N3, np.float64)))


def ds_set_deformation(h, q_N4, t_N3):
    _check("ds_set_deformation",
           lib().ds_set_deformation(h, _ptr(q_N4, np.float32), _ptr(t_N3, np.float32)))


def ds_get_inlier_mask(h, bits):
    _check("ds_get_inlier_mask", lib().ds_get_inlier_mask(h, _ptr(bits, np.uint32)))


def ds_get_ransac(h, w_M=None, kept_bits=None, score_nh=None):
    _check("ds_get_ransac", lib().ds_get_ransac(h, _ptr(w_M, np.float32),
                                                _ptr(kept_bits, np.uint32),
                                                _ptr(score_nh, np.float64)))


def ds_get_cost(h) -> float:
    F = ctypes.c_double()
    _check("ds_get_cost", lib().ds_get_cost(h, ctypes.byref(F)))
    return F.value


def ds_get_blend_table(h, pix_P=None, nid_P4=None, alpha_P4=None) -> int:
    P = ctypes.c_int32()
    rc = lib().ds_get_blend_table(h, ctypes.byref(P), _ptr(pix_P, np.int32),
                                  _ptr(nid_P4, np.int32), _ptr(alpha_P4, np.float32))
    _check("ds_get_blend_table", rc)
    return P.value


def ds_get_frame_points(h, pts4=None, nrm4=None):
    _check("ds_get_frame_points",
           lib().ds_get_frame_points(h, _ptr(pts4, np.float32), _ptr(nrm4, np.float32)))


def ds_linearize(h, w_arap_in=0.0, A_nn=None, b_n=None, cost3=None):
    wo = ctypes.c_double()
    rc = lib().ds_linearize(h, float(w_arap_in), _ptr(A_nn, np.float64), _ptr(b_n, np.float64),
                            _ptr(cost3, np.float64), ctypes.byref(wo))
    _check("ds_linearize", rc)
    return wo.value


def ds_set_tracing(h, on=True):
    _check("ds_set_tracing", lib().ds_set_tracing(h, 1 if on else 0))


def ds_get_phase_times(h):
    ms = np.zeros(4, np.float64)
    _check("ds_get_phase_times", lib().ds_get_phase_times(h, ms.ctypes.data))
    return ms


def ds_get_counters(h=None) -> int:
    """Kernels launched by the handle so far (h None: by the whole library)."""
    k = ctypes.c_int64()
    _check("ds_get_counters", lib().ds_get_counters(h, ctypes.byref(k)))
    return k.value


def ds_get_device_bytes(h) -> int:
    b = ctypes.c_int64()
    _check("ds_get_device_bytes", lib().ds_get_device_bytes(h, ctypes.byref(b)))
    return b.value


def ds_factor_tasks(nb: int, paired: int = 0) -> np.ndarray:
    """The block factorisation's task order within one problem, rows (type, I, J); paired: 0
    single blocks, 1 column pairs, 2 two rows x two columns."""
    n = ctypes.c_int32()
    _check("ds_factor_tasks", lib().ds_factor_tasks(nb, int(paired), None, 0, ctypes.byref(n)))
    out = np.zeros((n.value, 3), np.int32)
    _check("ds_factor_tasks", lib().ds_factor_tasks(nb, int(paired), out.ctypes.data, n.value,
                                                     ctypes.byref(n)))
    return out


def _dev_ptr(t, itemsize):
    """Device pointer of a contiguous torch CUDA tensor with the given element size."""
    if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous() and t.element_size() == itemsize):
        raise TypeError("expected a contiguous CUDA tensor with %d-byte elements" % itemsize)
    return t.data_ptr()


def ds_ransac_noalloc(depth0, W, H, K, match_idx, match_xyz, M, hyp, n_hyp, n_reweight, H_mm,
                      keep_frac, mask_bits, w_M, kept_bits, score_nh, stream=None):
    """RANSAC preselection into caller-provided device tensors, with no allocation in the
    library (see include/defsolve.h). Bit outputs may be int32 or uint32 tensors."""
    Kc = DsIntrinsics(*[float(k) for k in K])
    rc = lib().ds_ransac_noalloc(_dev_ptr(depth0, 4), int(W), int(H), Kc, _dev_ptr(match_idx, 4),
                                 _dev_ptr(match_xyz, 4), int(M), _dev_ptr(hyp, 4), int(n_hyp),
                                 int(n_reweight), float(H_mm), float(keep_frac),
                                 _dev_ptr(mask_bits, 4), _dev_ptr(w_M, 4), _dev_ptr(kept_bits, 4),
                                 _dev_ptr(score_nh, 8), stream)
    _check("ds_ransac_noalloc", rc)


def ds_selftest_bounded_wait(kind, budget_ns, peer_error=0):
    """(status, device milliseconds) of one bounded wait on a flag that nothing sets (see
    include/defsolve.h): DS_ERR_TIMEOUT is the designed outcome; other errors raise."""
    ms = ctypes.c_double(0.0)
    rc = lib().ds_selftest_bounded_wait(int(kind), int(budget_ns), int(peer_error), ctypes.byref(ms))
    if rc not in (DS_OK, DS_ERR_TIMEOUT):
        raise DsError("ds_selftest_bounded_wait", rc)
    return rc, ms.value


def ds_destroy(h):
    _check("ds_destroy", lib().ds_destroy(h))


def ds_version() -> str:
    return lib().ds_version().decode()


# ----------------------------------------------------------------------------- convenience


class Solver:
    """One deformation stream: template + control points + per-frame solves (host arrays)."""

    def __init__(self, template_depth, K, nodes, params: DsParams | None = None, stream=None):
        H, W = template_depth.shape
        self.W, self.H = W, H
        self.h = ds_create_template(np.ascontiguousarray(template_depth, np.float32), W, H, K,
                                    params, stream)
        self.nodes = np.ascontiguousarray(nodes, np.int32)
        self.N = len(self.nodes)
        ds_set_control_points(self.h, self.nodes)
        self.params = params

    def submit(self, depth, match_idx, match_xyz, hyp):
        self.M = len(match_idx)
        ds_submit_frame(self.h, np.ascontiguousarray(depth, np.float32),
                        np.ascontiguousarray(match_idx, np.int32),
                        np.ascontiguousarray(match_xyz, np.float32).reshape(-1, 3),
                        self.M, np.ascontiguousarray(hyp, np.int32))

    def solve(self, iters=10, stats=True):
        return ds_solve(self.h, iters, stats)

    def deformation(self):
        q = np.zeros((self.N, 4), np.float32)
        t = np.zeros((self.N, 3), np.float32)
        p = np.zeros((self.N, 3), np.float32)
        ds_get_deformation(self.h, q, t, p)
        return q, t, p

    def deformation64(self):
        q = np.zeros((self.N, 4), np.float64)
        t = np.zeros((self.N, 3), np.float64)
        ds_get_deformation64(self.h, q, t)
        return q, t

    def mask(self):
        bits = np.zeros((self.M + 31) // 32, np.uint32)
        ds_get_inlier_mask(self.h, bits)
        k = np.arange(self.M)
        return ((bits[k // 32] >> (k % 32).astype(np.uint32)) & 1).astype(bool)

    def close(self):
        if self.h is not None:
            ds_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- ORB features


def orb_default_params(**kw) -> DsOrbParams:
    p = DsOrbParams()
    lib().ds_orb_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def ds_orb_create(W, H, K, pattern, params: DsOrbParams | None = None, stream=None):
    o = ctypes.c_void_p()
    Kc = DsIntrinsics(*[float(k) for k in K])
    rc = lib().ds_orb_create(int(W), int(H), Kc, ctypes.byref(params) if params is not None else None,
                             _ptr(pattern, np.float64), stream, ctypes.byref(o))
    _check("ds_orb_create", rc)
    return o


def ds_orb_detect(o, image_hw, depth_hw=None):
    _check("ds_orb_detect", lib().ds_orb_detect(o, _ptr(image_hw, np.uint8), _ptr(depth_hw, np.float32)))


def ds_orb_num_keypoints(o):
    n, tot = ctypes.c_int32(), ctypes.c_int32()
    _check("ds_orb_num_keypoints", lib().ds_orb_num_keypoints(o, ctypes.byref(n), ctypes.byref(tot)))
    return n.value, tot.value


def ds_orb_get_keypoints(o, pix=None, score=None, bin_=None, desc=None):
    _check("ds_orb_get_keypoints", lib().ds_orb_get_keypoints(
        o, _ptr(pix, np.int32), _ptr(score, np.int32), _ptr(bin_, np.int32), _ptr(desc, np.uint32)))


def ds_orb_match(tmpl, live):
    _check("ds_orb_match", lib().ds_orb_match(tmpl, live))


def ds_orb_num_matches(live) -> int:
    m = ctypes.c_int32()
    _check("ds_orb_num_matches", lib().ds_orb_num_matches(live, ctypes.byref(m)))
    return m.value


def ds_orb_get_matches(live, tmpl_kp=None, live_kp=None, dist=None, tmpl_pixel=None, xyz=None):
    _check("ds_orb_get_matches", lib().ds_orb_get_matches(
        live, _ptr(tmpl_kp, np.int32), _ptr(live_kp, np.int32), _ptr(dist, np.int32),
        _ptr(tmpl_pixel, np.int32), _ptr(xyz, np.float32)))


def ds_orb_match_device(live):
    """Device addresses (ints) of the match arrays: template pixel per match, M x 3 points."""
    a, b = ctypes.c_void_p(), ctypes.c_void_p()
    _check("ds_orb_match_device", lib().ds_orb_match_device(live, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ds_orb_destroy(o):
    _check("ds_orb_destroy", lib().ds_orb_destroy(o))


class Orb:
    """One feature context (template or live side) over W x H images."""

    def __init__(self, W, H, K, pattern, params: DsOrbParams | None = None, stream=None):
        self.W, self.H = int(W), int(H)
        self.o = ds_orb_create(W, H, K, np.ascontiguousarray(pattern, np.float64), params, stream)

    def detect(self, image, depth=None):
        img = np.ascontiguousarray(image, np.uint8) if isinstance(image, np.ndarray) else image
        dep = (np.ascontiguousarray(depth, np.float32) if isinstance(depth, np.ndarray)
               else depth)
        ds_orb_detect(self.o, img, dep)

    def keypoints(self):
        n, tot = ds_orb_num_keypoints(self.o)
        pix = np.zeros(n, np.int32)
        score = np.zeros(n, np.int32)
        b = np.zeros(n, np.int32)
        desc = np.zeros((n, 8), np.uint32)
        ds_orb_get_keypoints(self.o, pix, score, b, desc)
        return dict(pix=pix, score=score, bin=b, desc=desc, n_total=tot)

    def match_from(self, tmpl: "Orb"):
        """Matches tmpl's keypoints to this (live) object's; returns the host copies."""
        ds_orb_match(tmpl.o, self.o)
        M = ds_orb_num_matches(self.o)
        out = dict(t=np.zeros(M, np.int32), l=np.zeros(M, np.int32), dist=np.zeros(M, np.int32),
                   tmpl_pix=np.zeros(M, np.int32), xyz=np.zeros((M, 3), np.float32))
        ds_orb_get_matches(self.o, out["t"], out["l"], out["dist"], out["tmpl_pix"], out["xyz"])
        return out

    def close(self):
        if self.o:
            ds_orb_destroy(self.o)
            self.o = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
