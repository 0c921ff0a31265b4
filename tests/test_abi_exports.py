"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point that
include/*.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                  if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ds_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_2007_08576_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["ds_create_template", "ds_set_control_points", "ds_submit_frame", "ds_solve",
                 "ds_get_deformation", "ds_destroy", "ds_status_str"]:
        assert name in syms


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(built):
    from paper_2007_08576_gb300 import defsolve
    assert sorted(defsolve.EXPORTS) == declared_symbols()
    defsolve.lib(built)
    assert defsolve.status_str(defsolve.DS_ERR_NOT_SPD).startswith("normal equations")


def test_default_params_are_the_papers(built):
    from paper_2007_08576_gb300 import defsolve
    p = defsolve.default_params()
    assert (p.w_orb, p.w_angle, p.w_rot, p.n_hyp, p.n_reweight) == (10.0, 20.0, 100.0, 30, 10)
    assert p.n_nearest == 4 and p.refine_steps == 2 and p.precision == defsolve.DS_PREC_FP64


def test_argument_errors_need_no_gpu(built):
    from paper_2007_08576_gb300 import defsolve as d
    L = d.lib(built)
    # null handle / null pointers are rejected before any CUDA call
    assert L.ds_solve(None, 10, None) == d.DS_ERR_ARG
    assert L.ds_set_control_points(None, None, 32) == d.DS_ERR_ARG
    assert L.ds_submit_frame(None, None, None, None, 0, None) == d.DS_ERR_ARG
    assert L.ds_destroy(None) == d.DS_OK
    h = ctypes.c_void_p()
    K = d.DsIntrinsics(80.0, 80.0, 39.5, 29.5)
    assert L.ds_create_template(None, 80, 60, K, None, None, ctypes.byref(h)) == d.DS_ERR_ARG
    # the bounded-wait self-test checks its arguments before touching the device
    ms = ctypes.c_double()
    assert L.ds_selftest_bounded_wait(2, 1000000, 0, ctypes.byref(ms)) == d.DS_ERR_ARG
    assert L.ds_selftest_bounded_wait(0, 10, 0, ctypes.byref(ms)) == d.DS_ERR_ARG
    assert L.ds_selftest_bounded_wait(0, 10**9, 0, ctypes.byref(ms)) == d.DS_ERR_ARG
    assert L.ds_selftest_bounded_wait(1, 1000000, 3, ctypes.byref(ms)) == d.DS_ERR_ARG
    # the factor tuner and the device-byte count reject a null batch / handle
    c = ctypes.c_int32()
    assert L.ds_batch_tune(None, 2, ctypes.byref(c), None) == d.DS_ERR_ARG
    assert L.ds_batch_factor_kernel(None, ctypes.byref(c), None) == d.DS_ERR_ARG
    b = ctypes.c_int64()
    assert L.ds_get_device_bytes(None, ctypes.byref(b)) == d.DS_ERR_ARG


def test_binding_fails_loudly_without_the_library():
    """No CPU fallback: with the shared library absent the binding raises instead of computing."""
    import subprocess
    import sys
    code = ("from paper_2007_08576_gb300 import defsolve as d\n"
            "d.LIB_PATH = '/nonexistent/libdefsolve.so'\n"
            "try:\n"
            "    d.Solver\n"
            "    d.lib()\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert "raised:" in r.stdout and "not built" in r.stdout
