"""CPU checks of the C ABI: the library builds, loads and exports every
function include/*.h declares; argument validation that happens before any
device call answers EINVAL.  No compute call runs here."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(bbfmm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1903_02153_gb300 import build
    build.build()
    from paper_1903_02153_gb300 import bbfmm
    return bbfmm


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["bbfmm_plan", "bbfmm_matvec", "bbfmm_destroy", "bbfmm_last_error"]:
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (bbfmm_\w+)", out))
    assert set(declared_functions()) <= exported
    # the binding wraps exactly the declared functions
    assert set(lib.EXPORTED) <= set(declared_functions())


def test_build_targets_sm103a_only():
    from paper_1903_02153_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_default_opts(lib):
    o = lib.bbfmm_default_opts()
    assert o.ell == 1.0 and o.svd_eps == 1e-7 and o.max_nrhs == 1 and o.precision == 0


@pytest.mark.parametrize("n,kid,p,depth", [(0, 1, 4, 3), (100, 7, 4, 3), (100, 1, 1, 3), (100, 1, 11, 3),
                                           (100, 1, 4, 9), (100, 1, 4, -1)])
def test_plan_rejects_bad_arguments(lib, n, kid, p, depth):
    pts = np.random.default_rng(0).random((max(n, 1), 3))
    h = ctypes.c_void_p()
    st = lib.lib().bbfmm_plan(pts.ctypes.data, n, kid, p, depth, None, None, ctypes.byref(h))
    assert st == lib.BBFMM_EINVAL
    assert h.value is None
    assert lib.bbfmm_last_error() != ""


def test_plan_rejects_bad_options(lib):
    pts = np.random.default_rng(0).random((10, 3))
    h = ctypes.c_void_p()
    for field, val in [("ell", 0.0), ("svd_eps", -1.0), ("max_nrhs", 0), ("precision", 9)]:
        o = lib.bbfmm_default_opts()
        setattr(o, field, val)
        st = lib.lib().bbfmm_plan(pts.ctypes.data, 10, 1, 4, 3, ctypes.byref(o), None, ctypes.byref(h))
        assert st == lib.BBFMM_EINVAL, field
    o = lib.bbfmm_default_opts()
    o.domain_given, o.side = 1, -2.0
    assert lib.lib().bbfmm_plan(pts.ctypes.data, 10, 1, 4, 3, ctypes.byref(o), None,
                                ctypes.byref(h)) == lib.BBFMM_EINVAL


def test_null_handles(lib):
    L = lib.lib()
    assert L.bbfmm_destroy(None) == 0
    assert L.bbfmm_matvec(None, None, None, 1, None) == lib.BBFMM_EINVAL
    assert L.bbfmm_plan_info(None, None) == lib.BBFMM_EINVAL
    c = ctypes.c_int(-1)
    assert L.bbfmm_matvec_launches(None, 1, ctypes.byref(c)) == lib.BBFMM_EINVAL and c.value == -1
    t = lib.bbfmm_tuning()
    assert L.bbfmm_get_tuning(None, 1, ctypes.byref(t)) == lib.BBFMM_EINVAL


def test_plan_targets_rejects_bad_arguments(lib):
    """Separate-target plans: NULL targets, or a target count out of range,
    answer EINVAL before any device call."""
    pts = np.random.default_rng(1).random((10, 3))
    L = lib.lib()
    h = ctypes.c_void_p()
    assert L.bbfmm_plan_targets(pts.ctypes.data, 10, None, 10, 1, 4, 3, None, None,
                                ctypes.byref(h)) == lib.BBFMM_EINVAL
    assert h.value is None
    for nt in (0, -1, 1 << 31):
        assert L.bbfmm_plan_targets(pts.ctypes.data, 10, pts.ctypes.data, nt, 1, 4, 3, None, None,
                                    ctypes.byref(h)) == lib.BBFMM_EINVAL, nt
    assert L.bbfmm_plan_targets(pts.ctypes.data, 0, pts.ctypes.data, 10, 1, 4, 3, None, None,
                                ctypes.byref(h)) == lib.BBFMM_EINVAL


def test_plan_rejects_bad_interp(lib):
    """interp must be CHEBYSHEV or UNIFORM, and UNIFORM (the Fourier-domain
    M2L, FP32) takes no tensor-core precision: EINVAL before any device call."""
    pts = np.random.default_rng(2).random((10, 3))
    h = ctypes.c_void_p()
    for interp, prec in [(2, 0), (-1, 0), (1, 4), (1, 2)]:
        o = lib.bbfmm_default_opts()
        o.interp, o.precision = interp, prec
        assert lib.lib().bbfmm_plan(pts.ctypes.data, 10, 1, 4, 3, ctypes.byref(o), None,
                                    ctypes.byref(h)) == lib.BBFMM_EINVAL, (interp, prec)


def test_unknown_user_kernel_id_is_rejected(lib):
    pts = np.random.default_rng(3).random((10, 3))
    h = ctypes.c_void_p()
    assert lib.lib().bbfmm_plan(pts.ctypes.data, 10, 1999, 4, 3, None, None, ctypes.byref(h)) == lib.BBFMM_EINVAL
    kid = ctypes.c_int(0)
    assert lib.lib().bbfmm_kernel_register(None, 0, 0, ctypes.byref(kid)) == lib.BBFMM_EINVAL
    assert lib.lib().bbfmm_kernel_register(b"x", 9, 0, ctypes.byref(kid)) == lib.BBFMM_EINVAL


def test_plan_rejects_bad_near_mode(lib):
    """near_mode must be AUTO, ORDERED or SYMMETRIC: EINVAL before any device call."""
    pts = np.random.default_rng(4).random((10, 3))
    h = ctypes.c_void_p()
    for mode in (3, -1, 7):
        o = lib.bbfmm_default_opts()
        o.near_mode = mode
        assert lib.lib().bbfmm_plan(pts.ctypes.data, 10, 1, 4, 3, ctypes.byref(o), None,
                                    ctypes.byref(h)) == lib.BBFMM_EINVAL, mode
        assert "near_mode" in lib.bbfmm_last_error()
