"""Thin ctypes binding of include/bbfmm.h (argument marshalling only).

Every function keeps the C name and calls straight into libbbfmm.so; every
stage of a matvec runs in the library's CUDA kernels.  There is no other code
path: if the library is missing, ``lib()`` raises.

Tensors are PyTorch CUDA tensors (device memory and streams only) or numpy /
pinned host arrays; the library finds out which from the pointer.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbbfmm.so")

BBFMM_OK, BBFMM_EINVAL, BBFMM_ENOMEM, BBFMM_ECUDA = 0, -1, -2, -3
BBFMM_ETIMEOUT, BBFMM_EBUSY, BBFMM_EINTERNAL = -4, -5, -6
BBFMM_K_INV_R, BBFMM_K_INV_R2, BBFMM_K_EXP, BBFMM_K_GAUSS = 1, 2, 3, 4
BBFMM_K_TEST_POLY, BBFMM_K_TEST_CONST = 100, 101
BBFMM_PREC_FP32, BBFMM_PREC_TF32, BBFMM_PREC_TF32X3, BBFMM_PREC_BF16X3, BBFMM_PREC_FP16X3 = 0, 1, 2, 3, 4

INTERPS = {"chebyshev": 0, "uniform": 1}   # BBFMM_INTERP_*
NEAR_MODES = {"auto": 0, "ordered": 1, "symmetric": 2}   # BBFMM_NEAR_*
BBFMM_K_USER_FIRST = 1000                   # ids of kernels from bbfmm_kernel_register

PRECISIONS = {"fp32": BBFMM_PREC_FP32, "tf32": BBFMM_PREC_TF32, "tf32x3": BBFMM_PREC_TF32X3,
              "bf16x3": BBFMM_PREC_BF16X3, "fp16x3": BBFMM_PREC_FP16X3}

EXPORTED = ["bbfmm_default_opts", "bbfmm_plan", "bbfmm_matvec", "bbfmm_destroy",
            "bbfmm_last_error", "bbfmm_plan_info", "bbfmm_get_coefficients",
            "bbfmm_get_leaf_cells", "bbfmm_stage_times", "bbfmm_set_timing", "bbfmm_status",
            "bbfmm_sort_points_static", "bbfmm_rand_eig", "bbfmm_plan_targets", "bbfmm_kernel_register",
            "bbfmm_get_tuning", "bbfmm_set_tuning", "bbfmm_autotune", "bbfmm_matvec_launches"]


class bbfmm_opts(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_double), ("svd_eps", ctypes.c_double),
                ("precision", ctypes.c_int), ("domain_given", ctypes.c_int),
                ("lo", ctypes.c_double * 3), ("side", ctypes.c_double),
                ("max_nrhs", ctypes.c_int), ("split_accumulate", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("keep_coefficients", ctypes.c_int),
                ("interp", ctypes.c_int), ("near_mode", ctypes.c_int), ("close_refine", ctypes.c_int),
                ("autotune", ctypes.c_int)]


class bbfmm_tuning(ctypes.Structure):
    _fields_ = [("near_mode", ctypes.c_int), ("m2l_tile", ctypes.c_int), ("m2l_stages", ctypes.c_int),
                ("measured", ctypes.c_int), ("near_box", ctypes.c_int), ("leaf_gemm", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


class bbfmm_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("depth", ctypes.c_int), ("order", ctypes.c_int),
                ("rank", ctypes.c_int), ("kernel", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_nrhs", ctypes.c_int), ("lo", ctypes.c_double * 3), ("side", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("nonempty_leaves", ctypes.c_int64),
                ("max_leaf_points", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64),
                ("m2l_pairs", ctypes.c_int64), ("n_targets", ctypes.c_int64), ("near_symmetric", ctypes.c_int),
                ("close_pairs", ctypes.c_int), ("p2p_evals", ctypes.c_int64), ("reserved", ctypes.c_int * 2)]


class BBFMMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("bbfmm status %d: %s" % (status, msg))
        self.status = status


_lib = None
_lock = threading.Lock()


def lib():
    """Load libbbfmm.so (built by paper_1903_02153_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libbbfmm.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            L.bbfmm_default_opts.argtypes = [ctypes.POINTER(bbfmm_opts)]
            L.bbfmm_default_opts.restype = None
            L.bbfmm_plan.argtypes = [vp, i64, i32, i32, i32, ctypes.POINTER(bbfmm_opts), vp,
                                     ctypes.POINTER(vp)]
            L.bbfmm_plan.restype = i32
            L.bbfmm_matvec.argtypes = [vp, vp, vp, i32, vp]
            L.bbfmm_matvec.restype = i32
            L.bbfmm_destroy.argtypes = [vp]
            L.bbfmm_destroy.restype = i32
            L.bbfmm_last_error.argtypes = []
            L.bbfmm_last_error.restype = ctypes.c_char_p
            L.bbfmm_plan_info.argtypes = [vp, ctypes.POINTER(bbfmm_info)]
            L.bbfmm_plan_info.restype = i32
            L.bbfmm_get_coefficients.argtypes = [vp, i32, i32, i32, vp]
            L.bbfmm_get_coefficients.restype = i32
            L.bbfmm_get_leaf_cells.argtypes = [vp, vp]
            L.bbfmm_get_leaf_cells.restype = i32
            L.bbfmm_stage_times.argtypes = [vp, vp]
            L.bbfmm_stage_times.restype = i32
            L.bbfmm_set_timing.argtypes = [vp, i32]
            L.bbfmm_set_timing.restype = i32
            L.bbfmm_status.argtypes = [vp, ctypes.POINTER(i32)]
            L.bbfmm_status.restype = i32
            L.bbfmm_sort_points_static.argtypes = [vp, i64, i32, ctypes.POINTER(f64), f64, vp, vp, vp]
            L.bbfmm_sort_points_static.restype = i32
            L.bbfmm_rand_eig.argtypes = [vp, vp, i32, i32, i32, ctypes.POINTER(f64), vp, vp]
            L.bbfmm_rand_eig.restype = i32
            L.bbfmm_plan_targets.argtypes = [vp, i64, vp, i64, i32, i32, i32, ctypes.POINTER(bbfmm_opts), vp,
                                             ctypes.POINTER(vp)]
            L.bbfmm_plan_targets.restype = i32
            L.bbfmm_kernel_register.argtypes = [ctypes.c_char_p, i32, i32, ctypes.POINTER(i32)]
            L.bbfmm_kernel_register.restype = i32
            L.bbfmm_get_tuning.argtypes = [vp, i32, ctypes.POINTER(bbfmm_tuning)]
            L.bbfmm_get_tuning.restype = i32
            L.bbfmm_set_tuning.argtypes = [vp, i32, ctypes.POINTER(bbfmm_tuning)]
            L.bbfmm_set_tuning.restype = i32
            L.bbfmm_autotune.argtypes = [vp, i32, vp]
            L.bbfmm_autotune.restype = i32
            L.bbfmm_matvec_launches.argtypes = [vp, i32, ctypes.POINTER(i32)]
            L.bbfmm_matvec_launches.restype = i32
            _lib = L
    return _lib


def _check(st):
    if st != BBFMM_OK:
        raise BBFMMError(st, bbfmm_last_error())
    return st


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (must be contiguous)."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not (x.flags.c_contiguous or x.flags.f_contiguous):
            raise ValueError("array must be contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(type(x))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def bbfmm_last_error() -> str:
    return lib().bbfmm_last_error().decode()


def bbfmm_default_opts() -> bbfmm_opts:
    o = bbfmm_opts()
    lib().bbfmm_default_opts(ctypes.byref(o))
    return o


def bbfmm_plan(points, kernel_id, cheb_order, depth, opts=None, stream=None):
    """points: (n, 3) float64 (torch CUDA tensor or numpy).  Returns a handle."""
    n = int(points.shape[0])
    h = ctypes.c_void_p()
    _check(lib().bbfmm_plan(_ptr(points), n, int(kernel_id), int(cheb_order), int(depth),
                            ctypes.byref(opts) if opts is not None else None, _stream(stream),
                            ctypes.byref(h)))
    return h


def bbfmm_plan_targets(sources, targets, kernel_id, cheb_order, depth, opts=None, stream=None):
    """sources (ns, 3), targets (nt, 3): float64 (torch CUDA tensors or
    numpy).  Returns a handle whose matvec maps ns weights to nt values."""
    h = ctypes.c_void_p()
    _check(lib().bbfmm_plan_targets(_ptr(sources), int(sources.shape[0]), _ptr(targets), int(targets.shape[0]),
                                    int(kernel_id), int(cheb_order), int(depth),
                                    ctypes.byref(opts) if opts is not None else None, _stream(stream),
                                    ctypes.byref(h)))
    return h


def bbfmm_kernel_register(source, homogeneity=0, symmetric=False):
    """Compile a user kernel (CUDA C defining bbfmm_kernel_f64 / _f32 of
    d = x - y); returns its kernel id for Plan / bbfmm_plan."""
    kid = ctypes.c_int(0)
    _check(lib().bbfmm_kernel_register(source.encode(), int(homogeneity), 1 if symmetric else 0,
                                       ctypes.byref(kid)))
    return kid.value


def bbfmm_matvec(plan, sigma, phi, nrhs=1, stream=None):
    """sigma: ns x nrhs, phi: nt x nrhs column-major float32 (torch tensors
    of shape (nrhs, n), or numpy arrays); phi is overwritten."""
    return _check(lib().bbfmm_matvec(plan, _ptr(sigma), _ptr(phi), int(nrhs), _stream(stream)))


def bbfmm_destroy(plan):
    return _check(lib().bbfmm_destroy(plan))


def bbfmm_plan_info(plan) -> bbfmm_info:
    info = bbfmm_info()
    _check(lib().bbfmm_plan_info(plan, ctypes.byref(info)))
    return info


def bbfmm_get_coefficients(plan, which, level, nrhs, order):
    out = np.zeros((8 ** level, nrhs, order ** 3), dtype=np.float32)
    _check(lib().bbfmm_get_coefficients(plan, int(which), int(level), int(nrhs), _ptr(out)))
    return out


def bbfmm_get_leaf_cells(plan, n):
    out = np.zeros((n, 3), dtype=np.int32)
    _check(lib().bbfmm_get_leaf_cells(plan, _ptr(out)))
    return out


def bbfmm_set_timing(plan, on=True):
    return _check(lib().bbfmm_set_timing(plan, 1 if on else 0))


def bbfmm_stage_times(plan):
    out = np.zeros(8, dtype=np.float32)
    _check(lib().bbfmm_stage_times(plan, _ptr(out)))
    return out


def bbfmm_status(plan):
    """Synchronize and return the device status word (raises on a timeout or
    a failed device-side check)."""
    w = ctypes.c_int(0)
    _check(lib().bbfmm_status(plan, ctypes.byref(w)))
    return w.value


def bbfmm_sort_points_static(points, depth, lo, side, perm, leaf_off, stream=None):
    """Leaf binning + Morton sort into caller buffers (device tensors) using
    the library's fixed scratch array; allocates nothing."""
    lo3 = (ctypes.c_double * 3)(*[float(v) for v in lo])
    return _check_plain(lib().bbfmm_sort_points_static(_ptr(points), int(points.shape[0]), int(depth), lo3,
                                                       float(side), _ptr(perm), _ptr(leaf_off),
                                                       _stream(stream)))


def bbfmm_rand_eig(plan, omega, k, power=0, vectors=True, stream=None):
    """Randomized eigen-decomposition of the plan's kernel matrix.  omega: a
    CUDA float32 tensor of shape (m, n) (n x m column-major).  Returns the k
    largest eigenvalues (numpy, decreasing) and, with ``vectors``, a CUDA
    tensor (k, n) of eigenvectors."""
    import torch
    m = int(omega.shape[0])
    evals = np.zeros(k, dtype=np.float64)
    evecs = torch.empty((k, omega.shape[1]), dtype=torch.float32, device=omega.device) if vectors else None
    _check(lib().bbfmm_rand_eig(plan, _ptr(omega.contiguous()), m, int(k), int(power),
                                evals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                _ptr(evecs) if vectors else None, _stream(stream)))
    return evals, evecs


def bbfmm_get_tuning(plan, nrhs=1) -> bbfmm_tuning:
    t = bbfmm_tuning()
    _check(lib().bbfmm_get_tuning(plan, int(nrhs), ctypes.byref(t)))
    return t


def bbfmm_set_tuning(plan, nrhs, near_mode, m2l_tile, m2l_stages=0, near_box=False, leaf_gemm=None):
    """near_mode: "ordered" / "symmetric" (or the BBFMM_NEAR_* value);
    leaf_gemm None keeps the plan's current choice for this nrhs."""
    if leaf_gemm is None:
        leaf_gemm = bool(bbfmm_get_tuning(plan, nrhs).leaf_gemm)
    t = bbfmm_tuning()
    t.leaf_gemm = 1 if leaf_gemm else 0
    t.near_mode = NEAR_MODES[near_mode] if isinstance(near_mode, str) else int(near_mode)
    t.m2l_tile = int(m2l_tile)
    t.m2l_stages = int(m2l_stages)
    t.near_box = 1 if near_box else 0
    return _check(lib().bbfmm_set_tuning(plan, int(nrhs), ctypes.byref(t)))


def bbfmm_autotune(plan, nrhs=1, stream=None):
    return _check(lib().bbfmm_autotune(plan, int(nrhs), _stream(stream)))


def bbfmm_matvec_launches(plan, nrhs=1):
    """Kernels one matvec with nrhs right-hand sides launches (the kernel
    nodes of its captured graph; a graphed matvec of that nrhs must have run)."""
    c = ctypes.c_int(0)
    _check(lib().bbfmm_matvec_launches(plan, int(nrhs), ctypes.byref(c)))
    return c.value


def _check_plain(st):
    # entry points that report only a status code (no message)
    if st != BBFMM_OK:
        raise BBFMMError(st, "")
    return st


STAGES = ["gather", "upward", "m2l", "downward", "l2p", "p2p", "combine", "total"]


class Plan:
    """Owning wrapper: ``Plan(points, kernel, p, depth, ...)``, then
    ``plan.matvec(sigma)`` with sigma a CUDA tensor (n,) or (nrhs, n).  With
    ``targets`` (nt, 3) the points are the sources and matvec returns the
    values at the targets, (nt,) or (nrhs, nt)."""

    def __init__(self, points, kernel, order, depth, ell=1.0, svd_eps=1e-7, precision="fp32",
                 domain=None, max_nrhs=1, stream=None, split_accumulate=True, use_graph=True,
                 keep_coefficients=False, targets=None, interp="chebyshev", near_mode="auto",
                 close_refine=True, autotune=True):
        import torch
        o = bbfmm_default_opts()
        o.split_accumulate = 1 if split_accumulate else 0
        o.use_graph = 1 if use_graph else 0
        o.keep_coefficients = 1 if keep_coefficients else 0
        o.close_refine = 1 if close_refine else 0
        o.autotune = 1 if autotune else 0
        o.interp = INTERPS[interp] if isinstance(interp, str) else int(interp)
        o.near_mode = NEAR_MODES[near_mode] if isinstance(near_mode, str) else int(near_mode)
        o.ell = float(ell)
        o.svd_eps = float(svd_eps)
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.max_nrhs = int(max_nrhs)
        if domain is not None:
            lo, side = domain
            o.domain_given = 1
            for d in range(3):
                o.lo[d] = float(lo[d])
            o.side = float(side)
        def f64(x):
            if isinstance(x, np.ndarray):
                return np.ascontiguousarray(x, dtype=np.float64)
            return x.to(torch.float64).contiguous()
        points = f64(points)
        self.n = int(points.shape[0])
        self.nt = self.n if targets is None else int(targets.shape[0])
        self.order = order
        self.depth = depth
        if targets is None:
            self.handle = bbfmm_plan(points, kernel, order, depth, o, stream)
        else:
            self.handle = bbfmm_plan_targets(points, f64(targets), kernel, order, depth, o, stream)

    def info(self):
        return bbfmm_plan_info(self.handle)

    def matvec(self, sigma, out=None, stream=None):
        import torch
        nrhs = 1 if sigma.dim() == 1 else int(sigma.shape[0])
        sigma = sigma.contiguous()
        if out is None:
            shape = (self.nt,) if sigma.dim() == 1 else (nrhs, self.nt)
            out = torch.empty(shape, dtype=torch.float32, device=sigma.device)
        bbfmm_matvec(self.handle, sigma, out, nrhs, stream)
        return out

    def close(self):
        if getattr(self, "handle", None) is not None:
            bbfmm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
