"""Python handle on the FP64 CPU oracle (bbfmm_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference legs of ``bench.py`` use it.  Nothing in the CUDA
package imports it, and it imports nothing from that package.

The C source follows the paper's definitions (Sec. 1 Eq. summation; Sec. 2.1
Def. 2.1; Sec. 2.2 Def. 2.2, Eq. low-rank-form; the four stages of Sec. 2.3).  This
module only compiles it with gcc, marshals numpy arrays, and adds the default
domain rule (bounding cube of the points).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bbfmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

K_INV_R, K_INV_R2, K_EXP, K_GAUSS, K_POLY, K_CONST = 1, 2, 3, 4, 100, 101
SINGULAR = {K_INV_R: -1, K_INV_R2: -2}   # kernel id -> degree of homogeneity


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP); returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-D_POSIX_C_SOURCE=199309L", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(ctypes.c_int64)
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            L.oracle_direct.argtypes = [i64, dp, i64, dp, dp, i32, i32, f64, dp]
            L.oracle_direct.restype = None
            L.oracle_bbfmm.argtypes = [i64, dp, dp, i32, i32, f64, i32, i32, dp, f64, i32,
                                       i64, lp, dp, dp, dp, dp]
            L.oracle_bbfmm.restype = i32
            L.oracle_bbfmm_targets.argtypes = [i64, dp, dp, i32, i32, f64, i32, i32, dp, f64, i32, i64, dp, dp, dp]
            L.oracle_bbfmm_targets.restype = i32
            L.oracle_cheb_nodes.argtypes = [i32, dp]
            L.oracle_set_user_kernel.argtypes = [ctypes.c_void_p]
            L.oracle_set_user_kernel.restype = None
            L.oracle_uniform_nodes.argtypes = [i32, dp]
            L.oracle_lagrange_1d.argtypes = [i32, dp, f64, dp]
            L.oracle_neighbors.argtypes = [i32, i64, i64, i64, lp]
            L.oracle_neighbors.restype = i32
            L.oracle_interaction_list.argtypes = [i32, i64, i64, i64, lp]
            L.oracle_interaction_list.restype = i32
            L.oracle_leaf_cells.argtypes = [i64, dp, dp, f64, i32, lp]
            L.oracle_kernel_matrix.argtypes = [i64, dp, i32, f64, dp]
            L.oracle_kernel_matrix.restype = None
            L.oracle_kernel.argtypes = [i32, f64, dp, dp]
            L.oracle_kernel.restype = f64
            L.oracle_num_threads.restype = i32
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _f64c(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _sigma_colmajor(sigma, n):
    s = np.asarray(sigma, dtype=np.float64)
    if s.ndim == 1:
        s = s[:, None]
    assert s.shape[0] == n
    return np.asfortranarray(s), s.shape[1]


def bounding_cube(points):
    """Default domain: lo = per-axis minimum, side = largest extent (1 if all
    points coincide).  Cells are min(floor((x-lo)/h), 2^D-1), so points on the
    upper face fall into the last cell."""
    pts = np.asarray(points, dtype=np.float64)
    lo = pts.min(axis=0)
    side = float((pts.max(axis=0) - lo).max())
    if not side > 0.0:
        side = 1.0
    return lo, side


def num_threads() -> int:
    return int(lib().oracle_num_threads())


K_USER = 1000   # the caller-supplied kernel set by use_user_kernel
_user_libs = {}


def use_user_kernel(c_body):
    """Make K_USER the kernel k(d) = the C function body ``c_body`` of
    ``double k(double d0, double d1, double d2)`` (d = x - y), compiled with
    gcc into its own small library (the caller states the kernel; the oracle
    only evaluates it).  Returns K_USER."""
    import hashlib
    key = hashlib.sha256(c_body.encode()).hexdigest()[:16]
    if key not in _user_libs:
        os.makedirs(_BUILD, exist_ok=True)
        src = os.path.join(_BUILD, "user_%s.c" % key)
        so = os.path.join(_BUILD, "libuser_%s.so" % key)
        with open(src, "w") as fh:
            fh.write("#include <math.h>\ndouble bbfmm_oracle_user_k(double d0, double d1, double d2)\n{\n%s\n}\n"
                     % c_body)
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", src, "-o", so, "-lm"], check=True)
        _user_libs[key] = ctypes.CDLL(so)
    fn = ctypes.cast(_user_libs[key].bbfmm_oracle_user_k, ctypes.c_void_p)
    lib().oracle_set_user_kernel(fn)
    return K_USER


def kernel(kid, x, y, ell=1.0):
    x = _f64c(x, (3,))
    y = _f64c(y, (3,))
    return float(lib().oracle_kernel(kid, ell, _dp(x), _dp(y)))


def direct(targets, sources, sigma, kid, ell=1.0):
    """FP64 direct sum (Eq. summation); sigma is (ns,) or (ns, nrhs)."""
    x = _f64c(targets)
    y = _f64c(sources)
    s, nrhs = _sigma_colmajor(sigma, y.shape[0])
    out = np.zeros((x.shape[0], nrhs), dtype=np.float64, order="F")
    lib().oracle_direct(x.shape[0], _dp(x), y.shape[0], _dp(y), _dp(s), nrhs, kid, ell, _dp(out))
    return out[:, 0] if np.ndim(sigma) == 1 else out


def kernel_matrix(points, kid, ell=1.0):
    """Dense FP64 kernel matrix K[i][j] = K(x_i, x_j) (the covariance matrix
    of the randomized PCA of Sec. 4.3); n x n, so small n only."""
    x = _f64c(points)
    n = x.shape[0]
    out = np.zeros((n, n), dtype=np.float64)
    lib().oracle_kernel_matrix(n, _dp(x), kid, ell, _dp(out))
    return out


def top_eigenvalues(points, kid, k, ell=1.0):
    """The k largest eigenvalues of the dense kernel matrix (numpy's symmetric
    eigensolver on kernel_matrix), in decreasing order."""
    w = np.linalg.eigvalsh(kernel_matrix(points, kid, ell))
    return w[::-1][:k].copy()


def rand_eig(K, omega, k, power=0):
    """The randomized PCA of Sec. 4.3 on a dense FP64 matrix, step by step
    (the randomized range finder with `power` subspace iterations, then the
    Rayleigh-Ritz eigen-decomposition of Halko, Martinsson & Tropp): Y = K W
    with W = omega^T (n x m); Q = qr(Y); repeat Y = K Q, Q = qr(Y) `power`
    times; B = Q^T K Q = V L V^T.  Returns the k largest eigenvalues
    (decreasing) and the matching columns of Q V."""
    Q, _ = np.linalg.qr(K @ np.asarray(omega, dtype=np.float64).T)
    for _ in range(power):
        Q, _ = np.linalg.qr(K @ Q)
    B = Q.T @ (K @ Q)
    w, V = np.linalg.eigh(0.5 * (B + B.T))
    order = np.argsort(w)[::-1][:k]
    return w[order], Q @ V[:, order]


def cheb_nodes(p):
    out = np.zeros(p)
    lib().oracle_cheb_nodes(p, _dp(out))
    return out


def uniform_nodes(p):
    out = np.zeros(p)
    lib().oracle_uniform_nodes(p, _dp(out))
    return out


def lagrange_1d(p, x, nodes="chebyshev"):
    s = cheb_nodes(p) if nodes == "chebyshev" else uniform_nodes(p)
    out = np.zeros(p)
    lib().oracle_lagrange_1d(p, _dp(s), float(x), _dp(out))
    return out


def neighbors(level, a, b, c):
    out = np.zeros((27, 3), dtype=np.int64)
    n = lib().oracle_neighbors(level, a, b, c, _lp(out))
    return out[:n]


def interaction_list(level, a, b, c):
    out = np.zeros((189, 3), dtype=np.int64)
    n = lib().oracle_interaction_list(level, a, b, c, _lp(out))
    return out[:n]


def leaf_cells(points, lo, side, depth):
    pts = _f64c(points)
    lo = _f64c(lo, (3,))
    out = np.zeros((pts.shape[0], 3), dtype=np.int64)
    lib().oracle_leaf_cells(pts.shape[0], _dp(pts), _dp(lo), float(side), depth, _lp(out))
    return out


NODE_SETS = {"chebyshev": 0, "uniform": 1}


def bbfmm(points, sigma, kid, p, depth, ell=1.0, lo=None, side=None, sample=None,
          dump=False, times=False, nodes="chebyshev"):
    """FP64 black-box FMM (Sec. 2.3).  Returns phi (n,) / (n, nrhs), or for a
    ``sample`` of target indices phi at those targets only.  With ``dump`` also
    returns lists M[l], F[l] of arrays (8^l, nrhs, p^3) in lexicographic box
    order; with ``times`` the four stage times in seconds.  ``nodes``: the
    interpolation node set, "chebyshev" or "uniform" (equally spaced, Sec. 2.2),
    the M2L always the dense operator K(x*_i, y*_j)."""
    pts = _f64c(points)
    n = pts.shape[0]
    s, nrhs = _sigma_colmajor(sigma, n)
    if lo is None or side is None:
        lo, side = bounding_cube(pts)
    lo = _f64c(lo, (3,))
    if sample is None:
        ns, samp, nout = -1, None, n
    else:
        samp = np.ascontiguousarray(sample, dtype=np.int64)
        ns, nout = samp.shape[0], samp.shape[0]
    phi = np.zeros((nout, nrhs), dtype=np.float64, order="F")
    p3 = p ** 3
    tot = sum(8 ** l for l in range(depth + 1)) * nrhs * p3
    Md = np.zeros(tot) if dump else None
    Fd = np.zeros(tot) if dump else None
    tm = np.zeros(4)
    rc = lib().oracle_bbfmm(n, _dp(pts), _dp(s), nrhs, kid, float(ell), p, depth, _dp(lo),
                            float(side), NODE_SETS[nodes], ns, _lp(samp) if samp is not None else None,
                            _dp(phi), _dp(Md) if dump else None, _dp(Fd) if dump else None,
                            _dp(tm))
    if rc != 0:
        raise ValueError("oracle_bbfmm rejected its arguments")
    res = phi[:, 0] if np.ndim(sigma) == 1 else phi
    extra = []
    if dump:
        Ms, Fs, off = [], [], 0
        for l in range(depth + 1):
            cnt = 8 ** l * nrhs * p3
            Ms.append(Md[off:off + cnt].reshape(8 ** l, nrhs, p3))
            Fs.append(Fd[off:off + cnt].reshape(8 ** l, nrhs, p3))
            off += cnt
        extra += [Ms, Fs]
    if times:
        extra.append(tm)
    return (res, *extra) if extra else res


def bbfmm_targets(sources, sigma, targets, kid, p, depth, ell=1.0, lo=None, side=None, nodes="chebyshev"):
    """FP64 black-box FMM with a target set apart from the sources (Sec. 1:
    the two sets may differ).  Both must lie in the cubical domain (default:
    the bounding cube of their union).  Returns phi at the targets, (nt,) or
    (nt, nrhs)."""
    src = _f64c(sources)
    tgt = _f64c(targets)
    s, nrhs = _sigma_colmajor(sigma, src.shape[0])
    if lo is None or side is None:
        lo, side = bounding_cube(np.concatenate([src, tgt]))
    lo = _f64c(lo, (3,))
    phi = np.zeros((tgt.shape[0], nrhs), dtype=np.float64, order="F")
    rc = lib().oracle_bbfmm_targets(src.shape[0], _dp(src), _dp(s), nrhs, kid, float(ell), p, depth, _dp(lo),
                                    float(side), NODE_SETS[nodes], tgt.shape[0], _dp(tgt), _dp(phi), None)
    if rc != 0:
        raise ValueError("oracle_bbfmm_targets rejected its arguments")
    return phi[:, 0] if np.ndim(sigma) == 1 else phi


def rel_err(approx, exact):
    """||approx - exact||_2 / ||exact||_2 (Sec. 4.1 error measure; Frobenius
    over all columns for several right-hand sides)."""
    a = np.asarray(approx, dtype=np.float64)
    e = np.asarray(exact, dtype=np.float64)
    return float(np.linalg.norm(a - e) / np.linalg.norm(e))
