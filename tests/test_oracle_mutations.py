"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that
the pins of test_oracle_pins.py catch each one.  The oracle source itself is
not changed: each mutant is a textual edit of a temporary copy, compiled with
gcc and loaded under its own name."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1903_02153_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "bbfmm_oracle.c")

MUTANTS = {
    # M2L operator applied transposed
    "m2l_transposed": ("acc += K[(int64_t)i * p3 + j] * Mb", "acc += K[(int64_t)j * p3 + i] * Mb"),
    # M2L source box on the wrong side of the target box
    "m2l_offset_sign": ("double y0 = tx * h + 0.5 * h * t->s[j1];",
                        "double y0 = -tx * h + 0.5 * h * t->s[j1];"),
    # interaction list also drops the boxes two cells away along x
    "ilist_wrong_adjacency": ("int adjacent = dx >= -1 && dx <= 1", "int adjacent = dx >= -2 && dx <= 2"),
    # P2P forgets the target's own leaf
    "p2p_drops_self_leaf": ("int64_t bj = or_lex(D, nb[3 * k], nb[3 * k + 1], nb[3 * k + 2]);",
                            "int64_t bj = or_lex(D, nb[3 * k], nb[3 * k + 1], nb[3 * k + 2]);"
                            " if (bj == bi) continue;"),
    # L2L maps the child nodes with the child's box size instead of the parent's
    "l2l_wrong_frame": ("xs[0] = 2.0 * (x0 - cp[0]) / hp;", "xs[0] = 2.0 * (x0 - cp[0]) / hc;"),
    # M2M uses the child's centre in place of the parent's
    "m2m_wrong_centre": ("xs[1] = 2.0 * (y1 - cp[1]) / hp;", "xs[1] = 2.0 * (y1 - cc[1]) / hp;"),
    # P2M drops the last point of every leaf
    "p2m_drops_point": ("for (int64_t q = t->lstart[bi]; q < t->lstart[bi + 1]; ++q) {\n            int64_t j = t->order[q];\n            for (int d = 0; d < 3; ++d)\n                xs[d] = 2.0 * (t->pts[3 * j + d] - ctr[d]) / h;",
                        "for (int64_t q = t->lstart[bi]; q + 1 < t->lstart[bi + 1]; ++q) {\n            int64_t j = t->order[q];\n            for (int d = 0; d < 3; ++d)\n                xs[d] = 2.0 * (t->pts[3 * j + d] - ctr[d]) / h;"),
    # L2P reads the local coefficients of the wrong rhs column stride
    "l2p_index_swap": ("acc += F[(int64_t)r * p3 + j] * L[j];", "acc += F[(int64_t)r * p3 + j] * L[p3 - 1 - j];"),
    # far field on one level skipped
    "m2l_skips_level2": ("for (int l = 2; l <= D; ++l)\n        or_m2l(&t, l);",
                         "for (int l = 3; l <= D; ++l)\n        or_m2l(&t, l);"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mutated = src.replace(old, new)
    c = tmp_path / (name + ".c")
    so = tmp_path / ("lib" + name + ".so")
    c.write_text(mutated)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                    "-D_POSIX_C_SOURCE=199309L", str(c), "-o", str(so), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_int64)
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.oracle_bbfmm.argtypes = [i64, dp, dp, i32, i32, f64, i32, i32, dp, f64, i32, i64, lp, dp, dp, dp, dp]
    L.oracle_bbfmm.restype = i32
    L.oracle_uniform_nodes.argtypes = [i32, dp]
    return L


def _run(L, x, s, kid, p, D, nodes=0):
    dp = ctypes.POINTER(ctypes.c_double)
    x = np.ascontiguousarray(x)
    s = np.ascontiguousarray(s)
    lo = np.zeros(3)
    phi = np.zeros(x.shape[0])
    rc = L.oracle_bbfmm(x.shape[0], x.ctypes.data_as(dp), s.ctypes.data_as(dp), 1, kid, 1.0, p, D,
                        lo.ctypes.data_as(dp), 1.0, nodes, -1, None, phi.ctypes.data_as(dp), None, None, None)
    assert rc == 0
    return phi


@pytest.mark.parametrize("nodes", ["chebyshev", "uniform"])
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_polynomial_pin_catches_mutant(oracle, tmp_path, name, nodes):
    old, new = MUTANTS[name]
    L = _build_mutant(tmp_path, name, old, new)
    x = W.uniform_points(1200, seed=31)
    s = W.uniform_sigma(1200, seed=32)
    ref = oracle.direct(x, x, s, 100)
    # the unmutated oracle reproduces the polynomial kernel to rounding ...
    assert oracle.rel_err(oracle.bbfmm(x, s, 100, p=4, depth=3, lo=np.zeros(3), side=1.0, nodes=nodes), ref) < 1e-12
    # ... each mutant does not, with either node set
    err = oracle.rel_err(_run(L, x, s, 100, 4, 3, oracle.NODE_SETS[nodes]), ref)
    assert err > 1e-8, (name, err)


def test_node_formula_pin_catches_mutant(oracle, tmp_path):
    """Any distinct nodes reproduce a polynomial kernel, so a wrong spacing of
    the equally spaced nodes is caught by the closed-form pin instead."""
    L = _build_mutant(tmp_path, "uniform_spacing", "s[k - 1] = -1.0 + 2.0 * (k - 1.0) / (p - 1.0);",
                      "s[k - 1] = -1.0 + 2.0 * (k - 1.0) / p;")
    out = np.zeros(5)
    L.oracle_uniform_nodes(5, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    np.testing.assert_array_equal(oracle.uniform_nodes(5), np.linspace(-1.0, 1.0, 5))
    assert not np.allclose(out, np.linspace(-1.0, 1.0, 5))
