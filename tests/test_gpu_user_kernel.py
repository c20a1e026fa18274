"""Kernels supplied by the caller (the black-box interface: the method needs
only evaluations of K, Sec. 1): CUDA C compiled at run time by
bbfmm_kernel_register, against the FP64 oracle evaluating the same formula
(written in C, oracle.use_user_kernel) and against the library's built-in
kernels.  Gates as elsewhere: <= 1e-5 from the oracle, error against the
direct sum <= 1.1 x the oracle's own."""
import numpy as np
import pytest

from paper_1903_02153_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

UNIT = (W.UNIT_LO, W.UNIT_SIDE)
K_INV_R, K_POLY = 1, 100

INV_R = """
__device__ double bbfmm_kernel_f64(double d0, double d1, double d2)
{ double r2 = d0 * d0 + d1 * d1 + d2 * d2; return r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0; }
__device__ float bbfmm_kernel_f32(float d0, float d1, float d2)
{ float r2 = d0 * d0 + d1 * d1 + d2 * d2; return r2 > 0.0f ? rsqrtf(r2) : 0.0f; }
"""

# inverse multiquadric 1 / sqrt(r^2 + c^2), c = 0.02: smooth, not homogeneous
IMQ = """
__device__ double bbfmm_kernel_f64(double d0, double d1, double d2)
{ return 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2 + 4e-4); }
__device__ float bbfmm_kernel_f32(float d0, float d1, float d2)
{ return rsqrtf(d0 * d0 + d1 * d1 + d2 * d2 + 4e-4f); }
"""
IMQ_C = "return 1.0 / sqrt(d0 * d0 + d1 * d1 + d2 * d2 + 4e-4);"

# not symmetric: exp(-|d| / 0.5) (1 + 0.3 d0)
SKEW = """
__device__ double bbfmm_kernel_f64(double d0, double d1, double d2)
{ return exp(-sqrt(d0 * d0 + d1 * d1 + d2 * d2) / 0.5) * (1.0 + 0.3 * d0); }
__device__ float bbfmm_kernel_f32(float d0, float d1, float d2)
{ return expf(-sqrtf(d0 * d0 + d1 * d1 + d2 * d2) / 0.5f) * (1.0f + 0.3f * d0); }
"""
SKEW_C = "return exp(-sqrt(d0 * d0 + d1 * d1 + d2 * d2) / 0.5) * (1.0 + 0.3 * d0);"

POLY = """
__device__ double bbfmm_kernel_f64(double d0, double d1, double d2)
{ return 1.0 + d0 - 2.0 * d1 * d2 + 3.0 * d0 * d0 * d1; }
__device__ float bbfmm_kernel_f32(float d0, float d1, float d2)
{ return 1.0f + d0 - 2.0f * d1 * d2 + 3.0f * d0 * d0 * d1; }
"""


@pytest.fixture(scope="module")
def bb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02153_gb300 import build
    build.build()
    from paper_1903_02153_gb300 import bbfmm
    bbfmm.lib()
    return bbfmm


@pytest.fixture(scope="module")
def kernels(bb):
    return {"inv_r": bb.bbfmm_kernel_register(INV_R, homogeneity=-1, symmetric=True),
            "imq": bb.bbfmm_kernel_register(IMQ, symmetric=True),
            "skew": bb.bbfmm_kernel_register(SKEW),
            "poly": bb.bbfmm_kernel_register(POLY)}


def run(bb, pts, sig, kid, p, depth, precision="fp32", interp="chebyshev", targets=None, eps=1e-7):
    dev = torch.device("cuda:0")
    sig = np.asarray(sig, dtype=np.float32)
    nrhs = 1 if sig.ndim == 1 else sig.shape[1]
    # the default launch choices, not the autotuner's measured ones: a user
    # kernel and the built-in it restates must run the same forms (the near
    # field's order and the leaf compression's form each move the result by
    # a few 1e-7) for their results to be compared at 1e-6
    plan = bb.Plan(torch.from_numpy(np.ascontiguousarray(pts)).to(dev), kid, p, depth, svd_eps=eps,
                   precision=precision, domain=UNIT, max_nrhs=nrhs, interp=interp, autotune=False,
                   targets=None if targets is None else torch.from_numpy(np.ascontiguousarray(targets)).to(dev))
    s = torch.from_numpy(np.ascontiguousarray(sig.T if nrhs > 1 else sig)).to(dev)
    out = plan.matvec(s)
    assert bb.bbfmm_status(plan.handle) == 0
    got = out.cpu().numpy().astype(np.float64)
    plan.close()
    return got.T if nrhs > 1 else got


def test_ids_are_distinct_and_above_the_builtins(bb, kernels):
    ids = list(kernels.values())
    assert len(set(ids)) == len(ids) and min(ids) >= bb.BBFMM_K_USER_FIRST


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_user_kernel_restating_inv_r_matches_the_builtin(bb, oracle, kernels, precision):
    n = 20_000
    pts = W.uniform_points(n, seed=401)
    sig = W.uniform_sigma(n, seed=402).astype(np.float32)
    got = run(bb, pts, sig, kernels["inv_r"], 5, 4, precision)
    ref_gpu = run(bb, pts, sig, K_INV_R, 5, 4, precision)
    ref = oracle.bbfmm(pts, sig.astype(np.float64), K_INV_R, 5, 4, lo=W.UNIT_LO, side=W.UNIT_SIDE)
    print("user 1/r %s: vs built-in %.2e, vs oracle %.2e" % (precision, oracle.rel_err(got, ref_gpu),
                                                              oracle.rel_err(got, ref)))
    assert oracle.rel_err(got, ref_gpu) < 1e-6
    assert oracle.rel_err(got, ref) <= 1e-5


@pytest.mark.parametrize("name,c_body,kind,p,depth,precision", [
    ("imq", IMQ_C, "uniform", 5, 4, "fp32"), ("imq", IMQ_C, "clustered", 5, 4, "fp16x3"),
    ("skew", SKEW_C, "uniform", 5, 3, "fp32"), ("skew", SKEW_C, "clustered", 6, 4, "tf32x3")])
def test_user_kernel_against_the_oracle(bb, oracle, kernels, name, c_body, kind, p, depth, precision):
    n = 20_000
    pts = W.make_points(kind, n, seed=403)
    sig = W.uniform_sigma(n, seed=404).astype(np.float32)
    got = run(bb, pts, sig, kernels[name], p, depth, precision)
    k = oracle.use_user_kernel(c_body)
    ref = oracle.bbfmm(pts, sig.astype(np.float64), k, p, depth, lo=W.UNIT_LO, side=W.UNIT_SIDE)
    idx = np.sort(np.random.default_rng(405).choice(n, 1500, replace=False))
    direct = oracle.direct(pts[idx], pts, sig.astype(np.float64), k)
    e_or = oracle.rel_err(ref[idx], direct)
    print("user %s %s p%d d%d %s: vs oracle %.2e, vs direct %.2e (oracle %.2e)"
          % (name, kind, p, depth, precision, oracle.rel_err(got, ref), oracle.rel_err(got[idx], direct), e_or))
    assert oracle.rel_err(got, ref) <= 1e-5
    # gate 2: errors add in quadrature, so it needs the GPU within ~0.46 e_or
    # of the oracle; the FP32 path sits ~1e-6 from it (gate 1), so gate 2 is
    # checked where the method's own error is above that floor (2e-6)
    if e_or >= 2e-6:
        assert oracle.rel_err(got[idx], direct) <= 1.1 * e_or


def test_user_polynomial_kernel_is_exact(bb, oracle, kernels):
    n = 6000
    pts = W.clustered_points(n, seed=406)
    sig = W.uniform_sigma(n, seed=407).astype(np.float32)
    got = run(bb, pts, sig, kernels["poly"], 4, 3, eps=0.0)
    direct = oracle.direct(pts, pts, sig.astype(np.float64), K_POLY)
    assert oracle.rel_err(got, direct) < 2e-6


def test_user_kernel_multiple_rhs(bb, oracle, kernels):
    n = 12_000
    pts = W.uniform_points(n, seed=408)
    sig = W.uniform_sigma(n, nrhs=3, seed=409).astype(np.float32)
    got = run(bb, pts, sig, kernels["imq"], 5, 4, "tf32x3")
    k = oracle.use_user_kernel(IMQ_C)
    ref = oracle.bbfmm(pts, sig.astype(np.float64), k, 5, 4, lo=W.UNIT_LO, side=W.UNIT_SIDE)
    for c in range(3):
        assert oracle.rel_err(got[:, c], ref[:, c]) <= 1e-5, c


def test_user_kernel_with_separate_targets_and_equally_spaced_nodes(bb, oracle, kernels):
    ns, nt = 15_000, 7_001
    src = W.uniform_points(ns, seed=410)
    tgt = W.clustered_points(nt, seed=411)
    sig = W.uniform_sigma(ns, seed=412).astype(np.float32)
    got = run(bb, src, sig, kernels["skew"], 5, 4, interp="uniform", targets=tgt)
    k = oracle.use_user_kernel(SKEW_C)
    ref = oracle.bbfmm_targets(src, sig.astype(np.float64), tgt, k, 5, 4, lo=W.UNIT_LO, side=W.UNIT_SIDE,
                               nodes="uniform")
    assert oracle.rel_err(got, ref) <= 1e-5


def test_bad_sources_are_rejected_with_the_compiler_log(bb):
    with pytest.raises(bb.BBFMMError, match="does not compile"):
        bb.bbfmm_kernel_register("__device__ double bbfmm_kernel_f64(double a, double b, double c) { return a +; }")
    with pytest.raises(bb.BBFMMError, match="bbfmm_kernel_f32"):   # the FP32 function is missing
        bb.bbfmm_kernel_register("__device__ double bbfmm_kernel_f64(double a, double b, double c) { return a; }")
