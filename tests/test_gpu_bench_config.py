"""The exact configurations bench.py times, gated against the oracle.

N = 1,048,576 uniform points, 1/r, p = 5, svd_eps = 1e-6, depth 5 and 6, one
right-hand side, run as the benchmark runs them (captured-graph replay): the
mixed form (FP16x3 tensor-core M2L) with the near field in AUTO and in
SYMMETRIC order, and the plain FP32 form (FP32 M2L, ordered near field).
On 4,096 sampled targets (Sec. 4.1 error measure on a sample; the oracle
evaluates the FMM and the direct sum at those targets only):

* gate 1: ||phi_gpu - phi_oracle|| / ||phi_oracle|| <= 1e-5;
* gate 2: err(phi_gpu vs direct) <= 1.1 err(phi_oracle vs direct);
* element-wise: max |phi_gpu - phi_oracle| / max |phi_oracle| <= 1e-5, which
  a few wrong leaves would fail even where the 2-norm passes.
"""
import numpy as np
import pytest

from paper_1903_02153_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 1 << 20
SAMPLE = 4096


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
def inputs():
    pts = W.uniform_points(N)
    sig = W.uniform_sigma(N).astype(np.float32)
    idx = np.sort(np.random.default_rng(1234).choice(N, SAMPLE, replace=False))
    return pts, sig, idx


_refs = {}


def references(oracle, inputs, depth):
    if depth not in _refs:
        pts, sig, idx = inputs
        s64 = sig.astype(np.float64)
        fmm = oracle.bbfmm(pts, s64, 1, 5, depth, lo=W.UNIT_LO, side=W.UNIT_SIDE, sample=idx)
        if "direct" not in _refs:
            _refs["direct"] = oracle.direct(pts[idx], pts, s64, 1)
        _refs[depth] = fmm
    return _refs[depth], _refs["direct"]


@pytest.mark.parametrize("depth", [5, 6])
@pytest.mark.parametrize("precision,near", [("fp16x3", "auto"), ("fp16x3", "symmetric"), ("fp32", "ordered")])
def test_benchmark_configuration_meets_both_gates(bb, oracle, inputs, depth, precision, near):
    pts, sig, idx = inputs
    dev = torch.device("cuda:0")
    plan = bb.Plan(torch.from_numpy(pts).to(dev), 1, 5, depth, svd_eps=1e-6, precision=precision,
                   domain=(W.UNIT_LO, W.UNIT_SIDE), near_mode=near)
    s = torch.from_numpy(sig).to(dev)
    phi = plan.matvec(s)
    again = plan.matvec(s)            # graph replay: the same bits
    torch.cuda.synchronize()
    assert torch.equal(phi, again)
    assert bb.bbfmm_status(plan.handle) == 0
    info = plan.info()
    plan.close()
    got = phi.cpu().numpy().astype(np.float64)[idx]
    ref, direct = references(oracle, inputs, depth)
    e1 = oracle.rel_err(got, ref)
    e_or = oracle.rel_err(ref, direct)
    e_gpu = oracle.rel_err(got, direct)
    emax = np.abs(got - ref).max() / np.abs(ref).max()
    print("depth %d %s %s (symmetric near field %d, %d close pairs): |gpu-oracle| %.2e, max-elem %.2e, "
          "err vs direct %.3e (oracle %.3e)" % (depth, precision, near, info.near_symmetric, info.close_pairs,
                                                e1, emax, e_gpu, e_or))
    if near == "symmetric":
        assert info.near_symmetric == 1
    assert e1 <= 1e-5
    assert e_gpu <= 1.1 * e_or
    assert emax <= 1e-5
