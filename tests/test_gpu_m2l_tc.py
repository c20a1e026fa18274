"""The tensor-core M2L (tcgen05: TF32, split 3xTF32, FP16x3, BF16x3) against
the FP64 oracle and the FP32 CUDA-core M2L, from the smallest tree up.

The split forms keep ~21 mantissa bits per product and sum the offsets in FP32
registers, so against the oracle they must be at least as close as the FP32
CUDA-core form (whose own FP32 accumulation over 189 offsets x r terms costs
~2e-6 at depth 5), and within the FP32 gates of the oracle (1e-5, and 1.1 x
the oracle's error against the direct sum).  One-pass TF32 (10 bits) is
reported with a loose bound only."""
import numpy as np
import pytest

from paper_1903_02153_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

UNIT = (W.UNIT_LO, W.UNIT_SIDE)


@pytest.fixture(scope="module")
def bb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02153_gb300 import build
    build.build()
    from paper_1903_02153_gb300 import bbfmm
    bbfmm.lib()
    return bbfmm


def run(bb, pts, sig, kid, p, depth, precision, ell=1.0, eps=1e-7, nrhs=1):
    dev = torch.device("cuda:0")
    plan = bb.Plan(torch.from_numpy(pts).to(dev), kid, p, depth, ell=ell, svd_eps=eps, precision=precision,
                   domain=UNIT, max_nrhs=nrhs)
    s = torch.from_numpy(np.ascontiguousarray(sig.T if nrhs > 1 else sig).astype(np.float32)).to(dev)
    phi = plan.matvec(s)
    status = bb.bbfmm_status(plan.handle)
    out = phi.cpu().numpy().astype(np.float64)
    plan.close()
    assert status == 0
    return out.T if nrhs > 1 else out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
@pytest.mark.parametrize("n,p,depth", [(2000, 4, 2), (6000, 4, 3), (20000, 5, 4), (60000, 5, 5)])
def test_split3_at_least_as_close_as_fp32(bb, oracle, n, p, depth, prec):
    pts = W.uniform_points(n, seed=71)
    sig = W.uniform_sigma(n, seed=72).astype(np.float32)
    a = run(bb, pts, sig, 1, p, depth, "fp32")
    b = run(bb, pts, sig, 1, p, depth, prec)
    samp = np.random.default_rng(73).choice(n, min(n, 3000), replace=False)
    ref = oracle.bbfmm(pts, sig.astype(np.float64), 1, p, depth, lo=W.UNIT_LO, side=W.UNIT_SIDE, sample=samp)
    e_fp32, e_split = oracle.rel_err(a[samp], ref), oracle.rel_err(b[samp], ref)
    assert e_split <= 1.1 * e_fp32 + 2e-7, (e_split, e_fp32)
    assert e_split <= 1e-5
    assert rel(b, a) < 4e-6   # the two forms differ by about the FP32 form's own error


def test_bf16x3_error_is_reported(bb, oracle):
    """Two-piece BF16 carries ~16 bits: reported against the oracle, bounded
    loosely (it is not one of the gated forms)."""
    n = 20000
    pts = W.uniform_points(n, seed=79)
    sig = W.uniform_sigma(n, seed=80).astype(np.float32)
    got = run(bb, pts, sig, 1, 5, 4, "bf16x3")
    ref = oracle.bbfmm(pts, sig.astype(np.float64), 1, 5, 4, lo=W.UNIT_LO, side=W.UNIT_SIDE)
    e = oracle.rel_err(got, ref)
    print("bf16x3 vs oracle: %.2e" % e)
    assert e < 1e-3


def test_tf32_one_pass_is_close(bb):
    pts = W.uniform_points(20000, seed=73)
    sig = W.uniform_sigma(20000, seed=74).astype(np.float32)
    a = run(bb, pts, sig, 1, 5, 4, "fp32")
    b = run(bb, pts, sig, 1, 5, 4, "tf32")
    e = rel(b, a)
    print("one-pass tf32 vs fp32: %.2e" % e)
    assert e < 1e-3


@pytest.mark.parametrize("kid,ell,kind,p,depth,eps,tol", [(3, 0.3, "clustered", 6, 4, 1e-7, 1e-5),
                                                          (2, 1.0, "uniform", 5, 4, 1e-7, 1e-5),
                                                          (1, 1.0, "uniform", 5, 4, 0.0, 1e-5)])
def test_tf32x3_vs_oracle(bb, oracle, kid, ell, kind, p, depth, eps, tol):
    """Against the oracle (uncompressed for 1/r).  The near field's closest
    pairs enter through their FP64 corrections, so 1/r^2 is held to the same
    1e-5 (with FP32 leaf-local coordinates alone those pairs cost 1.02e-5
    here).  The tensor-core forms track the FP32 form to within that form's
    own FP32 error."""
    n = 20000
    pts = W.make_points(kind, n, seed=75)
    sig = W.uniform_sigma(n, seed=76).astype(np.float32)
    got = run(bb, pts, sig, kid, p, depth, "tf32x3", ell=ell, eps=eps)
    half = run(bb, pts, sig, kid, p, depth, "fp16x3", ell=ell, eps=eps)
    plain = run(bb, pts, sig, kid, p, depth, "fp32", ell=ell, eps=eps)
    ref = oracle.bbfmm(pts, sig.astype(np.float64), kid, p, depth, ell=ell, lo=W.UNIT_LO, side=W.UNIT_SIDE)
    print("kernel %d: tf32x3 vs oracle %.2e, fp32 vs oracle %.2e" % (kid, oracle.rel_err(got, ref),
                                                                      oracle.rel_err(plain, ref)))
    assert oracle.rel_err(got, ref) <= tol
    assert rel(got, plain) < 4e-6
    assert oracle.rel_err(half, ref) <= tol
    assert rel(half, plain) < 4e-6


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
def test_split3_multiple_rhs(bb, prec):
    n = 12000
    pts = W.uniform_points(n, seed=77)
    sig = W.uniform_sigma(n, nrhs=4, seed=78).astype(np.float32)
    sig[:, 2] *= 1e4    # columns of very different magnitude share one scale per level
    a = run(bb, pts, sig, 1, 4, 4, "fp32", nrhs=4)
    b = run(bb, pts, sig, 1, 4, 4, prec, nrhs=4)
    for c in range(4):   # the small columns keep their accuracy under the shared FP16 scale
        assert rel(b[:, c], a[:, c]) < 2e-6, (c, rel(b[:, c], a[:, c]))


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "fp16x3", "bf16x3"])
def test_fewer_columns_than_the_plan_holds(bb, prec):
    """A plan made for 8 right-hand sides, called with 1, 3 and 8 columns (in
    that order, then 1 again): each call equals the same columns run through a
    plan made for exactly that many."""
    n = 15000
    dev = torch.device("cuda:0")
    pts = W.clustered_points(n, seed=81)
    sig = W.uniform_sigma(n, nrhs=8, seed=82).astype(np.float32)
    plan = bb.Plan(torch.from_numpy(pts).to(dev), 1, 4, 4, svd_eps=1e-7, precision=prec, domain=UNIT, max_nrhs=8)
    tol = 2e-5 if prec == "bf16x3" else 1e-6
    for k in (1, 3, 8, 1):
        s = torch.from_numpy(np.ascontiguousarray(sig[:, :k].T)).to(dev)
        got = plan.matvec(s if k > 1 else s[0]).cpu().numpy().astype(np.float64)
        got = got.T if k > 1 else got[:, None]
        assert bb.bbfmm_status(plan.handle) == 0
        want = run(bb, pts, sig[:, :k] if k > 1 else sig[:, 0], 1, 4, 4, prec, nrhs=k)
        want = want if k > 1 else want[:, None]
        for c in range(k):
            assert rel(got[:, c], want[:, c]) < tol, (k, c, rel(got[:, c], want[:, c]))
    plan.close()


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
@pytest.mark.parametrize("depth", [5, 6])
def test_split3_full_size_uniform_1M(bb, oracle, depth, prec):
    c = W.CONFIGS["uniform-1M-p5-d6"]
    n = c["n"]
    pts = W.uniform_points(n)
    sig = W.uniform_sigma(n).astype(np.float32)
    got = run(bb, pts, sig, 1, 5, depth, prec)
    plain = run(bb, pts, sig, 1, 5, depth, "fp32")
    idx = np.sort(np.random.default_rng(62).choice(n, 400, replace=False))
    ref = oracle.bbfmm(pts, sig.astype(np.float64), 1, 5, depth, lo=W.UNIT_LO, side=W.UNIT_SIDE, sample=idx)
    direct = oracle.direct(pts[idx], pts, sig.astype(np.float64), 1)
    e_or = oracle.rel_err(ref, direct)
    print("depth %d %s: vs fp32 %.2e, vs oracle %.2e, err %.2e (oracle %.2e)"
          % (depth, prec, rel(got, plain), oracle.rel_err(got[idx], ref), oracle.rel_err(got[idx], direct), e_or))
    assert rel(got, plain) < 4e-6
    assert oracle.rel_err(got[idx], ref) <= 1e-5
    assert oracle.rel_err(got[idx], direct) <= 1.1 * e_or


@pytest.mark.parametrize("depth", [5, 6])
@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_clustered_points_visit_only_occupied_tiles(bb, oracle, depth, prec):
    """Clustered points leave most boxes empty; the tensor-core M2L then visits
    only the tiles holding occupied targets.  Against the oracle at sampled
    targets, and against the FP32 form (which computes every tile)."""
    n = 200_000
    pts = W.clustered_points(n, seed=83)
    sig = W.uniform_sigma(n, seed=84).astype(np.float32)
    got = run(bb, pts, sig, 3, 5, depth, prec, ell=0.3)
    plain = run(bb, pts, sig, 3, 5, depth, "fp32", ell=0.3)
    idx = np.sort(np.random.default_rng(85).choice(n, 300, replace=False))
    ref = oracle.bbfmm(pts, sig.astype(np.float64), 3, 5, depth, ell=0.3, lo=W.UNIT_LO, side=W.UNIT_SIDE, sample=idx)
    assert oracle.rel_err(got[idx], ref) <= 1e-5
    assert rel(got, plain) < 4e-6


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
@pytest.mark.parametrize("eps", [1e-7, 1e-8])
def test_rank_above_128_runs_in_row_halves(bb, oracle, prec, eps):
    """exp(-r/0.3) at p = 6 has level ranks up to 152 (eps 1e-7) and 184
    (eps 1e-8): the coarse levels run each tile as two halves of 128 operator
    rows, the fine levels at their own lower rank.  Against the uncompressed
    oracle and the FP32 form."""
    n = 30_000
    pts = W.clustered_points(n, seed=86)
    sig = W.uniform_sigma(n, seed=87).astype(np.float32)
    dev = torch.device("cuda:0")
    plan = bb.Plan(torch.from_numpy(pts).to(dev), 3, 6, 4, ell=0.3, svd_eps=eps, precision=prec, domain=UNIT)
    assert plan.info().rank > 128
    plan.close()
    got = run(bb, pts, sig, 3, 6, 4, prec, ell=0.3, eps=eps)
    plain = run(bb, pts, sig, 3, 6, 4, "fp32", ell=0.3, eps=eps)
    ref = oracle.bbfmm(pts, sig.astype(np.float64), 3, 6, 4, ell=0.3, lo=W.UNIT_LO, side=W.UNIT_SIDE)
    print("rank>128 %s eps %.0e: vs oracle %.2e, fp32 vs oracle %.2e, vs fp32 %.2e"
          % (prec, eps, oracle.rel_err(got, ref), oracle.rel_err(plain, ref), rel(got, plain)))
    assert oracle.rel_err(got, ref) <= 1e-5
    assert rel(got, plain) < 4e-6
