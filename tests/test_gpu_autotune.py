"""The autotuner (opts.autotune, bbfmm_autotune / bbfmm_get_tuning /
bbfmm_set_tuning): launch choices per nrhs -- the near-field order of one-RHS
matvecs, the tensor-core M2L's tile size and pipeline depth -- measured and
kept per plan, cached per process.  Sec. 2.5 "Multiple right-hand-sides": the
work per launch grows with nrhs, and the best cut moves with it.

A choice changes how the work is cut, never what is computed: every
candidate's result is within FP32 rounding of every other's and within the
gates against the oracle, and a plan run with the tuner's choice gives the
same bits as a plan told that choice explicitly.
"""
import itertools

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


def make(bb, pts, kid=1, p=5, depth=4, precision="fp16x3", nrhs=1, autotune=True, ell=1.0):
    return bb.Plan(torch.from_numpy(pts).cuda(), kid, p, depth, ell=ell, svd_eps=1e-7, precision=precision,
                   domain=UNIT, max_nrhs=nrhs, autotune=autotune)


def sigma_dev(sig):
    return torch.from_numpy(np.ascontiguousarray(sig.T if sig.ndim == 2 else sig)).cuda()


def candidates(bb, plan, nrhs):
    """Every (near order, tile, stages, box items, leaf GEMM) the plan accepts
    for this nrhs."""
    ok = []
    for near, tile, st, box, lg in itertools.product(["ordered", "symmetric"], [128, 256], [0, 2, 3, 4],
                                                     [False, True], [False, True]):
        try:
            bb.bbfmm_set_tuning(plan.handle, nrhs, near, tile, st, near_box=box, leaf_gemm=lg)
        except bb.BBFMMError as e:
            assert e.status == bb.BBFMM_EINVAL
            continue
        ok.append((near, tile, st, box, lg))
    return ok


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kind,kid,ell,p,depth,precision", [("uniform", 1, 1.0, 5, 4, "fp16x3"),
                                                            ("clustered", 3, 0.3, 5, 5, "fp16x3"),
                                                            ("uniform", 2, 1.0, 4, 4, "tf32x3"),
                                                            ("uniform", 1, 1.0, 4, 4, "fp32")])
def test_every_candidate_gives_the_same_result(bb, oracle, kind, kid, ell, p, depth, precision):
    n = 60_000
    pts = W.make_points(kind, n, seed=700)
    sig = W.uniform_sigma(n, seed=701).astype(np.float32)
    plan = make(bb, pts, kid, p, depth, precision, ell=ell)
    cands = candidates(bb, plan, 1)
    if precision in ("fp16x3", "bf16x3"):
        assert {c[1] for c in cands} == {128, 256}
    assert {c[0] for c in cands} == {"ordered", "symmetric"}
    assert {(c[0], c[3]) for c in cands} == {("ordered", False), ("ordered", True), ("symmetric", False)}
    assert {c[4] for c in cands} == {False, True}     # the leaf compression GEMM or the pass
    s = sigma_dev(sig)
    outs = {}
    for c in cands:
        bb.bbfmm_set_tuning(plan.handle, 1, *c)
        t = bb.bbfmm_get_tuning(plan.handle, 1)
        assert (t.m2l_tile, t.m2l_stages, t.measured, t.near_box, t.leaf_gemm) == (
            c[1], c[2], 0, int(c[3]), int(c[4]))
        outs[c] = plan.matvec(s).cpu().numpy().astype(np.float64)
        assert bb.bbfmm_status(plan.handle) == 0
    plan.close()
    idx = np.sort(np.random.default_rng(702).choice(n, 2000, replace=False))
    ref = oracle.bbfmm(pts, sig.astype(np.float64), kid, p, depth, ell=ell, lo=W.UNIT_LO, side=W.UNIT_SIDE,
                       sample=idx)
    base = outs[cands[0]]
    for c, out in outs.items():
        d, e = rel(out, base), rel(out[idx], ref)
        print("%s %s k%d %s: vs first candidate %.2e, vs oracle %.2e" % (kind, precision, kid, c, d, e))
        assert d <= 2e-6          # another order of the same FP32 sums
        assert e <= 1e-5


def test_tuned_choice_is_a_candidate_and_reproducible(bb):
    n = 100_000
    pts = W.uniform_points(n, seed=703)
    sig = sigma_dev(W.uniform_sigma(n, seed=704).astype(np.float32))
    plan = make(bb, pts)
    t0 = bb.bbfmm_get_tuning(plan.handle, 1)
    assert t0.measured == 0               # nothing measured before the first matvec
    a = plan.matvec(sig).clone()          # the first matvec tunes (or takes the cache)
    t = bb.bbfmm_get_tuning(plan.handle, 1)
    assert t.measured == 1
    assert (t.near_mode, t.m2l_tile) in {(m, tl) for m in (1, 2) for tl in (128, 256)}
    bb.bbfmm_autotune(plan.handle, 1)     # measure again explicitly
    assert bb.bbfmm_get_tuning(plan.handle, 1).measured == 1
    # a plan told the first choice explicitly gives the same bits
    other = make(bb, pts, autotune=False)
    bb.bbfmm_set_tuning(other.handle, 1, t.near_mode, t.m2l_tile, t.m2l_stages, t.near_box, t.leaf_gemm)
    bb.bbfmm_set_tuning(plan.handle, 1, t.near_mode, t.m2l_tile, t.m2l_stages, t.near_box, t.leaf_gemm)
    b, c = plan.matvec(sig), other.matvec(sig)
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(b, c)
    # a second plan of the same shape takes the cached choice at its first matvec
    again = make(bb, pts)
    again.matvec(sig)
    t2 = bb.bbfmm_get_tuning(again.handle, 1)
    assert t2.measured == 1
    for pl in (plan, other, again):
        assert bb.bbfmm_status(pl.handle) == 0
        pl.close()


def test_several_rhs_and_defaults(bb):
    n = 50_000
    pts = W.uniform_points(n, seed=705)
    sig = W.uniform_sigma(n, nrhs=8, seed=706).astype(np.float32)
    plan = make(bb, pts, nrhs=8)
    with pytest.raises(bb.BBFMMError) as ei:   # the symmetric order is one-RHS only
        bb.bbfmm_set_tuning(plan.handle, 8, "symmetric", 256, 0)
    assert ei.value.status == bb.BBFMM_EINVAL
    with pytest.raises(bb.BBFMMError):         # no such tile size
        bb.bbfmm_set_tuning(plan.handle, 8, "ordered", 64, 0)
    with pytest.raises(bb.BBFMMError):         # more stages than fit
        bb.bbfmm_set_tuning(plan.handle, 8, "ordered", 256, 7)
    with pytest.raises(bb.BBFMMError):         # box items are a one-RHS form
        bb.bbfmm_set_tuning(plan.handle, 8, "ordered", 256, 0, near_box=True)
    cands = candidates(bb, plan, 8)
    assert cands and all(c[0] == "ordered" for c in cands)
    s = sigma_dev(sig)
    outs = []
    for c in cands:
        bb.bbfmm_set_tuning(plan.handle, 8, *c)
        outs.append(plan.matvec(s).cpu().numpy().astype(np.float64))
    for o in outs[1:]:
        assert rel(o, outs[0]) <= 2e-6
    plan.close()
    fixed = make(bb, pts, nrhs=8, autotune=False)
    fixed.matvec(s)
    t = bb.bbfmm_get_tuning(fixed.handle, 8)
    assert (t.measured, t.m2l_tile, t.m2l_stages, t.near_mode, t.near_box, t.leaf_gemm) == (0, 256, 0, 1, 0, 1)
    fixed.close()


@pytest.mark.parametrize("kind,n,depth", [("uniform", 300_000, 6), ("clustered", 200_000, 5), ("uniform", 5000, 1)])
def test_box_items_match_leaf_items(bb, oracle, kind, n, depth):
    """Leaves of a few points: the ordered near field by level-(D-1) box
    items gives the leaf items' result to FP32 rounding, and both match the
    oracle (the close pairs corrected in each form's frame)."""
    pts = W.make_points(kind, n, seed=707)
    sig = W.uniform_sigma(n, seed=708).astype(np.float32)
    plan = make(bb, pts, 1, 4, depth, "fp16x3")
    s = sigma_dev(sig)
    tile = bb.bbfmm_get_tuning(plan.handle, 1).m2l_tile
    bb.bbfmm_set_tuning(plan.handle, 1, "ordered", tile, 0, near_box=False)
    a = plan.matvec(s).cpu().numpy().astype(np.float64)
    bb.bbfmm_set_tuning(plan.handle, 1, "ordered", tile, 0, near_box=True)
    b = plan.matvec(s).cpu().numpy().astype(np.float64)
    assert bb.bbfmm_get_tuning(plan.handle, 1).near_box == 1
    assert bb.bbfmm_status(plan.handle) == 0
    plan.close()
    idx = np.sort(np.random.default_rng(709).choice(n, min(n, 1500), replace=False))
    ref = oracle.bbfmm(pts, sig.astype(np.float64), 1, 4, depth, lo=W.UNIT_LO, side=W.UNIT_SIDE, sample=idx)
    print("%s n=%d d%d: box vs leaf items %.2e; vs oracle %.2e / %.2e"
          % (kind, n, depth, rel(b, a), rel(b[idx], ref), rel(a[idx], ref)))
    assert rel(b, a) <= 2e-6
    assert rel(b[idx], ref) <= 1e-5 and rel(a[idx], ref) <= 1e-5


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "fp16x3", "bf16x3"])
@pytest.mark.parametrize("depth,nrhs,kind", [(2, 1, "uniform"), (5, 1, "uniform"), (6, 1, "clustered"),
                                             (4, 3, "uniform")])
def test_leaf_compression_gemm_matches_the_pass(bb, oracle, precision, depth, nrhs, kind):
    """The leaf level's compression as a 3 x TF32 tensor-core GEMM gives the
    pass's FP32 compression to FP32 rounding, for every M2L form (FP32 M~,
    its TF32 split, the 16-bit split with the level scale from the GEMM's max),
    one and several right-hand sides (a plan holding more columns than the
    call uses)."""
    n = {2: 3000, 4: 40_000, 5: 200_000, 6: 300_000}[depth]
    pts = W.make_points(kind, n, seed=710 + depth)
    sig = W.uniform_sigma(n, nrhs=nrhs, seed=711).astype(np.float32)
    plan = bb.Plan(torch.from_numpy(pts).cuda(), 1, 5, depth, svd_eps=1e-7, precision=precision, domain=UNIT,
                   max_nrhs=nrhs + 1, autotune=False)
    s = sigma_dev(sig)
    t = bb.bbfmm_get_tuning(plan.handle, nrhs)
    assert t.leaf_gemm == 1
    a = plan.matvec(s).cpu().numpy().astype(np.float64)
    bb.bbfmm_set_tuning(plan.handle, nrhs, t.near_mode, t.m2l_tile, t.m2l_stages, t.near_box, leaf_gemm=False)
    b = plan.matvec(s).cpu().numpy().astype(np.float64)
    assert bb.bbfmm_status(plan.handle) == 0
    plan.close()
    a, b = (a.T, b.T) if nrhs > 1 else (a, b)
    idx = np.sort(np.random.default_rng(712).choice(n, min(n, 1000), replace=False))
    ref = oracle.bbfmm(pts, sig.astype(np.float64), 1, 5, depth, lo=W.UNIT_LO, side=W.UNIT_SIDE, sample=idx)
    d, e = rel(a, b), rel(a[idx], ref)
    print("%s depth %d nrhs %d: GEMM vs pass %.2e, GEMM vs oracle %.2e" % (precision, depth, nrhs, d, e))
    assert d <= (2e-5 if precision == "bf16x3" else 2e-6)
    assert e <= (1e-4 if precision == "bf16x3" else 1e-5)


@pytest.mark.parametrize("kid,leaf_launches", [(1, 2), (3, 4)])
def test_launch_count_of_the_captured_graph(bb, kid, leaf_launches):
    """bbfmm_matvec_launches counts the kernel nodes of the matvec graph.  The
    leaf GEMMs add one compression and one decompression launch when the
    leaves and level D-1 share the operator (1/r: one scaled operator for
    every level), two each when they do not (exp(-r/ell): an operator per
    level).  The count is unavailable until a graph is captured, and again
    after a tuning change drops it."""
    n = 40_000
    pts = W.make_points("uniform", n, seed=720)
    s = sigma_dev(W.uniform_sigma(n, seed=721).astype(np.float32))
    plan = make(bb, pts, kid, 5, 4, "fp16x3", autotune=False, ell=0.3 if kid == 3 else 1.0)
    with pytest.raises(bb.BBFMMError):
        bb.bbfmm_matvec_launches(plan.handle, 1)
    tile = bb.bbfmm_get_tuning(plan.handle, 1).m2l_tile
    counts = {}
    for lg in (True, False):
        bb.bbfmm_set_tuning(plan.handle, 1, "ordered", tile, 0, leaf_gemm=lg)
        with pytest.raises(bb.BBFMMError):
            bb.bbfmm_matvec_launches(plan.handle, 1)
        plan.matvec(s)
        counts[lg] = bb.bbfmm_matvec_launches(plan.handle, 1)
    assert bb.bbfmm_status(plan.handle) == 0
    plan.close()
    # gather, upward pass, 16-bit split, near field, M2L, two downward launches, combine
    assert counts[False] >= 8
    assert counts[True] - counts[False] == leaf_launches
