"""The symmetric near field (BBFMM_NEAR_SYMMETRIC: K(x, y) = K(y, x), so each
pair of neighbour leaves is evaluated once and used both ways, Sec. 2.5) against
the ordered one (BBFMM_NEAR_ORDERED: every target leaf evaluates all its
pairs), against the FP64 direct sum where the near field is the whole result
(depth 0 and 1: every leaf is a neighbour of every other), and against the
FP64 oracle FMM.  The two orders add the same FP32 terms in different orders,
so they agree to FP32 rounding, not bitwise."""
import numpy as np
import pytest

from paper_1903_02153_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K_INV_R, K_INV_R2, K_EXP, K_GAUSS, K_POLY, K_CONST = 1, 2, 3, 4, 100, 101
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


def make_plan(bb, pts, kid, p, depth, near_mode, ell=1.0, precision="fp32", max_nrhs=1, targets=None,
              autotune=True):
    dev = torch.device("cuda:0")
    return bb.Plan(torch.from_numpy(np.ascontiguousarray(pts)).to(dev), kid, p, depth, ell=ell, svd_eps=1e-7,
                   precision=precision, domain=UNIT, max_nrhs=max_nrhs, near_mode=near_mode, autotune=autotune,
                   targets=None if targets is None else torch.from_numpy(np.ascontiguousarray(targets)).to(dev))


def matvec(bb, plan, sig):
    s = torch.from_numpy(np.ascontiguousarray(np.asarray(sig, dtype=np.float32))).to("cuda:0")
    out = plan.matvec(s)
    assert bb.bbfmm_status(plan.handle) == 0
    return out.cpu().numpy().astype(np.float64)


def run(bb, pts, sig, kid, p, depth, near_mode, **kw):
    plan = make_plan(bb, pts, kid, p, depth, near_mode, **kw)
    info = plan.info()
    got = matvec(bb, plan, sig)
    plan.close()
    return got, info


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_auto_chooses_by_leaf_occupancy(bb):
    """Without the autotuner, AUTO takes the symmetric form when the
    near-field pairs per point / 27 (the occupancy of the leaves the work
    meets) is 16..48, and not on the clustered set, whose pairs sit in dense
    leaves."""
    cases = [(W.uniform_points(16384, seed=515), 3, 1), (W.uniform_points(2048, seed=515), 3, 0),
             (W.uniform_points(60_000, seed=515), 3, 0), (W.uniform_points(30_000, seed=515), 4, 0),
             (W.uniform_points(100_000, seed=515), 4, 1), (W.clustered_points(200_000, seed=515), 5, 0)]
    for pts, depth, want in cases:
        plan = make_plan(bb, pts, K_INV_R, 4, depth, "auto", autotune=False)
        info = plan.info()
        plan.close()
        occ = info.p2p_pairs / (27.0 * len(pts))
        assert info.near_symmetric == want, (len(pts), depth, occ)
        assert info.near_symmetric == (16 <= occ <= 48)


def test_symmetric_form_is_chosen_where_it_applies(bb):
    pts = W.uniform_points(5000, seed=501)
    for kid, want in [(K_INV_R, 1), (K_INV_R2, 1), (K_EXP, 1), (K_GAUSS, 1), (K_CONST, 1), (K_POLY, 0)]:
        plan = make_plan(bb, pts, kid, 4, 2, "symmetric")
        assert plan.info().near_symmetric == want, kid
        plan.close()
    plan = make_plan(bb, pts, K_INV_R, 4, 2, "ordered")
    assert plan.info().near_symmetric == 0
    plan.close()
    plan = make_plan(bb, pts, K_INV_R, 4, 2, "symmetric", targets=W.uniform_points(700, seed=502))
    assert plan.info().near_symmetric == 0   # targets apart from the sources
    plan.close()
    # run-time compiled kernels: as registered
    body = """
__device__ double bbfmm_kernel_f64(double d0, double d1, double d2)
{ return exp(-sqrt(d0 * d0 + d1 * d1 + d2 * d2) / 0.4); }
__device__ float bbfmm_kernel_f32(float d0, float d1, float d2)
{ return expf(-sqrtf(d0 * d0 + d1 * d1 + d2 * d2) / 0.4f); }
"""
    for symmetric in (True, False):
        kid = bb.bbfmm_kernel_register(body, symmetric=symmetric)
        plan = make_plan(bb, pts, kid, 4, 2, "symmetric")
        assert plan.info().near_symmetric == int(symmetric)
        plan.close()


def test_symmetric_user_kernel_matches_builtin(bb):
    """exp(-r / 0.4) restated as a registered symmetric kernel takes the
    symmetric near field too and gives the built-in's result to rounding."""
    body = """
__device__ double bbfmm_kernel_f64(double d0, double d1, double d2)
{ return exp(-sqrt(d0 * d0 + d1 * d1 + d2 * d2) / 0.4); }
__device__ float bbfmm_kernel_f32(float d0, float d1, float d2)
{ return expf(-sqrtf(d0 * d0 + d1 * d1 + d2 * d2) / 0.4f); }
"""
    kid = bb.bbfmm_kernel_register(body, symmetric=True)
    n = 40_000
    pts = W.clustered_points(n, seed=513)
    sig = W.uniform_sigma(n, seed=514)
    got, info = run(bb, pts, sig, kid, 5, 4, "symmetric")
    ref, info_b = run(bb, pts, sig, K_EXP, 5, 4, "symmetric", ell=0.4)
    assert info.near_symmetric == 1 and info_b.near_symmetric == 1
    assert rel(got, ref) <= 2e-6


@pytest.mark.parametrize("kid,ell,kind,n,p,depth", [
    (K_INV_R, 1.0, "uniform", 60_000, 5, 4),     # ~15 points per leaf, every leaf one work item
    (K_INV_R, 1.0, "uniform", 200_000, 5, 3),    # ~390 points per leaf: every leaf split (no slots written)
    (K_INV_R2, 1.0, "clustered", 20_000, 4, 4),  # split and whole leaves side by side
    (K_EXP, 0.3, "clustered", 100_000, 5, 5),
    (K_GAUSS, 0.5, "jittered_grid", 50_000, 5, 4),
    (K_CONST, 1.0, "uniform", 3000, 4, 3),
])
def test_symmetric_matches_ordered_and_oracle(bb, oracle, kid, ell, kind, n, p, depth):
    """Gate against the oracle: 1e-5 for both orders (the closest pairs
    enter through their FP64 corrections, computed for the frame each order
    evaluates them in)."""
    pts = W.make_points(kind, n, seed=503)
    sig = W.uniform_sigma(n, seed=504).astype(np.float32).astype(np.float64)
    got, info = run(bb, pts, sig, kid, p, depth, "symmetric", ell=ell)
    ordered, info_o = run(bb, pts, sig, kid, p, depth, "ordered", ell=ell)
    assert info.near_symmetric == 1 and info_o.near_symmetric == 0
    d = rel(got, ordered)
    print("%s %s n=%d d%d (max leaf %d): auto vs ordered %.2e" % (kid, kind, n, depth, info.max_leaf_points, d))
    assert d <= 3e-6
    if n <= 60_000:
        ref = oracle.bbfmm(pts, sig, kid, p, depth, ell=ell, lo=W.UNIT_LO, side=W.UNIT_SIDE)
        e, e_o = rel(got, ref), rel(ordered, ref)
        print("   vs oracle: auto %.2e, ordered %.2e" % (e, e_o))
        assert e <= 1e-5 and e_o <= 1e-5


@pytest.mark.parametrize("kid,ell", [(K_INV_R, 1.0), (K_INV_R2, 1.0), (K_EXP, 0.2), (K_GAUSS, 0.3)])
@pytest.mark.parametrize("depth,kind,n", [(0, "uniform", 100), (0, "uniform", 3000), (1, "uniform", 800),
                                          (1, "clustered", 900)])
def test_near_field_alone_is_the_direct_sum(bb, oracle, kid, ell, depth, kind, n):
    """Depth 0 / 1: no far field, every leaf pair is a near pair (with
    <= 128 points per leaf every pair of distinct leaves is taken both ways;
    the clustered set also has split leaves).  1/r^2 of the closest pairs
    costs a few 1e-6 in FP32 (the ordered form's gate too)."""
    pts = W.make_points(kind, n, seed=505)
    sig = W.uniform_sigma(n, seed=506).astype(np.float32).astype(np.float64)
    got, info = run(bb, pts, sig, kid, 4, depth, "symmetric", ell=ell)
    ref = oracle.direct(pts, pts, sig, kid, ell=ell)
    assert rel(got, ref) <= (5e-6 if kid == K_INV_R2 else 1e-6)


@pytest.mark.parametrize("n", [1, 2, 3, 129, 257])
def test_tiny_and_ragged_point_counts(bb, oracle, n):
    """One point (its own leaf only), two or three points in different leaves,
    and counts just past one and two work items in a single leaf; against the
    direct sum at depth 0 / 1 and the oracle FMM at depth 2 (which has a far
    field)."""
    pts = W.uniform_points(n, seed=507 + n)
    sig = W.uniform_sigma(n, seed=508 + n).astype(np.float32).astype(np.float64)
    for depth in (0, 1, 2):
        got, _ = run(bb, pts, sig, K_EXP, 4, depth, "symmetric", ell=0.5)
        if depth < 2:
            ref = oracle.direct(pts, pts, sig, K_EXP, ell=0.5)
        else:
            ref = oracle.bbfmm(pts, sig, K_EXP, 4, depth, ell=0.5, lo=W.UNIT_LO, side=W.UNIT_SIDE)
        assert rel(got, ref) <= 2e-6, (n, depth)


def test_symmetric_form_is_repeatable_bitwise(bb):
    pts = W.clustered_points(80_000, seed=509)
    sig = W.uniform_sigma(80_000, seed=510)
    plan = make_plan(bb, pts, K_INV_R, 5, 4, "symmetric", precision="fp16x3")
    a = matvec(bb, plan, sig)
    for _ in range(3):
        assert np.array_equal(matvec(bb, plan, sig), a)
    plan.close()


def test_several_rhs_between_single_rhs_calls(bb, oracle):
    """Several right-hand sides take the ordered form and leave the slots of
    the symmetric one alone: a one-RHS call after them gives the same bits,
    and every column matches the one-RHS result."""
    n = 30_000
    pts = W.uniform_points(n, seed=511)
    sig3 = W.uniform_sigma(n, nrhs=3, seed=512)
    plan = make_plan(bb, pts, K_EXP, 5, 4, "symmetric", ell=0.4, max_nrhs=3)
    first = matvec(bb, plan, sig3[:, 0])
    many = matvec(bb, plan, np.ascontiguousarray(sig3.T)).T
    again = matvec(bb, plan, sig3[:, 0])
    assert np.array_equal(first, again)
    for c in range(3):
        one = matvec(bb, plan, sig3[:, c])
        assert rel(many[:, c], one) <= 2e-6, c
    plan.close()
