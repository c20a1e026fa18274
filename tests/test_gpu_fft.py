"""Equally spaced nodes with the Fourier-domain M2L (Sec. 2.2 node sets,
Sec. 2.5 "Fast M2L translation"): the CUDA path (forward DFT per box,
189-term sum per frequency, inverse DFT per box, FP32) against the FP64
oracle with the same node set, whose M2L is the dense operator K(x*_i, y*_j)
(the block-Toeplitz matrix the DFTs apply).  Gates as for the Chebyshev
path: relative 2-norm difference from the oracle <= 1e-5, error against the
direct sum <= 1.1 x the oracle's own."""
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


def run(bb, pts, sig, kid, p, depth, ell=1.0, keep=False, targets=None):
    dev = torch.device("cuda:0")
    sig = np.asarray(sig, dtype=np.float32)
    nrhs = 1 if sig.ndim == 1 else sig.shape[1]
    plan = bb.Plan(torch.from_numpy(np.ascontiguousarray(pts)).to(dev), kid, p, depth, ell=ell, domain=UNIT,
                   max_nrhs=max(nrhs, 2), interp="uniform", keep_coefficients=keep,
                   targets=None if targets is None else torch.from_numpy(np.ascontiguousarray(targets)).to(dev))
    s = torch.from_numpy(np.ascontiguousarray(sig.T if nrhs > 1 else sig)).to(dev)
    phi = plan.matvec(s)
    assert bb.bbfmm_status(plan.handle) == 0
    out = phi.cpu().numpy().astype(np.float64)
    out = out.T if nrhs > 1 else out
    if keep:
        return out, plan
    plan.close()
    return out


def oracle_u(oracle, pts, sig, kid, p, depth, ell=1.0, **kw):
    return oracle.bbfmm(pts, np.asarray(sig, dtype=np.float32).astype(np.float64), kid, p, depth, ell=ell,
                        lo=W.UNIT_LO, side=W.UNIT_SIDE, nodes="uniform", **kw)


@pytest.mark.parametrize("kid,ell,p,depth,kind", [(K_INV_R, 1.0, 4, 3, "uniform"), (K_INV_R, 1.0, 5, 4, "uniform"),
                                                  (K_EXP, 0.3, 5, 4, "clustered"), (K_GAUSS, 0.5, 4, 3, "uniform"),
                                                  (K_INV_R, 1.0, 6, 4, "uniform"), (K_EXP, 1.0, 7, 3, "uniform"),
                                                  (K_INV_R2, 1.0, 5, 3, "uniform"), (K_EXP, 0.3, 3, 5, "clustered")])
def test_fft_m2l_matches_uniform_node_oracle(bb, oracle, kid, ell, p, depth, kind):
    """Singular kernels run on uniform points only: on clustered points the
    near field's FP32 leaf-local coordinates dominate the 1/r error (very
    close pairs), as on the Chebyshev path; the far field on clustered points
    is checked stage by stage below."""
    n = 20_000
    pts = W.make_points(kind, n, seed=301)
    sig = W.uniform_sigma(n, seed=302).astype(np.float32)
    got = run(bb, pts, sig, kid, p, depth, ell)
    ref = oracle_u(oracle, pts, sig, kid, p, depth, ell)
    idx = np.sort(np.random.default_rng(303).choice(n, 1500, replace=False))
    direct = oracle.direct(pts[idx], pts, sig.astype(np.float64), kid, ell)
    e_or = oracle.rel_err(ref[idx], direct)
    e = oracle.rel_err(got, ref)
    print("fft m2l k%d p%d d%d %s: vs oracle %.2e, vs direct %.2e (oracle %.2e)"
          % (kid, p, depth, kind, e, oracle.rel_err(got[idx], direct), e_or))
    assert e <= 1e-5
    # gate 2: errors add in quadrature, so it needs the GPU within ~0.46 e_or
    # of the oracle; the FP32 path sits ~1e-6 from it (gate 1), so gate 2 is
    # checked where the method's own error is above that floor (2e-6)
    if e_or >= 2e-6:
        assert oracle.rel_err(got[idx], direct) <= 1.1 * e_or


@pytest.mark.parametrize("p,depth", [(3, 3), (4, 4)])
def test_fft_polynomial_kernel_is_exact(bb, oracle, p, depth):
    n = 6000
    pts = W.clustered_points(n, seed=304)
    sig = W.uniform_sigma(n, seed=305).astype(np.float32)
    got = run(bb, pts, sig, K_POLY, p, depth)
    direct = oracle.direct(pts, pts, sig.astype(np.float64), K_POLY)
    assert oracle.rel_err(got, direct) < 2e-6


@pytest.mark.parametrize("depth", [0, 1])
def test_fft_depth0_1_is_direct_sum(bb, oracle, depth):
    n = 3000
    pts = W.uniform_points(n, seed=306)
    sig = W.uniform_sigma(n, seed=307).astype(np.float32)
    got = run(bb, pts, sig, K_EXP, 4, depth, 0.5)
    assert oracle.rel_err(got, oracle.direct(pts, pts, sig.astype(np.float64), K_EXP, 0.5)) < 1e-6


@pytest.mark.parametrize("p,depth,kind", [(4, 3, "uniform"), (5, 4, "clustered")])
def test_fft_stage_coefficients_match_oracle(bb, oracle, p, depth, kind):
    """M (upward pass, U = V = I) and F (after the Fourier-domain M2L and
    L2L) on every level against the oracle's stage outputs."""
    n = 12_000
    pts = W.make_points(kind, n, seed=308)
    sig = W.uniform_sigma(n, seed=309).astype(np.float32)
    got, plan = run(bb, pts, sig, K_INV_R, p, depth, keep=True)
    ref, Ms, Fs = oracle_u(oracle, pts, sig, K_INV_R, p, depth, dump=True)
    cells = oracle.leaf_cells(pts, W.UNIT_LO, W.UNIT_SIDE, depth)
    for l in range(2, depth + 1):
        gm = bb.bbfmm_get_coefficients(plan.handle, 0, l, 1, p)
        gf = bb.bbfmm_get_coefficients(plan.handle, 1, l, 1, p)
        assert oracle.rel_err(gm, Ms[l]) < 2e-6, ("M", l)
        c = cells >> (depth - l)
        occ = np.unique(c[:, 0] + 2 ** l * (c[:, 1] + 2 ** l * c[:, 2]))
        assert oracle.rel_err(gf[occ], Fs[l][occ]) < 5e-6, ("F", l, oracle.rel_err(gf[occ], Fs[l][occ]))
    plan.close()
    assert oracle.rel_err(got, ref) < 5e-6


def test_fft_multiple_rhs(bb, oracle):
    n = 15_000
    pts = W.uniform_points(n, seed=310)
    sig = W.uniform_sigma(n, nrhs=3, seed=311).astype(np.float32)
    sig[:, 1] *= 1e3
    got = run(bb, pts, sig, K_EXP, 5, 4, 0.5)
    ref = oracle_u(oracle, pts, sig, K_EXP, 5, 4, 0.5)
    for c in range(3):
        assert oracle.rel_err(got[:, c], ref[:, c]) <= 1e-5, c


def test_fft_separate_targets(bb, oracle):
    ns, nt = 15_000, 9_001
    src = W.uniform_points(ns, seed=312)
    tgt = W.clustered_points(nt, seed=313)
    sig = W.uniform_sigma(ns, seed=314).astype(np.float32)
    got = run(bb, src, sig, K_INV_R, 5, 4, targets=tgt)
    ref = oracle.bbfmm_targets(src, sig.astype(np.float64), tgt, K_INV_R, 5, 4, lo=W.UNIT_LO, side=W.UNIT_SIDE,
                               nodes="uniform")
    assert got.shape == (nt,)
    assert oracle.rel_err(got, ref) <= 1e-5


def test_fft_same_result_eager_and_graph_and_repeated(bb):
    n = 50_000
    dev = torch.device("cuda:0")
    pts = torch.from_numpy(W.uniform_points(n, seed=315)).to(dev)
    sig = torch.from_numpy(W.uniform_sigma(n, seed=316).astype(np.float32)).to(dev)
    a = bb.Plan(pts, K_INV_R, 5, 5, domain=UNIT, interp="uniform", use_graph=False)
    b = bb.Plan(pts, K_INV_R, 5, 5, domain=UNIT, interp="uniform")
    ra = a.matvec(sig).cpu().numpy()
    rb1 = b.matvec(sig).cpu().numpy()
    rb2 = b.matvec(sig).cpu().numpy()
    a.close()
    b.close()
    np.testing.assert_array_equal(ra, rb1)
    np.testing.assert_array_equal(rb1, rb2)


@pytest.mark.parametrize("depth", [5, 6])
def test_fft_full_size_uniform_1M(bb, oracle, depth):
    n = 1 << 20
    pts = W.uniform_points(n)
    sig = W.uniform_sigma(n).astype(np.float32)
    got = run(bb, pts, sig, K_INV_R, 5, depth)
    idx = np.sort(np.random.default_rng(317).choice(n, 300, replace=False))
    ref = oracle_u(oracle, pts, sig, K_INV_R, 5, depth, sample=idx)
    direct = oracle.direct(pts[idx], pts, sig.astype(np.float64), K_INV_R)
    e_or = oracle.rel_err(ref, direct)
    print("fft 1M depth %d: vs oracle %.2e, vs direct %.2e (oracle %.2e)"
          % (depth, oracle.rel_err(got[idx], ref), oracle.rel_err(got[idx], direct), e_or))
    assert oracle.rel_err(got[idx], ref) <= 1e-5
    assert oracle.rel_err(got[idx], direct) <= 1.1 * e_or
