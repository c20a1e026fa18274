"""Targets apart from the sources (Sec. 1: phi(x_i) = sum_j K(x_i, y_j)
sigma_j with {x_i} and {y_j} different sets), through bbfmm_plan_targets,
against the FP64 oracle FMM with the same target set (oracle.bbfmm_targets)
and the FP64 direct sum.  Gates as for the square matvec: relative 2-norm
difference from the oracle <= 1e-5, error against the direct sum <= 1.1 x the
oracle's own."""
import ctypes

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


def gpu_targets(bb, src, sig, tgt, kid, p, depth, ell=1.0, eps=1e-7, precision="fp32", domain=UNIT):
    dev = torch.device("cuda:0")
    sig = np.asarray(sig, dtype=np.float32)
    nrhs = 1 if sig.ndim == 1 else sig.shape[1]
    plan = bb.Plan(torch.from_numpy(np.ascontiguousarray(src)).to(dev), kid, p, depth, ell=ell, svd_eps=eps,
                   precision=precision, domain=domain, max_nrhs=nrhs,
                   targets=torch.from_numpy(np.ascontiguousarray(tgt)).to(dev))
    s = torch.from_numpy(np.ascontiguousarray(sig.T if nrhs > 1 else sig)).to(dev)
    phi = plan.matvec(s)
    status = bb.bbfmm_status(plan.handle)
    out = phi.cpu().numpy().astype(np.float64)
    plan.close()
    assert status == 0
    return out.T if nrhs > 1 else out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", ["fp32", "fp16x3", "tf32x3"])
@pytest.mark.parametrize("kid,ell,p,depth", [(K_INV_R, 1.0, 5, 4), (K_EXP, 0.3, 5, 3), (K_GAUSS, 0.5, 4, 3)])
def test_targets_match_oracle_and_direct(bb, oracle, kid, ell, p, depth, precision):
    """Uniform sources, clustered targets of a different count (ragged leaves
    of both sets)."""
    ns, nt = 20_000, 13_001
    src = W.uniform_points(ns, seed=201)
    tgt = W.clustered_points(nt, seed=202)
    sig = W.uniform_sigma(ns, seed=203).astype(np.float32)
    got = gpu_targets(bb, src, sig, tgt, kid, p, depth, ell=ell, precision=precision)
    ref = oracle.bbfmm_targets(src, sig.astype(np.float64), tgt, kid, p, depth, ell=ell, lo=W.UNIT_LO,
                               side=W.UNIT_SIDE)
    idx = np.sort(np.random.default_rng(204).choice(nt, 1500, replace=False))
    direct = oracle.direct(tgt[idx], src, sig.astype(np.float64), kid, ell)
    e_or = oracle.rel_err(ref[idx], direct)
    print("targets k%d %s: vs oracle %.2e, vs direct %.2e (oracle %.2e)"
          % (kid, precision, oracle.rel_err(got, ref), oracle.rel_err(got[idx], direct), e_or))
    assert got.shape == (nt,)
    assert oracle.rel_err(got, ref) <= 1e-5
    assert oracle.rel_err(got[idx], direct) <= 1.1 * e_or


def test_polynomial_kernel_is_exact(bb, oracle):
    """A cubic kernel is reproduced exactly by Chebyshev interpolation with
    p >= 4 (Sec. 2.1), so the FMM at separate targets equals the direct sum
    up to FP32 rounding."""
    ns, nt = 6000, 4500
    src = W.uniform_points(ns, seed=205)
    tgt = W.uniform_points(nt, seed=206)
    sig = W.uniform_sigma(ns, seed=207).astype(np.float32)
    got = gpu_targets(bb, src, sig, tgt, K_POLY, 4, 3, eps=0.0)
    direct = oracle.direct(tgt, src, sig.astype(np.float64), K_POLY)
    assert rel(got, direct) < 2e-6


def test_same_points_as_targets_equal_the_square_plan(bb):
    """Targets = sources through the separate-target entry point gives the
    square plan's result bit for bit (same tree, same kernels, same order:
    the square plan with the ordered near field, which a target set always
    takes, and both with the default launch choices rather than each its own
    measured ones)."""
    n = 30_000
    dev = torch.device("cuda:0")
    pts = torch.from_numpy(W.clustered_points(n, seed=208)).to(dev)
    sig = torch.from_numpy(W.uniform_sigma(n, seed=209).astype(np.float32)).to(dev)
    for prec in ("fp32", "fp16x3"):
        a = bb.Plan(pts, K_INV_R, 5, 5, precision=prec, domain=UNIT, near_mode="ordered", autotune=False)
        b = bb.Plan(pts, K_INV_R, 5, 5, precision=prec, domain=UNIT, targets=pts.clone(), autotune=False)
        pa, pb = a.matvec(sig).cpu().numpy(), b.matvec(sig).cpu().numpy()
        ia, ib = a.info(), b.info()
        a.close()
        b.close()
        np.testing.assert_array_equal(pa, pb)
        assert ib.n_targets == n and ia.n_targets == n and ia.p2p_pairs == ib.p2p_pairs


def test_targets_on_sources_follow_the_r0_convention(bb, oracle):
    """Half the targets sit exactly on sources: the singular kernels take
    K = 0 there, like the oracle (and like the square matvec's diagonal)."""
    ns = 12_000
    src = W.uniform_points(ns, seed=210)
    rng = np.random.default_rng(211)
    tgt = np.concatenate([src[rng.choice(ns, 4000, replace=False)], W.uniform_points(4000, seed=212)])
    sig = W.uniform_sigma(ns, seed=213).astype(np.float32)
    for kid in (K_INV_R, K_INV_R2):
        got = gpu_targets(bb, src, sig, tgt, kid, 5, 4)
        ref = oracle.bbfmm_targets(src, sig.astype(np.float64), tgt, kid, 5, 4, lo=W.UNIT_LO, side=W.UNIT_SIDE)
        assert np.all(np.isfinite(got))
        assert oracle.rel_err(got, ref) <= (1e-5 if kid == K_INV_R else 2e-5)


@pytest.mark.parametrize("depth", [4, 5])
def test_few_clustered_targets_far_from_most_sources(bb, oracle, depth):
    """Targets in one small cube (most tree boxes hold no target, so the
    tensor-core M2L visits few tiles), sources everywhere; with the default
    domain (the bounding cube of both sets)."""
    ns, nt = 60_000, 3000
    src = W.uniform_points(ns, seed=214) * 2.0 - 0.5
    tgt = W.uniform_points(nt, seed=215) * 0.1 + np.array([0.2, 0.6, 0.3])
    sig = W.uniform_sigma(ns, seed=216).astype(np.float32)
    dev = torch.device("cuda:0")
    out = {}
    for prec in ("fp32", "fp16x3"):
        plan = bb.Plan(torch.from_numpy(src).to(dev), K_INV_R, 5, depth, precision=prec,
                       targets=torch.from_numpy(tgt).to(dev))
        info = plan.info()
        lo, side = oracle.bounding_cube(np.concatenate([src, tgt]))
        np.testing.assert_array_equal(np.array(info.lo[:]), lo)
        assert info.side == side and info.n == ns and info.n_targets == nt
        out[prec] = plan.matvec(torch.from_numpy(sig).to(dev)).cpu().numpy().astype(np.float64)
        plan.close()
    ref = oracle.bbfmm_targets(src, sig.astype(np.float64), tgt, K_INV_R, 5, depth)
    for prec, got in out.items():
        assert oracle.rel_err(got, ref) <= 1e-5, prec


def test_multiple_rhs_and_host_buffers(bb, oracle):
    """Four right-hand sides through the C ABI with host sigma (ns x 4) and
    host phi (nt x 4): the binding's staging copies use the two sizes."""
    ns, nt, nrhs = 9000, 7000, 4
    src = W.uniform_points(ns, seed=217)
    tgt = W.uniform_points(nt, seed=218)
    sig = np.asfortranarray(W.uniform_sigma(ns, nrhs=nrhs, seed=219).astype(np.float32))
    o = bb.bbfmm_default_opts()
    o.max_nrhs = nrhs
    o.domain_given, o.side = 1, W.UNIT_SIDE
    for d in range(3):
        o.lo[d] = W.UNIT_LO[d]
    o.precision = bb.PRECISIONS["tf32x3"]
    h = bb.bbfmm_plan_targets(src, tgt, K_EXP, 5, 4, o)
    phi = np.zeros((nt, nrhs), dtype=np.float32, order="F")
    phi[:] = np.nan
    bb.bbfmm_matvec(h, sig, phi, nrhs)
    info = bb.bbfmm_plan_info(h)
    bb.bbfmm_destroy(h)
    ref = oracle.bbfmm_targets(src, sig.astype(np.float64), tgt, K_EXP, 5, 4, ell=1.0, lo=W.UNIT_LO,
                               side=W.UNIT_SIDE)
    assert info.n == ns and info.n_targets == nt
    for c in range(nrhs):
        assert oracle.rel_err(phi[:, c], ref[:, c]) <= 1e-5, c


def test_p2p_pairs_count_targets_times_neighbour_sources(bb, oracle):
    ns, nt, depth = 5000, 3000, 3
    src = W.clustered_points(ns, seed=220)
    tgt = W.uniform_points(nt, seed=221)
    plan = bb.Plan(torch.from_numpy(src).cuda(), K_INV_R, 4, depth, domain=UNIT, targets=torch.from_numpy(tgt).cuda())
    info = plan.info()
    plan.close()
    cs = oracle.leaf_cells(src, W.UNIT_LO, W.UNIT_SIDE, depth)
    ct = oracle.leaf_cells(tgt, W.UNIT_LO, W.UNIT_SIDE, depth)
    m = 1 << depth
    hs = np.zeros((m, m, m), dtype=np.int64)
    np.add.at(hs, (cs[:, 0], cs[:, 1], cs[:, 2]), 1)
    pad = np.pad(hs, 1)
    near = sum(pad[1 + dx:1 + dx + m, 1 + dy:1 + dy + m, 1 + dz:1 + dz + m]
               for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1))
    assert info.p2p_pairs == int(near[ct[:, 0], ct[:, 1], ct[:, 2]].sum())
    assert info.nonempty_leaves == int((hs > 0).sum()) and info.max_leaf_points == int(hs.max())


def test_bad_arguments(bb):
    dev = torch.device("cuda:0")
    src = torch.from_numpy(W.uniform_points(500, seed=222)).to(dev)
    tgt = torch.from_numpy(W.uniform_points(300, seed=223)).to(dev)
    plan = bb.Plan(src, K_INV_R, 4, 2, domain=UNIT, targets=tgt, max_nrhs=4)
    with pytest.raises(bb.BBFMMError):       # the kernel matrix is not square
        bb.bbfmm_rand_eig(plan.handle, torch.randn(4, 500, device=dev), 2)
    plan.close()
    o = bb.bbfmm_default_opts()
    o.domain_given, o.side = 1, 1.0
    with pytest.raises(bb.BBFMMError):       # a target outside the given domain
        bb.bbfmm_plan_targets(src, tgt + 2.0, K_INV_R, 4, 2, o)
    h = ctypes.c_void_p()
    st = bb.lib().bbfmm_plan_targets(bb._ptr(src), 500, None, 300, K_INV_R, 4, 2, None, None, ctypes.byref(h))
    assert st == bb.BBFMM_EINVAL and h.value is None
