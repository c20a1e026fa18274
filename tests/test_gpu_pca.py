"""Randomized eigen-decomposition of the kernel matrix (the randomized PCA of
Sec. 4.3) through bbfmm_rand_eig, against the same algorithm on the dense
FP64 kernel matrix (oracle.rand_eig, same test block) and against a dense
eigensolver."""
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


def run(bb, pts, kid, ell, p, depth, omega, k, power, precision="fp32"):
    dev = torch.device("cuda:0")
    plan = bb.Plan(torch.from_numpy(pts).to(dev), kid, p, depth, ell=ell, svd_eps=1e-7, precision=precision,
                   domain=UNIT, max_nrhs=omega.shape[0])
    w, U = bb.bbfmm_rand_eig(plan.handle, torch.from_numpy(omega).to(dev), k, power=power)
    plan.close()
    return w, U.cpu().numpy().T.astype(np.float64)


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_gp_covariance_matches_dense_randomized_pca(bb, oracle, precision):
    """exp(-r/0.2) covariance on a jittered lattice (the paper's GP setting),
    60 test vectors, one subspace iteration: the leading 10 eigenvalues equal
    those of the same algorithm on the exact FP64 matrix to the FMM's accuracy,
    and the leading 3 equal the true ones."""
    n, kid, ell, m, k = 4000, 3, 0.2, 60, 10
    pts = W.make_points("jittered_grid", n, seed=95)
    omega = W.normal_sigma(n, m, seed=96).T.astype(np.float32)
    w, U = run(bb, pts, kid, ell, 5, 3, omega, k, 1, precision)
    K = oracle.kernel_matrix(pts, kid, ell)
    w_ref, _ = oracle.rand_eig(K, omega.astype(np.float64), k, power=1)
    exact = oracle.top_eigenvalues(pts, kid, k, ell)
    print("rand_eig %s: vs dense randomized %.2e, vs exact (top 3) %.2e"
          % (precision, np.max(np.abs(w - w_ref)) / w_ref[0], np.max(np.abs(w[:3] - exact[:3]) / exact[:3])))
    assert np.max(np.abs(w - w_ref)) <= 2e-5 * w_ref[0]
    assert np.max(np.abs(w[:3] - exact[:3]) / exact[:3]) <= 1e-3
    # eigenvectors: unit norm, and K u = lambda u to the accuracy of lambda
    np.testing.assert_allclose(np.linalg.norm(U, axis=0), 1.0, rtol=1e-4)
    res = np.linalg.norm(K @ U[:, :3] - U[:, :3] * w[:3], axis=0) / w[0]
    assert res.max() < 1e-2


def test_constant_kernel_has_one_eigenvalue(bb):
    """K = 1 1^T: a single eigenvalue N; the others are FP32 rounding noise of
    the matvec (K Omega has rank 1 up to ~1e-7 relative), below 1e-7 N."""
    n = 5000
    pts = W.uniform_points(n, seed=99)
    omega = W.normal_sigma(n, 8, seed=100).T.astype(np.float32)
    w, U = run(bb, pts, 101, 1.0, 4, 3, omega, 3, 0)
    assert abs(w[0] - n) <= 1e-5 * n
    assert np.all(np.abs(w[1:]) <= 1e-7 * n)
    # the eigenvector is the constant direction (cosine of the angle ~ 1)
    assert abs(np.sum(U[:, 0]) / np.sqrt(n)) >= 1.0 - 1e-5


def test_bad_arguments(bb):
    dev = torch.device("cuda:0")
    pts = W.uniform_points(1000, seed=101)
    plan = bb.Plan(torch.from_numpy(pts).to(dev), 3, 4, 2, ell=0.3, domain=UNIT, max_nrhs=4)
    omega = torch.randn(4, 1000, device=dev)
    with pytest.raises(bb.BBFMMError):
        bb.bbfmm_rand_eig(plan.handle, omega, 5)            # k > m
    with pytest.raises(bb.BBFMMError):
        bb.bbfmm_rand_eig(plan.handle, torch.randn(6, 1000, device=dev), 2)   # m > max_nrhs
    with pytest.raises(bb.BBFMMError):
        bb.bbfmm_rand_eig(plan.handle, omega.cpu(), 2)      # host test block
    plan.close()
