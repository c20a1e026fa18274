"""GPU test of bbfmm_sort_points_static, the entry point that allocates
nothing.

Some callers cannot call cudaMalloc when they build a tree (their device
memory is a budget another runtime reserved, or an allocation there would
stall other GPU work).  They hand the library the points and the output
buffers, and the sort keeps its temporaries in the library's fixed scratch
array.  The result must equal the tree build of the existing entry point
bbfmm_plan (read back through bbfmm_get_leaf_cells) exactly -- this is
integer index work -- on two calls in a row, the second of which reuses the
scratch the first one left behind."""
import numpy as np
import pytest

from paper_1903_02153_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def demorton(m, depth):
    x = np.zeros_like(m)
    y = np.zeros_like(m)
    z = np.zeros_like(m)
    for b in range(depth):
        x |= ((m >> (3 * b)) & 1) << b
        y |= ((m >> (3 * b + 1)) & 1) << b
        z |= ((m >> (3 * b + 2)) & 1) << b
    return np.stack([x, y, z], axis=1)


def cells_from_sort(perm, leaf_off, depth, n):
    counts = np.diff(leaf_off)
    leaf_of_sorted = np.repeat(np.arange(8 ** depth, dtype=np.int64), counts)
    cells = np.zeros((n, 3), dtype=np.int64)
    cells[perm] = demorton(leaf_of_sorted, depth)
    return cells


@pytest.fixture(scope="module")
def bb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02153_gb300 import build
    build.build()
    from paper_1903_02153_gb300 import bbfmm
    bbfmm.lib()
    return bbfmm


def test_static_sort_matches_plan_tree_build(bb):
    dev = torch.device("cuda:0")
    cases = [("clustered", 300_000, 6), ("uniform", 1 << 20, 5)]   # the second call uses the maximum n
    for kind, n, depth in cases:
        pts = W.make_points(kind, n, seed=81)
        d_pts = torch.from_numpy(pts).to(dev)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        off = torch.empty(8 ** depth + 1, dtype=torch.int32, device=dev)
        bb.bbfmm_sort_points_static(d_pts, depth, W.UNIT_LO, W.UNIT_SIDE, perm, off)
        p = perm.cpu().numpy().astype(np.int64)
        o = off.cpu().numpy().astype(np.int64)
        # a permutation, increasing inside every leaf, offsets covering all points
        assert o[0] == 0 and o[-1] == n and np.all(np.diff(o) >= 0)
        assert np.array_equal(np.sort(p), np.arange(n))
        inside = np.ones(n - 1, dtype=bool)
        inside[o[1:-1][(o[1:-1] > 0) & (o[1:-1] < n)] - 1] = False
        assert np.all(np.diff(p)[inside] > 0)
        # the same leaves as the tree build of bbfmm_plan
        plan = bb.Plan(d_pts, bb.BBFMM_K_INV_R, 4, depth, domain=(W.UNIT_LO, W.UNIT_SIDE))
        ref = bb.bbfmm_get_leaf_cells(plan.handle, n).astype(np.int64)
        plan.close()
        np.testing.assert_array_equal(cells_from_sort(p, o, depth, n), ref)


def test_static_sort_rejects_oversize_and_host_buffers(bb):
    dev = torch.device("cuda:0")
    n = (1 << 20) + 1
    d_pts = torch.rand(n, 3, dtype=torch.float64, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    off = torch.empty(8 ** 3 + 1, dtype=torch.int32, device=dev)
    with pytest.raises(bb.BBFMMError) as ei:
        bb.bbfmm_sort_points_static(d_pts, 3, W.UNIT_LO, W.UNIT_SIDE, perm, off)
    assert ei.value.status == bb.BBFMM_EINVAL
    host = np.random.default_rng(0).random((1000, 3))
    with pytest.raises(bb.BBFMMError):
        bb.bbfmm_sort_points_static(host, 3, W.UNIT_LO, W.UNIT_SIDE, perm[:1000], off)
