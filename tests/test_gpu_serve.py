"""The request loop on the GPU: every request's result is the same when it
runs alone (one slot, no batching) and when it runs in the mix (several slots
in flight, requests of one plan merged into a multi-RHS matvec), within the
FP32 tolerance of the path, and one of them is checked against the oracle."""
import numpy as np
import pytest

from paper_1903_02153_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02153_gb300 import build
    build.build()
    from paper_1903_02153_gb300 import serve
    return serve


POINTS = {}


def point_source(key):
    kind, n, seed, kid, ell, p, depth = key
    if (kind, n, seed) not in POINTS:
        POINTS[(kind, n, seed)] = W.make_points(kind, n, seed)
    return POINTS[(kind, n, seed)], kid, ell, p, depth


def requests(serve):
    keys = [("uniform", 20000, 1, 1, 1.0, 4, 3), ("clustered", 30000, 2, 3, 0.3, 5, 3),
            ("uniform", 40000, 3, 2, 1.0, 5, 4), ("clustered", 25000, 4, 4, 0.2, 4, 3)]
    rng = np.random.default_rng(5)
    out = []
    for i in range(14):
        key = keys[i % len(keys)]
        nrhs = [1, 3, 2, 1][i % 4]
        sig = rng.uniform(-1, 1, (key[1], nrhs)).astype(np.float32)
        out.append((key, sig))
    return out


@pytest.mark.parametrize("precision", ["fp16x3", "fp32"])
def test_result_alone_equals_result_in_the_mix(serve_mod, oracle, precision):
    S = serve_mod
    reqs = requests(S)
    ex1 = S.GpuExecutor(point_source, precision=precision, slots=1)
    alone_srv = S.Server(ex1, device_budget_bytes=8 << 30, slots=1, max_batch_nrhs=8, batching=False).start()
    alone = []
    for key, sig in reqs:
        alone.append(alone_srv.submit(S.Request(key, sig)).wait(120))
    alone_srv.stop()

    ex2 = S.GpuExecutor(point_source, precision=precision, slots=3)
    mix_srv = S.Server(ex2, device_budget_bytes=8 << 30, slots=3, max_batch_nrhs=8, batching=True).start()
    handles = [mix_srv.submit(S.Request(key, sig)) for key, sig in reqs]
    mixed = [h.wait(120) for h in handles]
    st = mix_srv.stats()
    mix_srv.stop()
    assert st["failed"] == 0 and st["mean_batch"] > 1
    for a, b in zip(alone, mixed):
        assert np.linalg.norm(a - b) <= 2e-6 * np.linalg.norm(a)
    key, sig = reqs[1]
    pts, kid, ell, p, depth = point_source(key)
    lo, side = oracle.bounding_cube(pts)
    ref = oracle.bbfmm(pts, sig.astype(np.float64), kid, p, depth, ell=ell, lo=lo, side=side)
    assert oracle.rel_err(mixed[1], ref) <= 1e-5
