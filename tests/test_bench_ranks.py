"""The several-GPU path of bench.py (one process per GPU, independent replicas:
the matvec does not shard across GPUs here) reduces only its timings: the
slowest rank's time, and the units of all ranks over it.  Checked with two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.slowest_rank([3.0, 5.0][rank], dist, torch.device("cpu"))
        e2e = bench.slowest_rank([0.007, 0.004][rank], dist, torch.device("cpu"))
        dist.barrier()
        q.put((rank, ms, e2e, bench.job_rate(world, 1e12, ms / 1e3)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_job_rate_over_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, rate in got:
        assert ms == 5.0 and e2e == 0.007         # every rank sees the slowest rank's times
        assert rate == pytest.approx(2 * 1e12 / 5e-3)


def test_without_a_group_the_local_values_stand():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank(2.5, None, None) == 2.5
    assert bench.job_rate(1, 10.0, 2.0) == 5.0
