"""The continuous-batching request loop, on the CPU with a fake executor:
batching of requests that share a plan, admission by a device-memory budget
with LRU eviction of idle plans, concurrent slots, and failures injected on
the host (refused plan allocation, failing launch, cancelled and malformed
requests).  No GPU is involved."""
import numpy as np
import pytest

from paper_1903_02153_gb300.serve import FakeExecutor, Request, Server


def factor(key):
    return 1.0 + (hash(key) % 7)


def make(key, n=10, nrhs=1, seed=0):
    return Request(key, np.random.default_rng(seed).standard_normal((n, nrhs)).astype(np.float32))


def test_results_and_batching_of_requests_sharing_a_plan():
    ex = FakeExecutor({"a": 10, "b": 10}, delay=0.01)
    srv = Server(ex, device_budget_bytes=100, slots=1, max_batch_nrhs=8)
    reqs = [make("a" if i % 2 == 0 else "b", nrhs=1 + i % 3, seed=i) for i in range(12)]
    for r in reqs:
        srv.submit(r)
    srv.start()
    for r in reqs:
        np.testing.assert_allclose(r.wait(5), r.sigma * factor(r.key), rtol=1e-6)
    srv.stop()
    launches = [e for e in ex.log if e[0] == "launch"]
    assert len(launches) < len(reqs)                       # requests were merged
    assert max(e[2] for e in launches) <= 8                  # within the batch limit
    st = srv.stats()
    assert st["requests"] == 12 and st["failed"] == 0 and st["mean_batch"] > 1
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_no_batching_runs_one_request_per_launch():
    ex = FakeExecutor({"a": 10}, delay=0.001)
    srv = Server(ex, 100, slots=2, max_batch_nrhs=8, batching=False)
    reqs = [make("a", seed=i) for i in range(5)]
    for r in reqs:
        srv.submit(r)
    srv.start()
    for r in reqs:
        r.wait(5)
    srv.stop()
    assert len([e for e in ex.log if e[0] == "launch"]) == 5


def test_memory_admission_and_lru_eviction():
    ex = FakeExecutor({"a": 40, "b": 40, "c": 40}, delay=0.002)
    srv = Server(ex, device_budget_bytes=100, slots=1, max_batch_nrhs=4).start()
    for key in ["a", "b", "c", "a", "c", "b"]:
        srv.submit(make(key)).wait(5)
    srv.stop()
    assert srv.evictions >= 2
    live_max = 0
    live = set()
    for e in ex.log:               # never more than 2 plans of 40 bytes resident
        if e[0] == "build":
            live.add(e[1])
        elif e[0] == "destroy":
            live.discard(e[1])
        live_max = max(live_max, len(live))
    assert live_max <= 2


def test_plan_larger_than_budget_fails_only_its_requests():
    ex = FakeExecutor({"big": 1000, "ok": 10})
    srv = Server(ex, 100, slots=2).start()
    big, ok = srv.submit(make("big")), srv.submit(make("ok"))
    with pytest.raises(RuntimeError, match="MemoryError"):
        big.wait(5)
    ok.wait(5)
    srv.stop()


def test_injected_build_and_launch_failures():
    ex = FakeExecutor({"a": 10, "bad": 10, "flaky": 10}, fail_build={"bad"}, fail_launch={"flaky"})
    srv = Server(ex, 100, slots=2).start()
    rs = [srv.submit(make(k, seed=i)) for i, k in enumerate(["a", "bad", "flaky", "a"])]
    rs[0].wait(5)
    rs[3].wait(5)
    with pytest.raises(RuntimeError, match="allocation refused"):
        rs[1].wait(5)
    with pytest.raises(RuntimeError, match="launch failed"):
        rs[2].wait(5)
    # the server keeps serving after the failures
    srv.submit(make("a", seed=9)).wait(5)
    assert srv.stats()["failed"] == 2
    srv.stop()


def test_cancel_before_dispatch_and_malformed_requests():
    ex = FakeExecutor({"a": 10})
    srv = Server(ex, 100, slots=1, max_batch_nrhs=4)
    r = srv.submit(make("a"))
    assert srv.cancel(r)
    with pytest.raises(RuntimeError, match="cancelled"):
        r.wait(1)
    with pytest.raises(ValueError):
        srv.submit(make("a", nrhs=5))                    # wider than a batch
    with pytest.raises(ValueError):
        Request("a", np.zeros((0, 1), dtype=np.float32))  # no points
    srv.start()
    srv.submit(make("a")).wait(5)
    srv.stop()


def test_slots_run_different_plans_concurrently():
    ex = FakeExecutor({"a": 10, "b": 10, "c": 10}, delay=0.05)
    srv = Server(ex, 100, slots=3, max_batch_nrhs=1)
    rs = [srv.submit(make(k, seed=i)) for i, k in enumerate("abc")]
    srv.start()
    for r in rs:
        r.wait(5)
    srv.stop()
    slots = {e[3] for e in ex.log if e[0] == "launch"}
    assert slots == {0, 1, 2}
    # all three were in flight together: total time well under 3 delays
    assert max(r.t_done for r in rs) - min(r.t_submit for r in rs) < 0.14


def test_slow_plan_build_does_not_block_resident_plans():
    ex = FakeExecutor({"a": 10, "slow": 10}, delay=0.002, build_delay={"slow": 0.5})
    srv = Server(ex, 100, slots=2, max_batch_nrhs=1).start()
    srv.submit(make("a")).wait(5)                         # "a" is resident
    slow = srv.submit(make("slow", seed=1))
    t0 = slow.t_submit
    fast = [srv.submit(make("a", seed=2 + i)) for i in range(5)]
    for r in fast:
        r.wait(5)
    # the requests of the resident plan finished while "slow" was being built
    assert max(r.t_done for r in fast) - t0 < 0.25
    assert not slow._done.is_set()
    np.testing.assert_allclose(slow.wait(5), slow.sigma * factor("slow"), rtol=1e-6)
    assert slow.t_done - t0 >= 0.5
    srv.stop()


def test_building_plans_count_against_the_budget():
    # two plans of 60 bytes in a 100-byte budget: the second waits for the
    # first to be resident and idle, then evicts it; never both at once
    ex = FakeExecutor({"a": 60, "b": 60}, delay=0.01, build_delay={"a": 0.1, "b": 0.1})
    srv = Server(ex, 100, slots=2, max_batch_nrhs=1).start()
    ra, rb = srv.submit(make("a")), srv.submit(make("b", seed=1))
    ra.wait(5)
    rb.wait(5)
    srv.stop()
    live, live_max = set(), 0
    for e in ex.log:
        if e[0] == "build":
            live.add(e[1])
        elif e[0] == "destroy":
            live.discard(e[1])
        live_max = max(live_max, len(live))
    assert live_max == 1 and srv.evictions == 1
