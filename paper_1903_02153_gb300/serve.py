"""Continuous-batching request loop for black-box FMM matvecs.

Requests (point set, kernel, p, depth, weights with nrhs columns) arrive at
any time.  A scheduler thread

* admits work by device memory: a request runs once its plan (tree +
  operators + coefficient grids, built by ``bbfmm_plan``) is resident; plans
  stay resident between requests and idle ones are evicted least-recently
  used when a new plan would not fit the budget;
* builds plans off the scheduling thread: a missing plan's estimated bytes
  are reserved and a builder thread makes it, while requests of resident
  plans keep being dispatched; a failed build fails only that plan's
  requests;
* batches as it goes: queued requests that share a plan are merged into one
  multi-right-hand-side matvec (Sec. 2.5 "Multiple right-hand-sides"), up to
  ``max_batch_nrhs`` columns;
* keeps ``slots`` matvecs in flight at once, each on its own CUDA stream, so
  work of different plans overlaps on the device; requests that arrive while
  others run are admitted as soon as a slot and the memory are free.

Latency is measured from submit() to the host seeing the batch's completion;
``stats()`` reports p50 / p99 and throughput (sum of N^2 * nrhs per second).

The GPU work is the library's (``bbfmm_plan`` / ``bbfmm_matvec`` through the
ctypes binding); the executor interface exists so that the scheduling logic
and its failure handling can be exercised on the CPU with a fake executor.
"""
from __future__ import annotations

import collections
import queue
import threading
import time

import numpy as np


class Request:
    """One matvec request.  ``key`` identifies the plan (same point set,
    kernel, length scale, p, depth => same plan); ``sigma`` is n x nrhs."""

    _next = 0

    def __init__(self, key, sigma, n=None, meta=None):
        sigma = np.asarray(sigma, dtype=np.float32)
        if sigma.ndim == 1:
            sigma = sigma[:, None]
        if sigma.shape[1] < 1 or sigma.shape[0] < 1:
            raise ValueError("a request needs at least one point and one right-hand side")
        self.key = key
        self.sigma = np.asfortranarray(sigma)
        self.n = sigma.shape[0] if n is None else n
        self.nrhs = sigma.shape[1]
        self.meta = meta or {}
        self.id = Request._next
        Request._next += 1
        self.t_submit = None
        self.t_done = None
        self.result = None
        self.error = None
        self.cancelled = False
        self.batch_size = 0
        self._done = threading.Event()

    def wait(self, timeout=None):
        if not self._done.wait(timeout):
            raise TimeoutError("request %d not done" % self.id)
        if self.error is not None:
            raise RuntimeError("request %d failed: %s" % (self.id, self.error))
        return self.result

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_submit


class _Plan:
    """A plan slot: reserved (estimated bytes, being built), then resident
    (handle set, actual bytes), or failed (error set)."""

    def __init__(self, key, nbytes):
        self.key = key
        self.handle = None
        self.bytes = nbytes
        self.ready = False
        self.error = None
        self.busy = False
        self.last_used = time.perf_counter()


class Server:
    def __init__(self, executor, device_budget_bytes, slots=4, max_batch_nrhs=32, batching=True):
        self.ex = executor
        self.budget = int(device_budget_bytes)
        self.nslots = int(slots)
        self.max_batch = int(max_batch_nrhs)
        self.batching = batching
        self.pending = collections.deque()
        self.plans = collections.OrderedDict()
        self.slots = [None] * self.nslots   # (token, plan, [requests], col offsets)
        self.done = []
        self.lock = threading.Lock()
        self.wake = threading.Event()
        self.running = False
        self.thread = None
        self.t_first = None
        self.t_last = None
        self.evictions = 0
        self.builds = 0
        self.build_q = queue.Queue()
        self.builder = None

    # -- public --------------------------------------------------------------
    def start(self):
        self.running = True
        self.thread = threading.Thread(target=self._loop, name="bbfmm-serve", daemon=True)
        self.builder = threading.Thread(target=self._build_loop, name="bbfmm-plan-builder", daemon=True)
        self.builder.start()
        self.thread.start()
        return self

    def stop(self):
        self.running = False
        self.wake.set()
        if self.thread is not None:
            self.thread.join()
        if self.builder is not None:
            self.build_q.put(None)
            self.builder.join()
        for p in list(self.plans.values()):
            if p.handle is not None:
                self.ex.destroy(p.handle)
        self.plans.clear()

    def submit(self, req):
        if req.nrhs > self.max_batch:
            raise ValueError("request nrhs %d exceeds max_batch_nrhs %d" % (req.nrhs, self.max_batch))
        req.t_submit = time.perf_counter()
        with self.lock:
            if self.t_first is None:
                self.t_first = req.t_submit
            self.pending.append(req)
        self.wake.set()
        return req

    def cancel(self, req):
        with self.lock:
            if req in self.pending:
                self.pending.remove(req)
                req.cancelled = True
                req.error = "cancelled"
                req.t_done = time.perf_counter()
                req._done.set()
                return True
        return False

    def stats(self):
        lat = np.array([r.latency for r in self.done if r.error is None])
        work = sum(float(r.n) ** 2 * r.nrhs for r in self.done if r.error is None)
        wall = (self.t_last - self.t_first) if self.t_last and self.t_first else float("nan")
        out = {"requests": len(self.done), "failed": sum(r.error is not None for r in self.done),
               "plans_resident": sum(p.ready for p in list(self.plans.values())),
               "plan_builds": self.builds, "plan_evictions": self.evictions,
               "mean_batch": float(np.mean([r.batch_size for r in self.done])) if self.done else 0.0}
        if lat.size:
            out.update({"p50_ms": 1e3 * float(np.percentile(lat, 50)),
                        "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                        "mean_ms": 1e3 * float(lat.mean()),
                        "throughput_N2_per_s": work / wall if wall > 0 else float("nan"),
                        "requests_per_s": len(lat) / wall if wall > 0 else float("nan")})
        return out

    # -- scheduler -----------------------------------------------------------
    def _used_bytes(self):
        return sum(p.bytes for p in self.plans.values())

    def _ensure_plan(self, key):
        """The resident plan for key, or None when it is not resident yet: a
        missing plan is reserved (idle resident plans are evicted, least
        recently used first, until its estimate fits the budget) and queued
        for the builder thread.  Raises MemoryError when it can never fit."""
        p = self.plans.get(key)
        if p is not None:
            if not p.ready:
                return None          # being built
            self.plans.move_to_end(key)
            return p
        need = self.ex.estimate_bytes(key, self.max_batch)
        if need > self.budget:
            raise MemoryError("plan needs %d bytes, budget %d" % (need, self.budget))
        while self._used_bytes() + need > self.budget:
            idle = [k for k, q in self.plans.items() if q.ready and not q.busy]
            if not idle:
                return None          # wait for a running batch or a build to finish
            victim = self.plans.pop(idle[0])
            self.ex.destroy(victim.handle)
            self.evictions += 1
        p = _Plan(key, need)
        self.plans[key] = p
        self.builds += 1
        self.build_q.put(p)
        return None

    def _build_loop(self):
        """Builder thread: makes the reserved plans one at a time (a build
        allocates its device memory and runs its own stream), then wakes the
        scheduler."""
        while True:
            p = self.build_q.get()
            if p is None:
                return
            try:
                handle = self.ex.build(p.key, self.max_batch)
                nbytes = self.ex.plan_bytes(handle)
                with self.lock:
                    p.handle, p.bytes, p.ready = handle, nbytes, True
            except Exception as e:                       # noqa: BLE001
                with self.lock:
                    p.error = repr(e)
            self.wake.set()

    def _reap_failed_builds(self):
        for key, p in list(self.plans.items()):
            if p.error is None:
                continue
            del self.plans[key]
            with self.lock:
                failed = [r for r in self.pending if r.key == key]
                for r in failed:
                    self.pending.remove(r)
            self._finish(failed, error=p.error)

    def _finish(self, reqs, results=None, error=None):
        now = time.perf_counter()
        for i, r in enumerate(reqs):
            r.t_done = now
            if error is not None:
                r.error = error
            else:
                r.result = results[i]
            r._done.set()
            self.done.append(r)
        self.t_last = now

    def _poll_slots(self):
        for s, job in enumerate(self.slots):
            if job is None:
                continue
            token, plan, reqs, offs = job
            if not self.ex.ready(token):
                continue
            try:
                out = self.ex.result(token)
                res = [np.array(out[:, offs[i]:offs[i] + r.nrhs]) for i, r in enumerate(reqs)]
                self._finish(reqs, res)
            except Exception as e:                       # noqa: BLE001
                self._finish(reqs, error=repr(e))
            plan.busy = False
            plan.last_used = time.perf_counter()
            self.slots[s] = None

    def _next_batch(self):
        """Oldest pending request whose plan is resident and free, plus the
        pending requests of the same plan that fit in the batch.  Requests
        whose plan is missing get it reserved and queued for building."""
        with self.lock:
            queue_ = list(self.pending)
        seen = set()
        for head in queue_:
            if head.key in seen:
                continue
            seen.add(head.key)
            p = self.plans.get(head.key)
            if p is not None and p.busy:
                continue
            try:
                p = self._ensure_plan(head.key)
            except Exception as e:                       # noqa: BLE001
                with self.lock:
                    failed = [r for r in self.pending if r.key == head.key]
                    for r in failed:
                        self.pending.remove(r)
                self._finish(failed, error=repr(e))
                continue
            if p is None:
                continue
            batch, cols = [], 0
            with self.lock:
                for r in list(self.pending):
                    if r.key != head.key:
                        continue
                    if cols + r.nrhs > self.max_batch or (batch and not self.batching):
                        break
                    batch.append(r)
                    cols += r.nrhs
                for r in batch:
                    self.pending.remove(r)
            return p, batch
        return None

    def _loop(self):
        while self.running:
            self._poll_slots()
            self._reap_failed_builds()
            launched = False
            for s in range(self.nslots):
                if self.slots[s] is not None:
                    continue
                nb = self._next_batch()
                if nb is None:
                    break
                plan, batch = nb
                if not batch:
                    continue
                offs, c = [], 0
                for r in batch:
                    offs.append(c)
                    c += r.nrhs
                sigma = np.concatenate([r.sigma for r in batch], axis=1) if len(batch) > 1 else batch[0].sigma
                for r in batch:
                    r.batch_size = len(batch)
                plan.busy = True
                try:
                    token = self.ex.launch(plan.handle, np.asfortranarray(sigma), s)
                except Exception as e:                   # noqa: BLE001
                    plan.busy = False
                    self._finish(batch, error=repr(e))
                    continue
                self.slots[s] = (token, plan, batch, offs)
                launched = True
            busy = any(j is not None for j in self.slots)
            with self.lock:
                idle = not self.pending
            if not launched:
                if busy:
                    time.sleep(20e-6)
                else:               # nothing queued, or waiting for a plan build
                    self.wake.wait(0.01 if idle else 0.001)
                    self.wake.clear()


# ---------------------------------------------------------------------------
class GpuExecutor:
    """Runs batches through the C ABI: one CUDA stream per slot; sigma goes in
    through pinned host memory and phi comes back the same way, so a batch's
    latency includes its transfers."""

    def __init__(self, point_source, precision="fp16x3", svd_eps=1e-6, slots=4, device=0, domain=None):
        import torch
        from . import bbfmm
        self.torch = torch
        self.bb = bbfmm
        self.point_source = point_source     # key -> (points, kernel, ell, p, depth)
        self.precision = precision
        self.svd_eps = svd_eps
        self.domain = domain                 # (lo, side) shared by all plans, or None: bounding cubes
        self.dev = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(slots)]
        self.build_stream = torch.cuda.Stream(device=self.dev)

    def estimate_bytes(self, key, max_nrhs):
        pts, kid, ell, p, depth = self.point_source(key)
        n, p3 = pts.shape[0], p ** 3
        grid = sum(8 ** l for l in range(2, depth + 1)) * max_nrhs * p3 * 4 * 6
        return int(grid + n * (16 + 4 + 12 * max_nrhs) * 2 + 64 * 2 ** 20)

    def build(self, key, max_nrhs):
        """Runs on the server's builder thread, on a stream of its own so that
        the build overlaps the matvecs in flight.  The plan's launch choices
        are measured here, for every power-of-two batch width up to
        max_nrhs (a batch of any width takes its bucket's choice), so that no
        request pays for a tuning sweep."""
        self.torch.cuda.set_device(self.dev)
        pts, kid, ell, p, depth = self.point_source(key)
        plan = self.bb.Plan(pts, kid, p, depth, ell=ell, precision=self.precision, svd_eps=self.svd_eps,
                            max_nrhs=max_nrhs, domain=self.domain, stream=self.build_stream)
        b = 1
        while b <= max_nrhs:
            self.bb.bbfmm_autotune(plan.handle, b, self.build_stream)
            b *= 2
        return plan

    def plan_bytes(self, plan):
        return int(plan.info().device_bytes)

    def destroy(self, plan):
        plan.close()

    def launch(self, plan, sigma, slot):
        torch = self.torch
        stream = self.streams[slot]
        nrhs = sigma.shape[1]
        host_in = torch.from_numpy(np.ascontiguousarray(sigma.T)).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        with torch.cuda.stream(stream):
            d_in = host_in.to(self.dev, non_blocking=True)
            d_out = torch.empty_like(d_in)
            self.bb.bbfmm_matvec(plan.handle, d_in, d_out, nrhs, stream)
            host_out.copy_(d_out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return (ev, host_out, d_in, d_out, host_in)

    def ready(self, token):
        return token[0].query()

    def result(self, token):
        token[0].synchronize()
        return token[1].numpy().T


class FakeExecutor:
    """CPU stand-in for tests of the scheduler: a 'matvec' multiplies sigma by
    a per-key factor after a fixed delay; build failures are injected by key."""

    def __init__(self, sizes, delay=0.002, fail_build=(), fail_launch=(), build_delay=None):
        self.sizes = dict(sizes)             # key -> plan bytes
        self.delay = delay
        self.build_delay = dict(build_delay or {})   # key -> seconds a build takes
        self.fail_build = set(fail_build)
        self.fail_launch = set(fail_launch)
        self.live = set()
        self.log = []

    def estimate_bytes(self, key, max_nrhs):
        return self.sizes[key]

    def build(self, key, max_nrhs):
        time.sleep(self.build_delay.get(key, 0.0))
        if key in self.fail_build:
            raise MemoryError("injected: plan allocation refused for %r" % (key,))
        self.live.add(key)
        self.log.append(("build", key))
        return key

    def plan_bytes(self, handle):
        return self.sizes[handle]

    def destroy(self, handle):
        self.live.discard(handle)
        self.log.append(("destroy", handle))

    def launch(self, handle, sigma, slot):
        if handle in self.fail_launch:
            raise RuntimeError("injected: launch failed for %r" % (handle,))
        self.log.append(("launch", handle, sigma.shape[1], slot))
        factor = 1.0 + (hash(handle) % 7)
        return (time.perf_counter() + self.delay, sigma * factor)

    def ready(self, token):
        return time.perf_counter() >= token[0]

    def result(self, token):
        return token[1]
