"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws point sets and
weight vectors (numpy PCG64, fixed seeds) so that the CUDA library, the CPU
oracle, the tests and the benchmark all see the same inputs.

Workloads (the paper draws its points uniformly in the unit cube, Sec. 4
"Parameters and notations"; its covariance experiments use exp(-r) with 120
right-hand sides, Sec. 4.3; its unstructured-mesh experiment uses a mesh that
is not available here, so a jittered, thinned lattice stands in for it):

* ``uniform``: N points i.i.d. U[0,1)^3, sigma ~ U(-1,1).
* ``clustered``: 8 centres ~ U[0,1]^3; each point = a uniformly chosen centre
  + N(0, 0.05^2 I), clipped to [0,1]^3; sigma ~ U(-1,1).
* ``jittered_grid``: 80^3 lattice sites (i + 1/2) h, h = 1/80, each moved by
  U(-0.4h, 0.4h)^3, thinned to N sites by dropping a random subset; sigma is
  N x nrhs standard normal (a randomized-PCA sketch block).
* ``serving_stream``: Poisson arrivals of requests with log-uniform N, mixed
  kernels, orders and right-hand-side counts.
"""
from __future__ import annotations

import numpy as np

SEED_POINTS = 1903
SEED_SIGMA = 2153
SEED_STREAM = 7

UNIT_LO = np.zeros(3)
UNIT_SIDE = 1.0


def uniform_points(n, seed=SEED_POINTS):
    return np.random.default_rng(seed).random((n, 3))


def clustered_points(n, seed=SEED_POINTS, nblobs=8, std=0.05):
    rng = np.random.default_rng(seed)
    centres = rng.random((nblobs, 3))
    which = rng.integers(0, nblobs, size=n)
    pts = centres[which] + rng.normal(0.0, std, size=(n, 3))
    return np.clip(pts, 0.0, 1.0)


def jittered_grid_points(n, seed=SEED_POINTS, m=80, jitter=0.4):
    rng = np.random.default_rng(seed)
    h = 1.0 / m
    idx = np.arange(m ** 3)
    ijk = np.stack([idx % m, (idx // m) % m, idx // (m * m)], axis=1).astype(np.float64)
    pts = (ijk + 0.5) * h + rng.uniform(-jitter * h, jitter * h, size=(m ** 3, 3))
    if n < m ** 3:
        keep = np.sort(rng.permutation(m ** 3)[:n])
        pts = pts[keep]
    return pts


def uniform_sigma(n, nrhs=1, seed=SEED_SIGMA):
    s = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, nrhs))
    return s[:, 0] if nrhs == 1 else np.asfortranarray(s)


def normal_sigma(n, nrhs=1, seed=SEED_SIGMA):
    s = np.random.default_rng(seed).standard_normal((n, nrhs))
    return s[:, 0] if nrhs == 1 else np.asfortranarray(s)


# Named configurations: (points, kernel id, kernel length scale, p, depth, nrhs).
# Kernel ids: 1 = 1/r, 2 = 1/r^2, 3 = exp(-r/ell), 4 = exp(-(r/ell)^2).
CONFIGS = {
    "uniform-4k-p4-d3": dict(kind="uniform", n=4096, kernel=1, ell=1.0, p=4, depth=3, nrhs=1),
    "uniform-1M-p5-d6": dict(kind="uniform", n=1 << 20, kernel=1, ell=1.0, p=5, depth=6, nrhs=1),
    "uniform-1M-p5-d5": dict(kind="uniform", n=1 << 20, kernel=1, ell=1.0, p=5, depth=5, nrhs=1),
    "clustered-2M-exp0.3-p6-d6": dict(kind="clustered", n=2_000_000, kernel=3, ell=0.3, p=6,
                                      depth=6, nrhs=1),
    "jittered-500k-exp0.2-p5-d5-rhs64": dict(kind="jittered_grid", n=500_000, kernel=3, ell=0.2,
                                             p=5, depth=5, nrhs=64),
}


def make_points(kind, n, seed=SEED_POINTS):
    if kind == "uniform":
        return uniform_points(n, seed)
    if kind == "clustered":
        return clustered_points(n, seed)
    if kind == "jittered_grid":
        return jittered_grid_points(n, seed)
    raise ValueError(kind)


def make_sigma(kind, n, nrhs, seed=SEED_SIGMA):
    if kind == "jittered_grid":
        return normal_sigma(n, nrhs, seed)
    return uniform_sigma(n, nrhs, seed)


def serving_stream(nreq, seed=SEED_STREAM, n_lo=10_000, n_hi=2_000_000, repeat_prob=0.5, plans=None):
    """Request descriptors for the serving loop: each request has a point-set
    recipe (kind, n, seed), kernel id, p, nrhs, depth.

    With ``plans=None`` a request reuses an earlier request's point set with
    probability ``repeat_prob`` (a plan-cache hit) and otherwise draws a new
    one; kernel and p are drawn per request.  With ``plans=k`` the stream
    draws from a fixed pool of k plan recipes (point set, kernel, p, depth),
    uniformly: the steady state of a service whose plans stay resident.
    nrhs is drawn from {1, 8, 32}.  Inter-arrival gaps are unit-rate
    exponential; callers scale them."""
    rng = np.random.default_rng(seed)
    kernels = [(1, 1.0), (2, 1.0), (3, 1.0), (4, 1.0)]

    def recipe():
        n = int(10 ** rng.uniform(np.log10(n_lo), np.log10(n_hi)))
        kind = "uniform" if rng.random() < 0.5 else "clustered"
        return kind, n, int(rng.integers(0, 2 ** 31))

    def depth_of(n):
        return int(np.clip(round(np.log(n / 32.0) / np.log(8.0)), 2, 7))

    pool = []
    for _ in range(plans or 0):
        kind, n, pseed = recipe()
        kid, ell = kernels[int(rng.integers(0, 4))]
        pool.append((kind, n, pseed, kid, ell, int(rng.choice([4, 5, 6])), depth_of(n)))
    reqs = []
    for i in range(nreq):
        if pool:
            kind, n, pseed, kid, ell, p, depth = pool[int(rng.integers(0, len(pool)))]
        else:
            if reqs and rng.random() < repeat_prob:
                base = reqs[int(rng.integers(0, len(reqs)))]
                kind, n, pseed = base["kind"], base["n"], base["point_seed"]
            else:
                kind, n, pseed = recipe()
            kid, ell = kernels[int(rng.integers(0, 4))]
            p = int(rng.choice([4, 5, 6]))
            depth = depth_of(n)
        nrhs = int(rng.choice([1, 8, 32]))
        reqs.append(dict(id=i, kind=kind, n=n, point_seed=pseed, sigma_seed=int(rng.integers(0, 2 ** 31)),
                         kernel=kid, ell=ell, p=p, nrhs=nrhs, depth=depth,
                         gap=float(rng.exponential(1.0))))
    return reqs
