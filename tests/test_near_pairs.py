"""The visiting rule of the symmetric near field (BBFMM_NEAR_SYMMETRIC, Sec. 2.5
symmetry of K), restated on the host and checked by brute force on small
trees: every ordered pair (target leaf, source leaf) of neighbours, the leaf
with itself included (Def. 2.1), is computed exactly once -- either as rows
of the target leaf's own work item, or as the column sums (slot) written by
the source leaf's work item -- and no (slot, point) has two writers.

The rule (the work item of leaf alpha; nid = 3x3x3 offset number, 13 = own):
  own leaf             one way (rows of alpha)
  nid > 13 (forward)   both ways if alpha holds <= 64 points, else one way
  nid < 13 (backward)  one way if that neighbour holds > 64 points, else skipped
A leaf of more than 128 points is several work items; only leaves of <= 64
take pairs both ways, so a slot is always written by a single work item."""
import itertools

import numpy as np
import pytest

SYM_MAX = 64


def nid_of(d):
    return (d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1)


def visits(counts):
    """Per (alpha, beta) neighbour pair: the list of ('rows', target, source)
    and ('slot', target, source) contributions the rule computes."""
    side = counts.shape[0]
    done = {}
    writers = {}
    for a in itertools.product(range(side), repeat=3):
        if counts[a] == 0:
            continue
        for d in itertools.product((-1, 0, 1), repeat=3):
            b = tuple(a[i] + d[i] for i in range(3))
            if min(b) < 0 or max(b) >= side or counts[b] == 0:
                continue
            nid = nid_of(d)
            if nid == 13:
                done.setdefault((a, b), []).append("rows")
            elif nid > 13:
                done.setdefault((a, b), []).append("rows")
                if counts[a] <= SYM_MAX:
                    done.setdefault((b, a), []).append("slot")
                    key = (b, 26 - nid)   # the slot of beta's points that alpha writes
                    writers[key] = writers.get(key, 0) + (1 if counts[a] <= 128 else 2)
            else:
                if counts[b] > SYM_MAX:
                    done.setdefault((a, b), []).append("rows")
    return done, writers


@pytest.mark.parametrize("seed,side", [(1, 2), (2, 3), (3, 4), (4, 4), (5, 5)])
def test_every_neighbour_pair_is_computed_once(seed, side):
    rng = np.random.default_rng(seed)
    # empty, small, two-way-sized, one-way-sized and split (> 128) leaves
    counts = rng.choice([0, 1, 5, 32, 64, 65, 100, 128, 129, 300], size=(side,) * 3)
    done, writers = visits(counts)
    for a in itertools.product(range(side), repeat=3):
        for d in itertools.product((-1, 0, 1), repeat=3):
            b = tuple(a[i] + d[i] for i in range(3))
            if min(b) < 0 or max(b) >= side:
                continue
            want = 1 if counts[a] > 0 and counts[b] > 0 else 0
            assert len(done.get((a, b), [])) == want, (a, b, counts[a], counts[b], done.get((a, b)))
    assert all(w == 1 for w in writers.values())


def test_slot_numbers_pair_up():
    """The slot alpha writes for beta = alpha + d is 26 - nid(d) = nid(-d):
    the number under which beta sees alpha, one of the 13 backward ones."""
    for d in itertools.product((-1, 0, 1), repeat=3):
        n = nid_of(d)
        if n > 13:
            assert 26 - n == nid_of(tuple(-x for x in d)) and 0 <= 26 - n < 13
