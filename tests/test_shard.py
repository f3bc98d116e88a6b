"""The LPT partitioner of xt_shard_lpt (host code, no GPU): each pair goes to
exactly one part, part totals are the pairs' in-band cell estimates counted
row by row, the split is deterministic, and its largest part is within the
LPT bound of the best split found by brute force on small cases."""
import itertools
import random

import numpy as np
import pytest

import paper_2301_09310_gb300 as xt
from paper_2301_09310_gb300 import build as xbuild


@pytest.fixture(scope="module", autouse=True)
def lib():
    xbuild.build()
    return xt.load_library()


def band_cells(ql, tl, w):
    """In-band cells of a whole pair with no z-drop, row by row."""
    return sum(max(0, min(ql, i + w + 1) - max(0, i - w)) for i in range(tl))


def test_every_pair_once_and_totals():
    rng = random.Random(31)
    for _ in range(40):
        n = rng.randint(0, 300)
        parts = rng.randint(1, 7)
        w = rng.choice([0, 1, 5, 100, 10**6])
        ql = np.array([rng.choice([0, 1, rng.randint(1, 60), rng.randint(100, 400)])
                       for _ in range(n)], np.int32)
        tl = np.array([max(0, q + rng.randint(-3, 40)) for q in ql], np.int32)
        shard, cells = xt.xt_shard_lpt(ql, tl, w, parts)
        assert shard.shape == (n,) and np.all((shard >= 0) & (shard < parts))
        est = np.array([band_cells(int(a), int(b), w) for a, b in zip(ql, tl)], np.int64)
        for p in range(parts):
            assert cells[p] == est[shard == p].sum()
        if n:
            # greedy assignment bound: no part exceeds the mean by more than a pair
            assert cells.max() <= est.sum() / parts + est.max()
        # the same call gives the same split
        again, _ = xt.xt_shard_lpt(ql, tl, w, parts)
        assert np.array_equal(shard, again)


def test_within_lpt_bound_of_optimum():
    rng = random.Random(32)
    for _ in range(60):
        n = rng.randint(2, 8)
        m = rng.choice([2, 3])
        ql = np.array([rng.randint(1, 40) for _ in range(n)], np.int32)
        tl = ql + np.int32(5)
        w = 100
        est = [band_cells(int(a), int(b), w) for a, b in zip(ql, tl)]
        best = min(max(sum(e for e, p in zip(est, assign) if p == k) for k in range(m))
                   for assign in itertools.product(range(m), repeat=n))
        _, cells = xt.xt_shard_lpt(ql, tl, w, m)
        assert cells.max() * 3 * m <= (4 * m - 1) * best


def test_ties_and_order():
    # equal estimates go out by pair index, to the lowest part first
    shard, cells = xt.xt_shard_lpt(np.full(6, 10, np.int32), np.full(6, 10, np.int32), 100, 3)
    assert shard.tolist() == [0, 1, 2, 0, 1, 2] and cells.tolist() == [200, 200, 200]
    # the largest pair first, then each to the least-loaded part
    shard, cells = xt.xt_shard_lpt(np.array([10, 20, 30, 40], np.int32),
                                   np.array([15, 25, 35, 45], np.int32), 100, 2)
    assert shard.tolist() == [1, 1, 1, 0] and cells.tolist() == [1800, 1700]


def test_rejects_bad_arguments():
    with pytest.raises(xt.XtError):
        xt.xt_shard_lpt(np.zeros(3, np.int32), np.zeros(3, np.int32), 100, 0)
    with pytest.raises(xt.XtError):
        xt.xt_shard_lpt(np.zeros(3, np.int32), np.zeros(3, np.int32), -1, 2)
