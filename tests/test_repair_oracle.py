"""Pins of the monotone relaxation and its repair (Section 2.4.3) in the
oracle, against brute force and invariants.  No GPU needed."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_27117_b300 import workloads as W


@pytest.mark.parametrize("idx", range(3))
def test_relaxation_keeps_the_optimum(idx):
    """With nonnegative costs the relaxed problem (customer rows >= 1) has
    the optimum of the original one (brute force over 12 binaries)."""
    orig = W.facility_location(nf=3, nc=3, idx=idx)
    rel = W.facility_location(nf=3, nc=3, idx=idx, relaxed=True)
    f1, b1, _, n1 = O.Evaluator(orig).brute_force()
    f2, b2, _, n2 = O.Evaluator(rel).brute_force()
    assert f1 and f2 and b1 == b2
    assert n2 > n1                       # supersets are feasible for the relaxation


@pytest.mark.parametrize("idx", range(3))
def test_repair_maps_relaxed_points_to_original_ones(idx):
    """Every point feasible for the relaxation, after the repair and the
    closure, is feasible for the original problem and costs no more."""
    orig = W.facility_location(nf=3, nc=3, idx=idx)
    rel = W.facility_location(nf=3, nc=3, idx=idx, relaxed=True)
    X = np.array(list(itertools.product([0, 1], repeat=rel.n)), np.uint8)
    v, o = O.Evaluator(rel)(X)
    Xf = X[v == 0].copy()
    of = o[v == 0]
    O.repair_min(Xf, rel.repair, np.asarray(rel.c, np.int64))
    O.closure(Xf, rel.closure)
    v2, o2 = O.Evaluator(orig)(Xf)
    assert np.all(v2 == 0)
    assert np.all(o2 <= of)


def test_repair_invariants():
    """On random candidates: the repaired candidate is a subset, every group
    keeps exactly one member iff it had one, and the kept member is a
    selected member of least cost (ties to the first listed)."""
    rng = np.random.default_rng(7)
    n, k = 40, 50
    gp = np.array([0, 5, 9, 9, 20, 33], np.int64)
    gi = rng.permutation(n)[:33].astype(np.int64)
    cost = rng.integers(0, 6, size=n).astype(np.int64)
    X = (rng.random((k, n)) < 0.3).astype(np.uint8)
    R = X.copy()
    O.repair_min(R, (gp, gi), cost)
    assert np.all(R <= X)
    for g in range(gp.size - 1):
        mem = gi[gp[g]:gp[g + 1]]
        for s in range(k):
            sel = mem[X[s, mem] == 1]
            kept = mem[R[s, mem] == 1]
            if sel.size == 0:
                assert kept.size == 0
            else:
                assert kept.size == 1
                cmin = cost[sel].min()
                first = next(m for m in mem if X[s, m] == 1 and cost[m] == cmin)
                assert kept[0] == first
    outside = np.setdiff1d(np.arange(n), gi)
    assert np.array_equal(R[:, outside], X[:, outside])
