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


# ---------------------------------------------------------------- general repair
def _rows_of(rows, n):
    rp, ri = rows
    return [ri[rp[r]:rp[r + 1]] for r in range(rp.size - 1)]


def _random_rows(rng, n, nr, size):
    mem = [np.sort(rng.choice(n, size=rng.integers(1, size + 1), replace=False))
           for _ in range(nr)]
    rp = np.cumsum([0] + [m.size for m in mem]).astype(np.int64)
    return rp, np.concatenate(mem).astype(np.int64)


@pytest.mark.parametrize("seed", range(4))
def test_reverse_delete_invariants(seed):
    """On random overlapping covering rows: the repaired candidate is a
    subset; every row covered before stays covered; the result is a minimal
    cover (each kept row variable is the only selected member of some row);
    the cost never rises; variables outside the rows are untouched."""
    rng = np.random.default_rng(seed)
    n, nr, k = 30, 12, 60
    rows = _random_rows(rng, n, nr, 7)
    cost = rng.integers(0, 9, size=n).astype(np.int64)
    X = (rng.random((k, n)) < 0.45).astype(np.uint8)
    R = O.repair_rows(X.copy(), rows, cost)
    mem = _rows_of(rows, n)
    in_rows = np.zeros(n, bool)
    in_rows[rows[1]] = True
    assert np.all(R <= X)
    assert np.array_equal(R[:, ~in_rows], X[:, ~in_rows])
    for s in range(k):
        for m in mem:
            if X[s, m].any():
                assert R[s, m].any()
        for v in np.flatnonzero(R[s] & in_rows):
            assert any(R[s, m].sum() == 1 for m in mem if v in m)
        assert cost @ R[s] <= cost @ X[s]


def test_reverse_delete_on_disjoint_groups_is_least_cost_repair():
    """With disjoint rows the general repair keeps, per row, the cheapest
    selected member, ties to the lower index: exactly the least-cost group
    repair (itself pinned above and by brute force)."""
    rng = np.random.default_rng(3)
    n, k = 50, 80
    perm = rng.permutation(n)[:40]
    gp = np.array([0, 6, 13, 13, 25, 40], np.int64)
    gi = np.concatenate([np.sort(perm[gp[g]:gp[g + 1]]) for g in range(5)]).astype(np.int64)
    cost = rng.integers(0, 4, size=n).astype(np.int64)
    X = (rng.random((k, n)) < 0.5).astype(np.uint8)
    A = O.repair_min(X.copy(), (gp, gi), cost)
    B = O.repair_rows(X.copy(), (gp, gi), cost)
    assert np.array_equal(A, B)


@pytest.mark.parametrize("idx", range(2))
def test_reverse_delete_brute_force_3d_assignment(idx):
    """The relaxed 3D assignment I = 2 (8 binaries, 6 covering rows, costs
    >= 1): over all 256 points, every point covering all rows is repaired
    into a minimal cover that still covers them, at no higher cost; the
    covers of exactly I variables are the assignments, and the cheapest
    repaired cover of I variables is the original optimum (brute force)."""
    orig = W.assign3d(I=2, idx=idx)
    rel = W.assign3d(I=2, idx=idx, sampler="relaxed")
    X = np.array(list(itertools.product([0, 1], repeat=rel.n)), np.uint8)
    v, o = O.Evaluator(rel)(X)
    R = O.repair_rows(X[v == 0].copy(), rel.repair_rows, np.asarray(rel.c, np.int64))
    v2, o2 = O.Evaluator(rel)(R)
    assert np.all(v2 == 0) and np.all(o2 <= o[v == 0])
    f, best, _, _ = O.Evaluator(orig).brute_force()
    exact = R.sum(axis=1) == 2
    vo, oo = O.Evaluator(orig)(R[exact])
    assert np.all(vo == 0) and f and oo.min() == best
