"""Pins of the oracle's TU reformulation (Thm. 5) against brute force: on
small instances whose equality rows J are totally unimodular, the
reformulated problem over x_Ibar has the same optimum (plus the constant
c0') and its feasible points map one to one onto the original feasible
points with equal objectives.  No GPU needed."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from oracle import tu as T
from paper_2510_27117_b300 import workloads as W


def _assignment2d(n, idx):
    """min c^T x over n x n permutation matrices: rows sum_j x_ij = 1 and
    columns sum_i x_ij = 1 (bipartite incidence matrix, TU)."""
    rng = np.random.default_rng(100 + idx)
    N = n * n
    rows, cols = [], []
    for i in range(n):
        for j in range(n):
            v = i * n + j
            rows += [i, n + j]
            cols += [v, v]
    B = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(2 * n, N))
    c = rng.integers(-5, 10, size=N).astype(np.float64)
    return W.Instance(f"assign2d_{n}_{idx}", N, c, B=B, d=np.ones(2 * n))


def _all_points(inst):
    """Every binary point with its (viol, obj) under the oracle evaluator."""
    X = np.array(list(itertools.product([0, 1], repeat=inst.n)), np.uint8)
    v, o = O.Evaluator(inst)(X)
    return X, v, o


def _check_equivalent(inst, J, I):
    R, info = T.tu_reformulate(inst, J, I)
    X, v, o = _all_points(inst)
    Xr, vr, orr = _all_points(R)
    feas = {tuple(x): val for x, val, vv in zip(X, o, v) if vv == 0}
    feas_r = [(x, val) for x, val, vv in zip(Xr, orr, vr) if vv == 0]
    assert len(feas_r) == len(feas) > 0
    mapped = T.tu_recover(info, np.array([x for x, _ in feas_r]))
    c0 = info["c0"]
    assert float(c0).is_integer()
    for (xr, val), x in zip(feas_r, mapped):
        assert tuple(x) in feas                       # maps onto a feasible point
        assert feas[tuple(x)] == val + int(c0)        # with the same objective
    assert min(feas.values()) == min(val for _, val in feas_r) + int(c0)
    return R, info


@pytest.mark.parametrize("idx", range(3))
def test_tu_assignment_spanning_tree(idx):
    """J = all rows but the last column row, I = the tree x_00..x_0(n-1),
    x_10, x_20 (B_JI invertible but not a permutation)."""
    n = 3
    inst = _assignment2d(n, idx)
    J = [0, 1, 2, 3, 4]
    I = [0, 1, 2, 3, 6]
    R, info = _check_equivalent(inst, J, I)
    assert R.n == 4 and R.m2 == 1


@pytest.mark.parametrize("idx", range(2))
def test_tu_facility_location_pivots(idx):
    """Customer rows sum_i x_ij = 1 with one pivot x_i0j each (B_JI = I)."""
    inst = W.facility_location(nf=3, nc=3, idx=idx)
    nf = 3
    J = list(range(3))
    # x index nf + j*nf + i; pivot i0 = j mod nf
    I = [nf + j * nf + (j % nf) for j in range(3)]
    R, info = _check_equivalent(inst, J, I)
    assert R.m2 == 0


@pytest.mark.parametrize("idx", range(3))
def test_tu_with_quadratic_term(idx):
    """A non-symmetric integer Q, general rows A x >= b and one equality
    sum_{k < 4} x_k = 1 eliminated through x_2 (a wrong Q', c' or c0' term
    changes some feasible objective)."""
    rng = np.random.default_rng(200 + idx)
    n = 9
    Q = rng.integers(-4, 5, size=(n, n)).astype(np.float64)
    A = sp.csr_matrix(rng.integers(-2, 3, size=(2, n)).astype(np.float64))
    b = np.array([-3.0, -2.0])
    B = sp.csr_matrix((np.ones(4), ([0, 0, 0, 0], [0, 1, 2, 3])), shape=(1, n))
    c = rng.integers(-6, 7, size=n).astype(np.float64)
    inst = W.Instance(f"tuq_{idx}", n, c, A=A, b=b, B=B, d=np.ones(1), Q=Q)
    _check_equivalent(inst, [0], [2])


# ------------------------------------------------ library transform vs oracle
def _as_dense(M, shape):
    if M is None:
        return np.zeros(shape)
    return M.toarray() if sp.issparse(M) else np.asarray(M, np.float64)


def _same_problem(L, R):
    """The library's reformulation equals the oracle's exactly (integral data;
    empty rows and zero entries compared as dense arrays)."""
    assert L.n == R.n
    assert np.array_equal(L.c, R.c)
    assert np.array_equal(_as_dense(L.A, (L.m1, L.n)), _as_dense(R.A, (R.m1, R.n)))
    assert np.array_equal(np.asarray(L.b), np.asarray(R.b))
    assert L.m2 == R.m2
    if L.m2:
        assert np.array_equal(_as_dense(L.B, (L.m2, L.n)), _as_dense(R.B, (R.m2, R.n)))
        assert np.array_equal(np.asarray(L.d), np.asarray(R.d))
    assert (L.Q is None) == (R.Q is None)
    if L.Q is not None:
        assert np.array_equal(_as_dense(L.Q, (L.n, L.n)), _as_dense(R.Q, (R.n, R.n)))


@pytest.mark.parametrize("idx", range(2))
def test_library_tu_matches_oracle_facility(idx):
    from paper_2510_27117_b300 import gfors as G
    inst = W.facility_location(nf=4, nc=5, idx=idx)
    nf = 4
    J = list(range(5))
    I = [nf + j * nf + ((3 * j) % nf) for j in range(5)]
    L, t = G.tu_reformulate(inst, J, I)
    R, info = T.tu_reformulate(inst, J, I)
    _same_problem(L, R)
    assert L.meta["tu_c0"] == info["c0"]
    # recovery agrees with the oracle's on every feasible reformulated point
    Xr = np.array(list(itertools.product([0, 1], repeat=min(L.n, 14))), np.uint8)
    Xr = np.hstack([Xr, np.zeros((Xr.shape[0], L.n - Xr.shape[1]), np.uint8)])
    v, _ = O.Evaluator(R)(Xr)
    ok = Xr[v == 0]
    assert np.array_equal(t.recover(ok), T.tu_recover(info, ok))


@pytest.mark.parametrize("idx", range(3))
def test_library_tu_matches_oracle_quadratic(idx):
    from paper_2510_27117_b300 import gfors as G
    rng = np.random.default_rng(300 + idx)
    n = 11
    Q = rng.integers(-4, 5, size=(n, n)).astype(np.float64)
    A = sp.csr_matrix(rng.integers(-2, 3, size=(3, n)).astype(np.float64))
    b = np.array([-3.0, -2.0, -4.0])
    # two equality rows with pivots x_2 (sign -1) and x_7 (+1); a third row kept
    Bd = np.zeros((3, n))
    Bd[0, [0, 1, 2, 3]] = [1, 1, -1, 1]
    Bd[1, [4, 5, 7]] = [1, -1, 1]
    Bd[2, [2, 7, 9]] = [1, 1, 1]
    inst = W.Instance(f"tuql_{idx}", n, rng.integers(-6, 7, size=n).astype(np.float64),
                      A=A, b=b, B=sp.csr_matrix(Bd), d=np.array([0.0, 1.0, 1.0]),
                      Q=sp.csr_matrix(Q) if idx % 2 else Q)
    L, t = G.tu_reformulate(inst, [1, 0], [7, 2])
    R, info = T.tu_reformulate(inst, [1, 0], [7, 2])
    _same_problem(L, R)
    assert L.meta["tu_c0"] == info["c0"]


def _spanning_tree(n):
    """Rows J: all n row sums and the first n-1 column sums of the n x n
    assignment; columns I: x_0j for every j and x_i0 for i >= 1 (a spanning
    tree of the bipartite graph, B_JI invertible, not a permutation)."""
    J = list(range(2 * n - 1))
    I = [j for j in range(n)] + [i * n for i in range(1, n)]
    return J, I


@pytest.mark.parametrize("n,idx", [(3, 0), (3, 1), (6, 2), (9, 3)])
def test_library_tu_general_pivots_match_oracle(n, idx):
    """A general B_JI goes through exact Gauss-Jordan elimination and gives
    the oracle's reformulation entry by entry."""
    from paper_2510_27117_b300 import gfors as G
    inst = _assignment2d(n, idx)
    J, I = _spanning_tree(n)
    L, t = G.tu_reformulate(inst, J, I)
    R, info = T.tu_reformulate(inst, J, I)
    _same_problem(L, R)
    assert L.meta["tu_c0"] == info["c0"]


def test_library_tu_rejects_non_tu_and_singular():
    from paper_2510_27117_b300 import gfors as G
    # a 2 x 2 block with determinant 2 on the pivot columns: not TU
    Bd = np.array([[1.0, 1.0, 0.0, 1.0], [1.0, -1.0, 1.0, 0.0]])
    inst = W.Instance("nontu", 4, np.ones(4), B=sp.csr_matrix(Bd), d=np.array([1.0, 0.0]))
    with pytest.raises(G.GforsError) as e:
        G.tu_reformulate(inst, [0, 1], [0, 1])
    assert e.value.status == 6                      # GFORS_E_UNSUPPORTED
    # two equal rows on the pivot columns: B_JI singular
    Bd = np.array([[1.0, 1.0, 1.0, 0.0], [1.0, 1.0, 0.0, 1.0]])
    inst = W.Instance("sing", 4, np.ones(4), B=sp.csr_matrix(Bd), d=np.array([1.0, 1.0]))
    with pytest.raises(G.GforsError) as e:
        G.tu_reformulate(inst, [0, 1], [0, 1])
    assert e.value.status == 1                      # GFORS_E_ARG
