"""Exact evaluation (viol_s, obj_s of Eq. (1)) through the C ABI against the
FP64 oracle on instances built to reach every evaluation path: two-variable
rows in long strided runs around hub variables (every truth table,
inequalities and equalities, either variable order), short runs and single
rows; linear objectives whose 32-variable cost spans need few or many bit
planes (and more than 12); candidate sets that are dense, one-hot sparse
(at most one bit per candidate in each 32-variable slab) and ragged in the
candidate count (several passes over the candidate words)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2510_27117_b300 import workloads as W

pytestmark = pytest.mark.gpu
G = pytest.importorskip("paper_2510_27117_b300.gfors")

NH = 12                       # hub variables: even k at index k, odd k at n - 1 - k


def _instance(seed):
    rng = np.random.default_rng(seed)
    n = 4096
    rows_a, rhs_a, rows_b, rhs_b = [], [], [], []
    # long runs: hub k with members v = NH + k + NH q (stride NH), one row
    # form per hub; even hubs have the lowest indices (first in their rows),
    # odd hubs the highest (second in their rows)
    hub = [k if k % 2 == 0 else n - 1 - k for k in range(NH)]
    forms = [(1, -1, 0), (-1, 1, 0), (1, 1, 1), (-1, -1, -1), (2, -1, 0), (1, 2, 2),
             (-1, 3, 0), (3, 3, 3), (1, -2, -1), (-2, -2, -3), (1, 1, 2), (5, -4, 1)]
    for k in range(NH):
        a, b, r = forms[k]
        for q in range(200 + 7 * k):
            v = NH + k + NH * q
            if v >= n - NH:
                break
            rows_a.append({v: a, hub[k]: b})
            rhs_a.append(r)
    # equality runs (B rows): x_v = x_h and x_v + x_h = 1
    for k in range(3):
        for q in range(120):
            v = NH + 3000 + k + 3 * q
            if v >= n - NH:
                break
            rows_b.append({v: 1, hub[k]: -1} if k != 1 else {v: 1, hub[k]: 1})
            rhs_b.append(0 if k != 1 else 1)
    # short runs (below the run threshold) and scattered pairs
    for q in range(40):
        h = hub[int(rng.integers(0, NH))]
        for t in range(int(rng.integers(2, 9))):
            v = int(rng.integers(NH, n - NH))
            rows_a.append({v: int(rng.choice([-1, 1])), h: int(rng.choice([-1, 1]))})
            rhs_a.append(int(rng.integers(-1, 2)))
    # single-variable rows
    for q in range(30):
        v = int(rng.integers(NH, n - NH))
        rows_a.append({v: 1})
        rhs_a.append(int(rng.integers(0, 2)))

    def csr(rows):
        ptr, idx, val = [0], [], []
        for r in rows:
            for c_, x in sorted(r.items()):
                idx.append(c_)
                val.append(float(x))
            ptr.append(len(idx))
        return sp.csr_matrix((np.array(val), np.array(idx, np.int32), np.array(ptr)),
                             shape=(len(rows), n))

    c = rng.integers(-50, 51, size=n).astype(np.float64)
    c[1024:1536] = rng.integers(-3, 4, size=512)            # narrow spans
    c[2048:2112] = rng.integers(-(1 << 20), 1 << 20, 64)    # spans over 12 planes
    c[3000:3100] = 7.0                                      # zero span
    return W.Instance(f"evalpaths_{seed}", n, c, A=csr(rows_a),
                      b=np.array(rhs_a, np.float64), B=csr(rows_b),
                      d=np.array(rhs_b, np.float64))


def _candidates(kind, k, n, rng):
    if kind == "dense":
        return (rng.random((k, n)) < 0.5).astype(np.uint8)
    if kind == "sparse":
        # one set bit per candidate in each 32-variable slab, hubs set at random
        X = np.zeros((k, n), np.uint8)
        pick = rng.integers(0, 32, size=(k, n // 32)) + 32 * np.arange(n // 32)[None, :]
        X[np.arange(k)[:, None], pick] = 1
        X[:, :NH] = rng.random((k, NH)) < 0.5
        X[:, n - NH:] = rng.random((k, NH)) < 0.5
        return X
    # mixed: sparse slabs with a few dense ones
    X = _candidates("sparse", k, n, rng)
    for s in rng.choice(n // 32, size=8, replace=False):
        X[:, 32 * s:32 * s + 32] = rng.random((k, 32)) < 0.6
    return X


@pytest.mark.parametrize("k", [96, 256, 300])
@pytest.mark.parametrize("kind", ["dense", "sparse", "mixed"])
def test_eval_paths_match_oracle(kind, k):
    inst = _instance(7)
    H = G.load(inst, G.default_params(k_b=(k + 31) // 32 * 32, seed=0x5EED0101))
    X = _candidates(kind, k, inst.n, np.random.default_rng(k))
    viol, obj = H.eval_candidates(X)
    vo, oo = O.Evaluator(inst)(X)
    H.destroy()
    assert np.array_equal(viol, vo)
    assert np.array_equal(obj, oo)
    assert (vo > 0).any()

