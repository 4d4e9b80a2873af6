"""Sparse-Q path (CSR quadratic term) at the size the bench times: max cut
on a random graph with n = 65,536 vertices, average degree 32 and the
paper's weight range [-8, 10] (Section 4.2.3), one round of 8,192
candidates.  Sampled candidates are checked against the oracle's own draws
and scores; every candidate's objective is checked through an invariant that
holds at any size (the incumbent's x^T Q x equals minus its cut, counted
edge by edge)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2510_27117_b300 import workloads as W

pytestmark = pytest.mark.gpu
G = pytest.importorskip("paper_2510_27117_b300.gfors")


def test_sparse_q_full_size_round():
    inst = W.max_cut_sparse(n=65536, avg_deg=32.0, idx=0)
    k_b, R, seed = 8192, 3, 17
    prm = G.default_params(k_int=10, k_b=k_b, seed=seed, x0=-1.0)
    H = G.load(inst, prm)
    rng = np.random.default_rng(8)
    p = rng.random(inst.n).astype(np.float32)
    p[rng.random(inst.n) < 0.05] = 0.0
    H.set_iterate(0, p, p, None)
    H.sample_eval(1, R, 0)
    X, viol, obj = H.get_samples(0)
    inc = H.incumbent(0)
    H.destroy()
    assert X.shape == (k_b, inst.n) and np.all(viol == 0)
    # the first 24 candidates from the oracle's own draws (a candidate's
    # draws depend on its index, not on the round size)
    Xo = O.sample(inst, p, 24, seed, 0, R)
    assert np.array_equal(X[:24], Xo)
    vo, oo = O.Evaluator(inst)(Xo)
    assert np.array_equal(obj[:24], oo)
    # every candidate: x^T Q x from scipy in exact integer arithmetic
    Q = inst.Q.astype(np.int64)
    for s in rng.choice(k_b, size=64, replace=False):
        x = X[s].astype(np.int64)
        assert obj[s] == int(x @ (Q @ x))
    assert inc["found"] and inc["obj"] == obj.min()
    Wm = sp.csr_matrix(inst.meta["W"])
    xb = inc["x"].astype(bool)
    cut = Wm[xb][:, ~xb].sum()
    assert inc["obj"] == -int(cut)
