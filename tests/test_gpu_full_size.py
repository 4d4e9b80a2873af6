"""Parity at the sizes the bench times, on sampled outputs the oracle can
compute one by one and on properties that hold at any size:
- the 512-knapsack batch (sum n = 2.75e7, 4,096 candidates per instance, the
  fused single-row path): candidates re-drawn by the oracle from their
  Philox counters and scored exactly;
- one 1,000 x 10,000 facility-location instance (1e7 binaries, one-hot
  groups + closure, learned-proposal-free): the incumbent is feasible for
  the original data with the reported objective."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_27117_b300 import workloads as W

pytestmark = pytest.mark.gpu
G = pytest.importorskip("paper_2510_27117_b300.gfors")


def test_knapsack_batch_full_size_sampled():
    insts = W.knapsack_batch(ninst=512)
    seed, R = 0x5EED0002, 3
    prm = G.default_params(k_int=50, k_b=4096, seed=seed, x0=0.5)
    H = G.load_batch(insts, prm)
    H.pdhg_steps(50)
    H.sample_eval(1, R, 0)
    rng = np.random.default_rng(12)
    for q in rng.choice(len(insts), size=4, replace=False):
        q = int(q)
        I = insts[q]
        x, _, _, _ = H.get_iterate(q)
        _, viol, obj = H.get_samples(q, want_x=False)
        assert viol.size == 4096
        for s in list(rng.choice(4096, size=3, replace=False)) + [4095]:
            Xs = O.bernoulli(x, 1, seed, q, R, first=int(s))
            v, o = O.Evaluator(I)(Xs)
            assert viol[s] == v[0] and obj[s] == o[0]
        inc = H.incumbent(q)
        if inc["found"]:
            v, o = O.Evaluator(I)(inc["x"][None, :])
            assert v[0] == 0 and o[0] == inc["obj"]
    H.destroy()


def test_facility_location_full_size_incumbent():
    inst = W.facility_location(1000, 10000, idx=0)
    prm = G.default_params(k_int=50, k_b=256, seed=0x5EED0001, x0=0.5)
    H = G.load_batch([inst], prm)
    for r in range(4):
        H.pdhg_steps(50)
        H.sample_eval(4, 4 * r, 0)
    inc = H.incumbent(0)
    _, viol, obj = H.get_samples(0, want_x=False)
    H.destroy()
    assert inc["found"]
    v, o = O.Evaluator(inst)(inc["x"][None, :])
    assert v[0] == 0 and o[0] == inc["obj"]
    # every candidate's objective is at least the incumbent's, and the
    # incumbent is the least feasible objective of its own round or earlier
    feas = viol == 0
    if feas.any():
        assert obj[feas].min() >= inc["obj"]
