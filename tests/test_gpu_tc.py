"""Tensor-core (tcgen05) dense scoring: exact against the CUDA-core scorer
and the integer oracle, including ragged M / N tails and the full
n = 4096, 8,192-candidate max-cut round."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_27117_b300 import workloads as W

pytestmark = pytest.mark.gpu
G = pytest.importorskip("paper_2510_27117_b300.gfors")


def _scores(inst, k_b, mode, R=5, seed=11):
    prm = G.default_params(k_int=10, k_b=k_b, seed=seed, x0=-1.0, eval_mode=mode)
    H = G.load(inst, prm)
    rng = np.random.default_rng(3)
    p = rng.random(inst.n).astype(np.float32)
    H.set_iterate(0, p, p, None)
    H.sample_eval(1, R, 0)
    X, viol, obj = H.get_samples(0)
    inc = H.incumbent(0)
    H.destroy()
    return p, X, viol, obj, inc


@pytest.mark.parametrize("n,k_b,mode", [(300, 96, 3), (200, 512, 3), (513, 288, 3),
                                        (640, 1024, 3), (1100, 544, 3),
                                        (513, 288, 6), (300, 96, 6)])
def test_tc_matches_simt_and_oracle_small(n, k_b, mode):
    """mode 3: the tcgen05 scorer with FP8 E4M3 operands (exact for these
    +-1 graphs); mode 6: bf16 operands."""
    inst = W.max_cut(n=n, idx=7)
    p, X, viol, obj, inc = _scores(inst, k_b, mode)
    _, X2, viol2, obj2, inc2 = _scores(inst, k_b, 4)
    assert np.array_equal(X, X2)
    assert np.array_equal(obj, obj2) and np.all(viol == 0)
    Xo = O.sample(inst, p, k_b, 11, 0, 5)
    assert np.array_equal(X, Xo)
    vo, oo = O.Evaluator(inst)(Xo)
    assert np.array_equal(obj, oo)
    assert inc["obj"] == inc2["obj"] == oo.min()


def test_tc_full_size_round():
    inst = W.max_cut(n=4096, idx=0)
    p, X, viol, obj, inc = _scores(inst, 8192, 3)
    _, X2, viol2, obj2, inc2 = _scores(inst, 8192, 4)
    _, X6, viol6, obj6, inc6 = _scores(inst, 8192, 6)
    assert np.array_equal(obj, obj2)
    assert np.array_equal(obj, obj6)
    assert inc["obj"] == inc2["obj"] and inc["sample"] == inc2["sample"]
    # sampled candidates scored by the oracle from its own draws
    Xo = O.sample(inst, p, 24, 11, 0, 5)
    assert np.array_equal(X[:24], Xo)
    vo, oo = O.Evaluator(inst)(Xo)
    assert np.array_equal(obj[:24], oo)
    # x^T Q x = -cut for the best candidate, counted edge by edge
    Wm = inst.meta["W"]
    xb = inc["x"].astype(bool)
    cut = Wm[np.ix_(xb, ~xb)].sum()
    assert inc["obj"] == -int(cut)


@pytest.mark.parametrize("mode", [3, 4])
def test_dense_scoring_with_linear_term(mode):
    """Dense Q plus a nonzero linear term: objective counted once."""
    inst = W.max_cut(n=257, idx=8)
    inst.c = np.random.default_rng(2).integers(-9, 10, size=257).astype(np.float64)
    prm = G.default_params(k_b=64, seed=5, eval_mode=mode)
    H = G.load(inst, prm)
    X = (np.random.default_rng(4).random((64, 257)) < 0.4).astype(np.uint8)
    viol, obj = H.eval_candidates(X)
    vo, oo = O.Evaluator(inst)(X)
    assert np.array_equal(obj, oo) and np.all(viol == 0)
    H.destroy()


def test_tc_fp8_paper_weight_range():
    """The paper's max-cut weights (integers in [-8, 10]): W2 = 2 w lies in
    the even integers of [-16, 20], all exact in E4M3, so the FP8 scorer
    runs; it must agree with bf16 tensor cores, CUDA cores and the oracle."""
    inst = W.max_cut(n=700, idx=3, weights="int8_10")
    p, X, viol, obj, inc = _scores(inst, 256, 3)
    _, X6, _, obj6, _ = _scores(inst, 256, 6)
    _, X4, _, obj4, _ = _scores(inst, 256, 4)
    assert np.array_equal(X, X6) and np.array_equal(X, X4)
    assert np.array_equal(obj, obj6) and np.array_equal(obj, obj4)
    vo, oo = O.Evaluator(inst)(X)
    assert np.array_equal(obj, oo)
