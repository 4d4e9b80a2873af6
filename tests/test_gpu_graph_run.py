"""Alg. 1 as one CUDA-graph launch (gfors_run_graph: a conditional while
node per run, CheckHalt evaluated on the device) against the host loop
(gfors_run): identical iterates, incumbents (objective, round, candidate,
x), CheckHalt statistics and iteration counts, on every PDHG path the graph
captures (one-row batches, one block or one thread-block cluster per
instance, bucketed launches with
one-hot groups and closure, dense Q with per-iteration launches and
tensor-core scoring), with halting by CheckHalt and by the iteration
budget, and with the learned proposals."""
import numpy as np
import pytest

from paper_2510_27117_b300 import workloads as W

pytestmark = pytest.mark.gpu
G = pytest.importorskip("paper_2510_27117_b300.gfors")
P = pytest.importorskip("paper_2510_27117_b300.proposal")

CASES = {
    "knapsack_batch": (lambda: [W.knapsack(n, idx=40 + q) for q, n in
                                enumerate((3001, 777, 9000))], {}, "one_row"),
    "setcover_batch": (lambda: [W.set_cover(n=400, m=40, density=0.08, idx=60 + q)
                                for q in range(3)], {}, "cluster"),
    "setcover_batch_small": (lambda: [W.set_cover(n=400, m=40, density=0.08, idx=60 + q)
                                      for q in range(3)], dict(pdhg_mode=3), "small"),
    "assign3d": (lambda: [W.assign3d(I=24, idx=3)], {}, "buckets"),
    "facloc": (lambda: [W.facility_location(nf=30, nc=400, idx=2)], {}, "buckets"),
    "maxcut_launch": (lambda: [W.max_cut(n=300, idx=1)], dict(pdhg_mode=1, x0=-1.0),
                      "buckets"),
}


def _both(name, max_iters, proposal=0, W_prop=None, **kw):
    make, extra, path = CASES[name]
    insts = make()
    prm_kw = dict(k_int=10, k_b=128, seed=0x5EED0011)
    prm_kw.update(extra)
    prm_kw.update(kw)
    out = []
    for graph in (False, True):
        H = G.load_batch(insts, G.default_params(**prm_kw))
        assert H.pdhg_path() == path
        if W_prop is not None:
            H.set_proposal(W_prop)
        if graph:
            it, trig = H.run_graph(max_iters, proposal=proposal)
        else:
            it, trig = H.run(max_iters, proposal=proposal), None
        res = dict(it=it, trig=trig,
                   inc=[H.incumbent(q) for q in range(len(insts))],
                   x=[H.get_iterate(q)[0] for q in range(len(insts))],
                   st=[H.lp_stats(q) for q in range(len(insts))])
        H.destroy()
        out.append(res)
    return out


def _same(a, b):
    assert a["it"] == b["it"]
    for ia, ib in zip(a["inc"], b["inc"]):
        assert ia["found"] == ib["found"]
        if ia["found"]:
            assert (ia["obj"], ia["round"], ia["sample"]) == (ib["obj"], ib["round"],
                                                               ib["sample"])
            assert np.array_equal(ia["x"], ib["x"])
    for xa, xb in zip(a["x"], b["x"]):
        assert np.array_equal(xa, xb)
    for sa, sb in zip(a["st"], b["st"]):
        assert np.array_equal(sa, sb, equal_nan=True)


@pytest.mark.parametrize("name", list(CASES))
def test_graph_run_equals_host_loop_budget(name):
    """The iteration budget ends the loop (CheckHalt off: tolerance 0, long
    stall window); 95 iterations leave 5 after the last trigger."""
    a, b = _both(name, 95, halt_tol=0.0, stall_window=1000)
    _same(a, b)
    assert b["trig"] == 9


@pytest.mark.parametrize("name", ["knapsack_batch", "setcover_batch", "setcover_batch_small",
                                  "facloc"])
def test_graph_run_equals_host_loop_checkhalt(name):
    """CheckHalt ends the loop early (loose tolerance, short stall window):
    the device decides at the same trigger as the host loop."""
    a, b = _both(name, 2000, halt_tol=1e-2, stall_window=3)
    _same(a, b)
    assert b["it"] < 2000 and b["trig"] == b["it"] // 10


@pytest.mark.parametrize("proposal", [1, 2, 3])
@pytest.mark.parametrize("name", ["assign3d", "facloc"])
def test_graph_run_learned_proposals(name, proposal):
    a, b = _both(name, 60, proposal=proposal, W_prop=P.init_weights(3), halt_tol=0.0,
                 stall_window=1000)
    _same(a, b)


def test_graph_run_targets_stop_at_first_hit():
    """With targets the loop stops after the first trigger at which every
    instance holds a feasible incumbent no worse than its target."""
    insts = CASES["knapsack_batch"][0]()
    prm = G.default_params(k_int=10, k_b=128, seed=0x5EED0011, halt_tol=0.0,
                           stall_window=1000)
    H = G.load_batch(insts, prm)
    trace = []
    for t in range(30):
        H.pdhg_steps(10)
        H.sample_eval(1, t, 0)
        trace.append([H.incumbent(q, want_x=False)["obj"] for q in range(3)])
    H.destroy()
    tgt = trace[-1]
    first = next(t for t, b in enumerate(trace) if all(x <= y for x, y in zip(b, tgt)))
    H = G.load_batch(insts, prm)
    it, trig = H.run_graph(300, targets=tgt)
    objs = [H.incumbent(q, want_x=False)["obj"] for q in range(3)]
    H.destroy()
    assert trig == first + 1 and it == 10 * (first + 1)
    assert all(o <= t for o, t in zip(objs, tgt))


def test_graph_run_unsupported_forms():
    H = G.load(W.max_cut(n=300, idx=1), G.default_params(k_int=10, k_b=64, x0=-1.0))
    assert H.pdhg_path() == "persistent"
    with pytest.raises(G.GforsError) as e:
        H.run_graph(50)
    assert e.value.status == 6
    H.destroy()
    H = G.load(W.knapsack(500, idx=1), G.default_params(k_int=7, k_b=64))
    with pytest.raises(G.GforsError) as e:
        H.run_graph(70)
    assert e.value.status == 6
    H.destroy()


def test_graph_reused_across_calls_and_rebuilt_after_lane_change():
    """One instantiated graph serves successive calls (the budget and the
    first trigger come from device memory); a lane change rebuilds it.
    Results equal the host loop's over the same sequence of calls."""
    insts = CASES["assign3d"][0]()
    prm = G.default_params(k_int=10, k_b=128, seed=0x5EED0011, halt_tol=0.0,
                           stall_window=1000)
    A = G.load_batch(insts, prm)
    A.run(40)
    A.run(90)
    B = G.load_batch(insts, prm)
    B.run_graph_prepare(0)
    assert B.run_graph(40) == (40, 4)
    B.set_lanes(B.get_lanes())              # same lanes, new structure version
    assert B.run_graph(90) == (90, 5)
    a = dict(it=90, inc=[A.incumbent(0)], x=[A.get_iterate(0)[0]], st=[A.lp_stats(0)])
    b = dict(it=90, inc=[B.incumbent(0)], x=[B.get_iterate(0)[0]], st=[B.lp_stats(0)])
    _same(a, b)
    A.destroy()
    B.destroy()
