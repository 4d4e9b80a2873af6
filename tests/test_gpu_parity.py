"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on
identical seeded inputs.  Bit-exact for sampling, evaluation and the
incumbent; 1e-6 of the absolute-sum scale per PDHG step; 1e-9 relative for
the FP64 spectral norms; 1e-4 relative for LP limits."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import oracle as O
from paper_2510_27117_b300 import workloads as W

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2510_27117_b300.gfors")


def _params(**kw):
    base = dict(k_int=10, k_b=256, seed=0x5EED0000 + 7, x0=0.5)
    base.update(kw)
    return G.default_params(**base), O.Params(**{k: v for k, v in base.items()
                                                  if k in O.Params.__dataclass_fields__})


CASES = {
    "setcover": lambda: W.set_cover(n=500, m=60, density=0.05, idx=3),
    # too large for one block's shared memory (bucketed launches; with
    # pdhg_mode 2 the cooperative one-launch path)
    "assign3d_l2": lambda: W.assign3d(I=24, idx=3),
    "knapsack": lambda: W.knapsack(3001, idx=5),
    "tiny": lambda: W.tiny_bip(n=14, m1=4, m2=1, idx=2),
    "maxcut": lambda: W.max_cut(n=300, idx=1),
    # the paper's weight range on the sparse-Q path: a dense graph handed
    # over as CSR, and a sparse random graph
    "maxcut_csr": lambda: W.max_cut(n=300, idx=1, weights="int8_10", sparse=True),
    "maxcut_sparse": lambda: W.max_cut_sparse(n=3000, avg_deg=12.0, idx=1),
    "assign3d": lambda: W.assign3d(I=8, idx=1),
    "facloc": lambda: W.facility_location(nf=12, nc=40, idx=2),
    # the monotone relaxation: customer rows >= 1, Bernoulli draws, repair
    "facloc_rel": lambda: W.facility_location(nf=12, nc=40, idx=2, relaxed=True),
    # the same shape after the library's TU reformulation (Thm. 5)
    "facloc_tu": lambda: G.tu_reformulate(
        W.facility_location(nf=12, nc=40, idx=2),
        *W.facility_tu_pivots(W.facility_location(nf=12, nc=40, idx=2), 12, 40))[0],
    # the full-size max-cut instance: 4,096 int8 entries per row (1,024 words,
    # a multiple of 128) take the bounds-free row loop of the dense GEMV
    "maxcut_4096": lambda: W.max_cut(n=4096, idx=0),
    # more than 2,048 customers: every facility column y_i is a long CSC
    # column (chunked partial sums plus a finalising pass)
    "facloc_long": lambda: W.facility_location(nf=6, nc=3000, idx=2),
    # 40 long facility columns of one length: a full slice of 32 and one of 8
    # (interleaved sliced-ELL partial sums)
    "facloc_slices": lambda: W.facility_location(nf=40, nc=2100, idx=3),
}


# ------------------------------------------------------------ Preprocess
@pytest.mark.parametrize("name", list(CASES))
def test_preprocess_norms(name):
    inst = CASES[name]()
    gp, op = _params()
    H = G.load(inst, gp)
    S = O.preprocess(inst, op.seed, 0)
    sc = H.get_scales(0)
    assert abs(sc[0] - S.normQ_raw) <= 1e-9 * max(S.normQ_raw, 1e-300)
    assert abs(sc[1] - S.s_obj) <= 1e-9 * S.s_obj
    if S.m:
        nk = S.s_K
        assert abs(sc[2] - nk) <= 1e-9 * nk
    assert abs(sc[3] - S.normQ) <= 1e-9 * max(S.normQ, 1e-300)
    H.destroy()


# ------------------------------------------------------------ PDHG step
def _step_tolerance(S, t1, t2, rho, x, xb, y, y1):
    K = sp.csr_matrix((S.Kv, S.Kc, S.Kp), shape=(S.m, S.n))
    Ka = abs(K)
    if S.qkind == 1:
        qa = np.abs(S.Qd) @ np.abs(x)
    elif S.qkind == 2:
        qa = abs(sp.csr_matrix((S.Qv, S.Qc, S.Qp), shape=(S.n, S.n))) @ np.abs(x)
    else:
        qa = np.zeros(S.n)
    tol_y = 1e-6 * (np.abs(y) + t2 * (Ka @ np.abs(xb) + np.abs(S.r))) + 1e-7
    tol_x = 1e-6 * (np.abs(x) + t1 * (np.abs(S.c) + rho + Ka.T @ np.abs(y1) + 2 * qa
                                      + 2 * rho * np.abs(x))) + 1e-7
    return tol_x, tol_y


@pytest.mark.parametrize("name,mode", [(c, 0) for c in CASES] +
                         [("assign3d_l2", 2), ("maxcut_4096", 1), ("facloc_long", 1),
                          ("facloc_long", 2)])
def test_pdhg_single_step(name, mode):
    inst = CASES[name]()
    gp, op = _params(pdhg_mode=mode)
    H = G.load(inst, gp)
    S = O.preprocess(inst, op.seed, 0)
    rng = np.random.default_rng(11)
    x = rng.random(inst.n).astype(np.float32)
    x[rng.random(inst.n) < 0.1] = 0.0
    x[rng.random(inst.n) < 0.1] = 1.0
    xb = (x + 0.3 * (rng.random(inst.n) - 0.5)).astype(np.float32)
    y = (rng.random(S.m) * 0.5).astype(np.float32)
    if S.m:
        y[S.m1:] -= 0.25
    k, rho = 7, 0.125
    H.set_iterate(0, x, xb, y)
    H.set_counters(k, rho)
    H.pdhg_steps(1)
    gx, gxb, gxp, gy = H.get_iterate(0)
    cap = (S.qkind != 0)
    t1, t2 = O.step_sizes(op.sigma, S.normQ, rho, cap)
    ox, oxb, oy, _ = O.pdhg_step(S, t1, t2, rho, x.astype(np.float64), xb.astype(np.float64),
                                 y.astype(np.float64))
    tol_x, tol_y = _step_tolerance(S, t1, t2, rho, x.astype(np.float64),
                                   xb.astype(np.float64), y.astype(np.float64), oy)
    assert np.all(np.abs(gx - ox) <= tol_x)
    assert np.all(np.abs(gxb - oxb) <= 2 * tol_x + 1e-7)
    assert np.array_equal(gxp, x)
    if S.m:
        assert np.all(np.abs(gy - oy) <= tol_y)
    assert gx.min() >= 0 and gx.max() <= 1
    if S.m1:
        assert gy[:S.m1].min() >= 0
    H.destroy()


# ------------------------------------------------------------ sampling + eval
@pytest.mark.parametrize("name,mode", [("setcover", 0), ("knapsack", 1), ("knapsack", 2),
                                       ("tiny", 0), ("maxcut", 0), ("assign3d", 0),
                                       ("facloc", 0), ("maxcut_csr", 0),
                                       ("maxcut_sparse", 0), ("facloc_tu", 0),
                                       ("facloc_rel", 0), ("facloc_slices", 0)])
def test_sampling_and_evaluation_bit_exact(name, mode):
    inst = CASES[name]()
    gp, op = _params(eval_mode=mode, k_b=96 if name != "maxcut" else 128)
    H = G.load(inst, gp)
    rng = np.random.default_rng(5)
    p = rng.random(inst.n).astype(np.float32)
    p[rng.random(inst.n) < 0.05] = 0.0
    p[rng.random(inst.n) < 0.05] = 1.0
    H.set_iterate(0, p, p, None)
    R = 13
    H.sample_eval(1, R, 0)
    X, viol, obj = H.get_samples(0)
    Xo = O.sample(inst, p, gp.k_b, op.seed, 0, R)
    assert X.shape == Xo.shape
    assert np.array_equal(X, Xo)
    vo, oo = O.Evaluator(inst)(Xo)
    assert np.array_equal(viol, vo)
    assert np.array_equal(obj, oo)
    # incumbent = oracle's incumbent rule on the same scores
    st = dict(found=0, obj=0, round=0, sample=-1)
    O.incumbent_update(st, vo, oo, R)
    inc = H.incumbent(0)
    assert inc["found"] == st["found"]
    if st["found"]:
        assert inc["obj"] == st["obj"] and inc["round"] == R and inc["sample"] == st["sample"]
        assert np.array_equal(inc["x"], Xo[st["sample"]])
    H.destroy()


@pytest.mark.parametrize("I,k_b", [(7, 64), (64, 96), (33, 160)])
def test_axial_sampler_bit_exact(I, k_b):
    """Axial 3D picks (one warp per candidate, slabs staged per step) against
    the oracle: odd I (lanes with partial ranges), I = 64 (128 pairs per
    lane) and a candidate count that leaves idle warps; proposals with zeros
    so that some steps fall back to the uniform pick."""
    inst = W.assign3d(I=I, idx=2)
    gp, op = _params(k_b=k_b)
    H = G.load(inst, gp)
    rng = np.random.default_rng(I)
    p = rng.random(inst.n).astype(np.float32) ** 3
    p[rng.random(inst.n) < 0.3] = 0.0
    if I == 7:
        p[:] = 0.0                                   # every step uniform
    H.set_iterate(0, p, p, None)
    H.sample_eval(1, 4, 0)
    X, viol, obj = H.get_samples(0)
    Xo = O.sample(inst, p, k_b, op.seed, 0, 4)
    assert np.array_equal(X, Xo)
    assert np.all(viol == 0)                          # axial picks are feasible
    H.destroy()


@pytest.mark.parametrize("idx", range(3))
def test_eval_candidates_brute_force(idx):
    inst = W.tiny_bip(n=12, m1=4, m2=1, idx=40 + idx)
    gp, op = _params(k_b=256)
    H = G.load(inst, gp)
    codes = np.arange(1 << inst.n, dtype=np.int64)
    X = ((codes[:, None] >> np.arange(inst.n)[None, :]) & 1).astype(np.uint8)
    viol, obj = H.eval_candidates(X)
    ev = O.Evaluator(inst)
    vo, oo = ev(X)
    assert np.array_equal(viol, vo) and np.array_equal(obj, oo)
    found, best, bx, nf = ev.brute_force()
    feas = viol == 0
    assert feas.sum() == nf
    if found:
        assert obj[feas].min() == best
    H.destroy()


@pytest.mark.parametrize("form", ["dense", "csr", "sparse"])
def test_maxcut_scoring_is_minus_cut(form):
    if form == "sparse":
        inst = W.max_cut_sparse(n=200, avg_deg=20.0, idx=4)
    else:
        inst = W.max_cut(n=200, idx=4, weights="int8_10" if form == "csr" else "pm1",
                         sparse=form == "csr")
    gp, _ = _params(k_b=64)
    H = G.load(inst, gp)
    rng = np.random.default_rng(1)
    X = (rng.random((64, 200)) < 0.5).astype(np.uint8)
    viol, obj = H.eval_candidates(X)
    Wm = inst.meta["W"]
    Wm = Wm.toarray() if sp.issparse(Wm) else Wm
    for s in range(64):
        x = X[s].astype(np.float64)
        cut = 0.5 * np.sum(Wm * (x[:, None] != x[None, :]))
        assert obj[s] == -int(round(cut)) and viol[s] == 0
    H.destroy()


# ------------------------------------------------------------ LP limits
def test_knapsack_lp_limit():
    inst = W.knapsack(2000, idx=9)
    gp, _ = _params(rho_min=0.0, rho_max=0.0, delta=0.0, k_int=1000000)
    H = G.load(inst, gp)
    H.pdhg_steps(30000)
    x, _, _, _ = H.get_iterate(0)
    v, _ = O.knapsack_lp(inst.meta["w"], inst.meta["p"], inst.meta["cap"])
    got = float(inst.meta["p"] @ x.astype(np.float64))
    assert abs(got - v) <= 1e-4 * abs(v)
    st = H.lp_stats(0)
    assert st[0] < 1e-4 and st[1] < 1e-4
    H.destroy()


def test_setcover_lp_limit_and_dual_bound():
    import scipy.optimize as so
    inst = W.set_cover(n=400, m=50, density=0.06, idx=4)
    gp, op = _params(rho_min=0.0, rho_max=0.0, k_int=1000000)
    H = G.load(inst, gp)
    S = O.preprocess(inst, op.seed, 0)
    K = sp.csr_matrix((S.Kv, S.Kc, S.Kp), shape=(S.m, S.n)).toarray()
    res = so.linprog(S.c, A_ub=K, b_ub=-S.r, bounds=[(0, 1)] * S.n, method="highs")
    H.pdhg_steps(40000)
    st = H.lp_stats(0)
    assert st[4] <= res.fun + 1e-6                    # weak duality (certificate)
    assert abs(st[3] - res.fun) <= 1e-4 * abs(res.fun)
    assert st[0] < 1e-4 and st[1] < 1e-4
    H.destroy()


# ------------------------------------------------------------ batching, checkpoint
def test_batched_equals_single():
    insts = [W.knapsack(n, idx=100 + q) for q, n in enumerate([1500, 4000, 777, 2600])]
    gp, _ = _params(k_int=20, k_b=128)
    HB = G.load_batch(insts, gp)
    HB.run(100)
    for q, I in enumerate(insts):
        gq, _ = _params(k_int=20, k_b=128, inst_base=q)
        H1 = G.load(I, gq)
        H1.run(100)
        a, b = HB.incumbent(q), H1.incumbent(0)
        assert a["found"] == b["found"] and a["obj"] == b["obj"]
        assert np.array_equal(a["x"], b["x"])
        xa = HB.get_iterate(q)[0]
        xb = H1.get_iterate(0)[0]
        assert np.array_equal(xa, xb)
        H1.destroy()
    HB.destroy()


def test_checkpoint_resume_bit_exact():
    inst = W.set_cover(n=300, m=40, density=0.08, idx=6)
    gp, _ = _params(k_int=10, k_b=64)
    A = G.load(inst, gp)
    A.run(60)
    blob = A.state_export()
    A.run(120)
    B = G.load(inst, gp)
    B.state_import(blob)
    B.run(120)
    for H in (A, B):
        H.final_round()
    a, b = A.incumbent(0), B.incumbent(0)
    assert a["obj"] == b["obj"] and np.array_equal(a["x"], b["x"])
    assert np.array_equal(A.get_iterate(0)[0], B.get_iterate(0)[0])
    A.destroy()
    B.destroy()


# ------------------------------------------------------------ end to end
@pytest.mark.parametrize("idx", range(3))
def test_run_never_beats_brute_force(idx):
    inst = W.tiny_bip(n=12, m1=3, m2=1, idx=30 + idx)
    gp, _ = _params(k_int=10, k_b=256, seed=100 + idx)
    H = G.load(inst, gp)
    H.run(400)
    inc = H.incumbent(0)
    ev = O.Evaluator(inst)
    found, best, bx, nf = ev.brute_force()
    if inc["found"]:
        assert found and inc["obj"] >= best
        v, o = ev(inc["x"][None, :])
        assert v[0] == 0 and o[0] == inc["obj"]
    H.destroy()


@pytest.mark.parametrize("n", [700, 1024])
def test_persistent_dense_path_matches_launch_path(n):
    """One cooperative launch per call (matrix resident in shared memory,
    blocks meeting at a grid barrier between iterations) against
    per-iteration launches.  Both paths sum each row with the same routine, so the iterates
    must agree exactly; the persistent path is called in uneven pieces so that
    penalty updates (every k_int = 10 iterations) fall inside a launch and
    between launches.  n = 1024 gives rows of 256 words, which take the
    bounds-free row loop; n = 700 the general one."""
    inst = W.max_cut(n=n, idx=6)
    out = []
    for mode, pieces in ((0, (7, 7, 11)), (1, (25,))):
        gp, _ = _params(k_int=10, k_b=64, x0=-1.0, pdhg_mode=mode)
        H = G.load(inst, gp)
        for k in pieces:
            H.pdhg_steps(k)
        x, xb, xp, _ = H.get_iterate(0)
        sc = H.get_scales(0)
        out.append((x, xb, sc))
        H.destroy()
    (xa, xba, sa), (xb_, xbb, sb) = out
    assert np.array_equal(xa, xb_)
    assert np.array_equal(xba, xbb)
    assert sa[6] == sb[6] and sa[7] == sb[7]        # same step sizes (same rho)


# ------------------------------------------------------------ autotuner
def test_autotune_cache_and_parity(tmp_path):
    """gfors_autotune picks lane counts from 1..32 per bucket, stores them
    under the handle's key, and a second handle of the same shape class
    takes them from the cache.  Every lane choice keeps a PDHG step within
    the per-step tolerance of the FP64 oracle."""
    inst = W.set_cover(n=3000, m=300, density=0.02, idx=4)
    gp, op = _params()
    cache = tmp_path / "tune.json"
    H = G.load(inst, gp)
    lanes, hit = H.autotune(cache)
    assert not hit and set(lanes.tolist()) <= {1, 2, 4, 8, 16, 32}
    assert np.array_equal(H.get_lanes(), lanes)
    assert np.array_equal(G.tune_cache_lookup(cache, H.tune_key()), lanes)
    H2 = G.load(inst, gp)
    lanes2, hit2 = H2.autotune(cache)
    assert hit2 and np.array_equal(lanes2, lanes)
    H2.destroy()
    # the tuner touched no state: iterates still those of the load
    x0, xb0, _, y0 = H.get_iterate(0)
    assert np.all(x0 == np.float32(0.5)) and np.all(y0 == 0)
    S = O.preprocess(inst, op.seed, 0)
    rng = np.random.default_rng(5)
    x = rng.random(inst.n).astype(np.float32)
    xb = (x + 0.2 * (rng.random(inst.n) - 0.5)).astype(np.float32)
    y = (rng.random(S.m) * 0.5).astype(np.float32)
    k, rho = 3, 0.25
    t1, t2 = O.step_sizes(op.sigma, S.normQ, rho, False)
    ox, oxb, oy, _ = O.pdhg_step(S, t1, t2, rho, x.astype(np.float64), xb.astype(np.float64),
                                 y.astype(np.float64))
    tol_x, tol_y = _step_tolerance(S, t1, t2, rho, x.astype(np.float64),
                                   xb.astype(np.float64), y.astype(np.float64), oy)
    for choice in (lanes, np.ones(10, np.int32), np.full(10, 32, np.int32),
                   np.array([2, 4, 2, 32, 8, 16, 2, 1, 4, 2], np.int32)):
        H.set_lanes(choice)
        H.set_iterate(0, x, xb, y)
        H.set_counters(k, rho)
        H.pdhg_steps(1)
        gx, gxb, _, gy = H.get_iterate(0)
        assert np.all(np.abs(gx - ox) <= tol_x)
        assert np.all(np.abs(gy - oy) <= tol_y)
    H.destroy()


def test_single_row_path_matches_generic_path():
    """Batches of one-row instances (knapsack) take the fused single-row
    iteration (primal step + K xbar partials, per-instance dual step); it
    must follow the generic bucket / long-row path up to FP32 summation
    order of K xbar, also across a set_iterate in the middle (partials
    recomputed from the new state) and with uneven instance sizes."""
    insts = [W.knapsack(n, idx=20 + q) for q, n in enumerate((3001, 777, 9000))]
    rng = np.random.default_rng(9)
    xs = [rng.random(I.n).astype(np.float32) for I in insts]
    out = []
    for mode in (0, 1):
        gp, _ = _params(k_int=10, pdhg_mode=mode)
        H = G.load_batch(insts, gp)
        H.pdhg_steps(13)
        for q, I in enumerate(insts):
            H.set_iterate(q, xs[q], xs[q], None)
        H.pdhg_steps(17)
        out.append([H.get_iterate(q) for q in range(len(insts))])
        H.destroy()
    for (xa, xba, _, ya), (xb, xbb, _, yb) in zip(*out):
        assert np.max(np.abs(xa - xb)) < 1e-5
        assert np.max(np.abs(xba - xbb)) < 2e-5
        assert np.max(np.abs(ya - yb)) <= 1e-5 * (1 + np.max(np.abs(yb)))


@pytest.mark.parametrize("name", ["setcover", "maxcut", "knapsack"])
def test_candidate_ranges_reproduce_whole_round(name):
    """Disjoint candidate ranges of the same rounds (as on several devices)
    give, after the lexicographic min of their incumbent keys, the incumbent
    of the whole rounds on one handle."""
    import torch
    from paper_2510_27117_b300 import shard as SH
    inst = CASES[name]()
    gp, _ = _params(k_b=256, x0=-1.0 if name == "maxcut" else 0.5)
    keys = []
    for rng_ in [(0, 256), (0, 96), (96, 256)]:
        H = G.load(inst, gp)
        H.pdhg_steps(10)
        if rng_ == (0, 256):
            H.sample_eval(3, 0, 0)
        else:
            H.sample_eval_range(3, 0, 0, *rng_)
        k = torch.zeros(3, dtype=torch.int64, device="cuda")
        H.incumbent_key_async(0, k.data_ptr())
        torch.cuda.synchronize()
        keys.append(k.cpu().numpy())
        inc = H.incumbent(0, want_x=False)
        if inc["found"]:
            assert keys[-1].tolist() == [inc["obj"], inc["round"], inc["sample"]]
        H.destroy()
    whole = keys[0]
    parts = np.stack([np.append(keys[1], 0), np.append(keys[2], 1)])
    assert SH.min_key(parts)[:3].tolist() == whole.tolist()


def test_cooperative_path_matches_launch_path():
    """L2-sized sparse problems run as one cooperative launch per call (dual
    step, grid barrier, primal step, grid barrier); against per-iteration
    launches over calls of uneven length, across penalty updates."""
    inst = W.assign3d(I=24, idx=5)
    out = []
    for mode, pieces in ((2, (7, 13, 5)), (1, (25,))):
        gp, _ = _params(k_int=10, pdhg_mode=mode)
        H = G.load(inst, gp)
        for k in pieces:
            H.pdhg_steps(k)
        out.append((H.get_iterate(0), H.get_scales(0)))
        H.destroy()
    (xa, xba, _, ya), sa = out[0]
    (xb, xbb, _, yb), sb = out[1]
    assert np.max(np.abs(xa - xb)) < 1e-5 and np.max(np.abs(xba - xbb)) < 2e-5
    assert np.max(np.abs(ya - yb)) <= 1e-5 * (1 + np.max(np.abs(yb)))
    assert sa[6] == sb[6] and sa[7] == sb[7]


@pytest.mark.parametrize("I,gamma,L,k_b", [(6, 1, 6, 64), (16, 2, 16, 96), (64, 1, 64, 128),
                                           (9, 0, 3, 32), (12, 1, 0, 64)])
def test_alg4_sampler_bit_exact(I, gamma, L, k_b):
    """Algorithm 4 on the device against the oracle: identical candidates
    (top entries with ties, greedy partial assignment, Philox completion,
    best-improvement interchanges), all feasible, same objectives."""
    inst = W.assign3d(I=I, idx=3, sampler="alg4", gamma=gamma, L=L)
    gp, op = _params(k_b=k_b)
    H = G.load(inst, gp)
    rng = np.random.default_rng(I + gamma)
    p = np.round(rng.random(inst.n) ** 3, 2).astype(np.float32)     # many ties
    H.set_iterate(0, p, p, None)
    H.sample_eval(1, 6, 0)
    X, viol, obj = H.get_samples(0)
    Xo = O.sample(inst, p, k_b, op.seed, 0, 6)
    assert np.array_equal(X, Xo)
    assert np.all(viol == 0)
    vo, oo = O.Evaluator(inst)(Xo)
    assert np.array_equal(obj, oo)
    H.destroy()


def test_tu_incumbent_maps_back():
    """GFORS on a TU-reformulated facility-location instance: the incumbent,
    mapped back by x_I = s + S x_Ibar, is feasible for the original problem
    with objective = reformulated objective + c0' (Thm. 5)."""
    inst = W.facility_location(nf=12, nc=40, idx=5)
    J, I = W.facility_tu_pivots(inst, 12, 40)
    R, tu = G.tu_reformulate(inst, J, I)
    gp, _ = _params(k_b=1024, k_int=50)
    H = G.load(R, gp)
    for r in range(20):
        H.pdhg_steps(50)
        H.sample_eval(1, r, 0)
    inc = H.incumbent(0)
    H.destroy()
    assert inc["found"]
    X = tu.recover(inc["x"][None, :])
    v, o = O.Evaluator(inst)(X)
    assert v[0] == 0 and o[0] == inc["obj"] + int(tu.c0)


@pytest.mark.parametrize("k_b", [96, 2048])
def test_repair_groups_bit_exact(k_b):
    """Monotone-relaxation repair on the device against the oracle: groups
    longer than a warp (nf = 70), dense draws (p near 1) so that many members
    compete, and a candidate count that leaves a partial word."""
    inst = W.facility_location(nf=70, nc=9, idx=4, relaxed=True)
    gp, op = _params(k_b=k_b)
    H = G.load(inst, gp)
    rng = np.random.default_rng(k_b)
    p = (0.5 + 0.5 * rng.random(inst.n)).astype(np.float32)
    H.set_iterate(0, p, p, None)
    H.sample_eval(1, 3, 0)
    X, viol, obj = H.get_samples(0)
    H.destroy()
    Xo = O.sample(inst, p, k_b, op.seed, 0, 3)
    assert np.array_equal(X, Xo)
    vo, oo = O.Evaluator(inst)(Xo)
    assert np.array_equal(viol, vo) and np.array_equal(obj, oo)
    # every customer keeps at most one facility
    assert X[:, 70:].reshape(k_b, 9, 70).sum(-1).max() <= 1


def test_async_io_matches_sync():
    """gfors_set_iterate_async / gfors_incumbent_async / gfors_synchronize give
    the results of the synchronous calls."""
    inst = CASES["setcover"]()
    gp, _ = _params(k_b=256)
    rng = np.random.default_rng(3)
    x = rng.random(inst.n).astype(np.float32)
    keys = []
    for asyn in (False, True):
        H = G.load(inst, gp)
        if asyn:
            H.set_iterate_async(0, x, x, None)
        else:
            H.set_iterate(0, x, x, None)
        H.pdhg_steps(20)
        H.sample_eval(1, 5, 0)
        if asyn:
            k = np.zeros(3, np.int64)
            H.incumbent_async(0, k)
            H.synchronize()
        else:
            inc = H.incumbent(0, want_x=False)
            big = np.iinfo(np.int64).max
            k = np.array([inc["obj"], inc["round"], inc["sample"]] if inc["found"]
                         else [big, big, big], np.int64)
        keys.append(k)
        H.destroy()
    assert np.array_equal(keys[0], keys[1])


# ------------------------------------------------------------ penalty schedule
@pytest.mark.parametrize("kind,delta", [("maxcut", 0.35), ("maxcut", 0.2), ("setcover", 0.35),
                                        ("knapsack", 0.2)])
def test_penalty_schedule_matches_oracle(kind, delta):
    """UpdatePenalty (Section 3) as the device advances it, across several
    sampling triggers, against orc_rho_update: rho_n = clip(rho_min (1 +
    n/T)^p, rho_{n-1} + delta, rho_max), the counter advancing once per k_int
    iterations.  With the step-size cap on, tau1 = min(sqrt(sigma),
    1/(4 (||Q_hat|| + rho))) pins the device's rho; delta = 0.35 makes the
    minimum increment win at n = 1, 2, 3 and rho_max cap n = 4, delta = 0.2
    lets the growth law win first.  Max cut runs the persistent dense kernel
    (every block advances the schedule), set cover the small-instance kernel,
    knapsack the one-row kernels."""
    inst = {"maxcut": lambda: W.max_cut(n=300, idx=1), "setcover": CASES["setcover"],
            "knapsack": CASES["knapsack"]}[kind]()
    sched = dict(rho_min=0.3, rho_max=1.5, T=3.0, p=2.0, delta=delta)
    gp, op = _params(k_int=10, tau_cap_by_L=1, x0=-1.0 if kind == "maxcut" else 0.5, **sched)
    H = G.load(inst, gp)
    S = O.preprocess(inst, op.seed, 0)
    args = (sched["rho_min"], sched["rho_max"], sched["T"], sched["p"], sched["delta"])
    rhos = [O.rho_update(0, 0.0, *args)]
    k = 0
    seen = set()
    for piece in (7, 16, 12, 10, 20):
        H.pdhg_steps(piece)
        k += piece
        n_next = k // 10                         # counter of iteration k + 1
        while len(rhos) <= n_next:
            rhos.append(O.rho_update(len(rhos), rhos[-1], *args))
        want = rhos[n_next]
        seen.add(want)
        t1, t2 = O.step_sizes(op.sigma, S.normQ, want, True)
        sc = H.get_scales(0)
        assert abs(sc[6] - t1) <= 1e-9 * t1 and abs(sc[7] - t2) <= 1e-9 * t2, (k, want)
        st = H.lp_stats(0)
        assert st[6] == want and st[7] == k
    assert len(seen) >= 4 and 1.5 in seen
    H.destroy()


# ------------------------------------------------------------ CheckHalt sums
def _f32(a):
    return None if a is None else np.asarray(a, np.float32).astype(np.float64)


@pytest.mark.parametrize("name", ["setcover", "knapsack", "tiny", "facloc", "assign3d",
                                  "maxcut", "maxcut_sparse"])
def test_lp_stats_match_oracle(name):
    """gfors_lp_stats (FP64 device reductions) entry by entry against
    orc_halt_stats on the same iterate.  The device reduces over its FP32
    copy of the scaled data, so the oracle is given that data rounded to FP32
    as well; what remains is FP64 summation order plus, rarely, a one-ulp
    difference of an FP32 entry where the two FP64 norm estimates straddle a
    rounding boundary (<= 6e-8 of one term), hence 1e-8 of each quantity's
    absolute-sum scale.  With Q != 0 the Q x and Q dx terms come from the
    FP32 GEMV of the PDHG kernels (<= ~6 eps of the absolute sum, as in the
    single-step tolerance), hence 1e-6 of the scale for those."""
    inst = CASES[name]()
    gp, op = _params()
    H = G.load(inst, gp)
    S = O.preprocess(inst, op.seed, 0)
    rng = np.random.default_rng(21)
    x = rng.random(inst.n).astype(np.float32)
    x[rng.random(inst.n) < 0.1] = 0.0
    x[rng.random(inst.n) < 0.1] = 1.0
    y = (rng.random(S.m) * 0.5).astype(np.float32)
    if S.m:
        y[S.m1:] -= 0.25
    rho = 0.125
    H.set_iterate(0, x, x, y)
    H.set_counters(7, rho)
    H.pdhg_steps(1)
    gx, _, gxp, gy = (v.astype(np.float64) for v in H.get_iterate(0))
    st = H.lp_stats(0)
    H.destroy()
    S32 = O.Scaled(**{f: getattr(S, f) for f in S.__dataclass_fields__})
    S32.Kv, S32.r, S32.c = _f32(S.Kv), _f32(S.r), _f32(S.c)
    if S.qkind == 2:
        S32.Qv = _f32(S.Qv)
    t1, _ = O.step_sizes(op.sigma, S.normQ, rho, S.qkind != 0)
    hs = O.halt_stats(S32, t1, rho, gx, gxp, gy)
    K = abs(sp.csr_matrix((S.Kv, S.Kc, S.Kp), shape=(S.m, S.n)))
    if S.qkind == 1:
        Qa = np.abs(S.Qd)
    elif S.qkind == 2:
        Qa = abs(sp.csr_matrix((S.Qv, S.Qc, S.Qp), shape=(S.n, S.n)))
    else:
        Qa = None
    ax, adx = np.abs(gx), np.abs(gx - gxp)
    qtol = 1e-6 if S.qkind == 1 else 1e-8
    tol = 1e-8
    # [0] primal residual
    sc0 = np.linalg.norm(K @ ax + np.abs(S.r)) / (1 + np.linalg.norm(S.r)) if S.m else 0.0
    assert abs(st[0] - hs[0]) <= tol * sc0 + 1e-15
    # [2] binary gap, [6] rho, [7] k
    assert abs(st[2] - hs[2]) <= 1e-13
    assert st[6] == rho and st[7] == 8
    # [3] c^T x + x^T Q x
    sc3 = np.abs(S.c) @ ax + (ax @ (Qa @ ax) if Qa is not None else 0.0)
    assert abs(st[3] - hs[3]) <= qtol * sc3 + 1e-15
    # [5] ||s^x|| (Thm. 2)
    sc5 = np.linalg.norm(adx / t1 + 2 * rho * adx + (2 * (Qa @ adx) if Qa is not None else 0))
    assert abs(st[5] - hs[5]) <= qtol * sc5 + 1e-15
    if S.qkind == 0:
        # [4] Lagrangian dual bound, [1] relative gap against it
        sc4 = np.abs(S.r) @ np.abs(gy) + np.sum(np.abs(S.c) + K.T @ np.abs(gy))
        assert abs(st[4] - hs[4]) <= tol * sc4 + 1e-15
        den = 1 + abs(hs[3]) + abs(hs[4])
        assert abs(st[1] - hs[1]) <= 2 * tol * (sc3 + sc4) / den + 1e-15
    else:
        assert np.isnan(st[4]) and st[1] == st[5]
        assert abs(hs[1] - hs[5]) == 0.0


# ------------------------------------------------------------ general repair
def _covering_instance(n, nr, seed):
    """Random overlapping 0/1 covering rows (relaxed equalities), costs >= 0."""
    rng = np.random.default_rng(seed)
    mem = [np.sort(rng.choice(n, size=rng.integers(2, 40), replace=False)) for _ in range(nr)]
    rp = np.cumsum([0] + [m.size for m in mem]).astype(np.int64)
    ri = np.concatenate(mem).astype(np.int64)
    A = sp.csr_matrix((np.ones(ri.size), ri.astype(np.int32), rp), shape=(nr, n))
    c = rng.integers(0, 30, size=n).astype(np.float64)
    return W.Instance(f"cover_rel_{seed}", n, c, A=A, b=np.ones(nr), repair_rows=(rp, ri))


@pytest.mark.parametrize("case,k_b", [("a3d6", 96), ("a3d12", 160), ("cover", 2048),
                                      ("a3d8_batch", 128)])
def test_repair_rows_bit_exact(case, k_b):
    """Reverse-delete repair on the device against the oracle: relaxed 3D
    assignments (three overlapping rows per variable), random overlapping
    covering rows with dense draws (many members compete), a candidate
    count with a partial word, and a batch in which one instance has no
    repair rows."""
    if case == "a3d6":
        insts = [W.assign3d(I=6, idx=1, sampler="relaxed")]
    elif case == "a3d12":
        insts = [W.assign3d(I=12, idx=2, sampler="relaxed")]
    elif case == "cover":
        insts = [_covering_instance(300, 60, 5)]
    else:
        insts = [W.assign3d(I=8, idx=3, sampler="relaxed"), CASES["setcover"](),
                 W.assign3d(I=8, idx=4, sampler="relaxed")]
    gp, op = _params(k_b=k_b)
    H = G.load_batch(insts, gp)
    rng = np.random.default_rng(k_b)
    ps = []
    for q, I in enumerate(insts):
        p = (0.3 + 0.7 * rng.random(I.n)).astype(np.float32)
        H.set_iterate(q, p, p, None)
        ps.append(p)
    H.sample_eval(1, 5, 0)
    for q, I in enumerate(insts):
        X, viol, obj = H.get_samples(q)
        Xo = O.sample(I, ps[q], k_b, op.seed, q, 5)
        assert np.array_equal(X, Xo), (case, q)
        vo, oo = O.Evaluator(I)(Xo)
        assert np.array_equal(viol, vo) and np.array_equal(obj, oo)
    H.destroy()


def test_repair_rows_equal_group_repair_on_facility_location():
    """On the relaxed facility location the customer rows are disjoint, so
    reverse delete keeps each customer's cheapest selected facility: the
    candidates equal those of the least-cost group repair."""
    base = W.facility_location(nf=40, nc=30, idx=6, relaxed=True)
    rows = base.repair
    alt = W.facility_location(nf=40, nc=30, idx=6, relaxed=True)
    alt.repair, alt.repair_rows = None, rows
    gp, _ = _params(k_b=256)
    out = []
    for I in (base, alt):
        H = G.load(I, gp)
        p = (0.5 + 0.5 * np.random.default_rng(2).random(I.n)).astype(np.float32)
        H.set_iterate(0, p, p, None)
        H.sample_eval(1, 3, 0)
        out.append(H.get_samples(0))
        H.destroy()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("kind", ["setcover", "setcover_batch", "tiny", "assign_small"])
def test_cluster_path_matches_one_block_path(kind):
    """One thread-block cluster per instance (rows and columns split over
    the CTAs, xbar and y exchanged in distributed shared memory) against one
    block per instance (pdhg_mode 3): every row and column is summed the
    same way, so the iterates agree exactly; calls of uneven length put
    penalty updates inside and between launches.  'tiny' has fewer rows and
    columns than CTAs; its rows carry several coefficient values."""
    insts = {"setcover": lambda: [CASES["setcover"]()],
             "setcover_batch": lambda: [W.set_cover(n=700, m=90, density=0.05, idx=70 + q)
                                        for q in range(5)],
             "tiny": lambda: [W.tiny_bip(n=14, m1=4, m2=1, idx=5, with_Q=False)],
             "assign_small": lambda: [W.assign3d(I=6, idx=2)]}[kind]()
    out = []
    for mode, path in ((0, "cluster"), (3, "small")):
        gp, _ = _params(k_int=10, pdhg_mode=mode)
        H = G.load_batch(insts, gp)
        assert H.pdhg_path() == path
        for k in (7, 13, 5, 20):
            H.pdhg_steps(k)
        out.append(([H.get_iterate(q) for q in range(len(insts))],
                    [H.get_scales(q) for q in range(len(insts))]))
        H.destroy()
    for (a, sa), (b, sb) in zip(zip(*out[0]), zip(*out[1])):
        for name, u, v in zip(("x", "xbar", "x_prev", "y"), a, b):
            bad = np.flatnonzero(u != v)
            assert bad.size == 0, (name, bad[:10], u[bad[:5]], v[bad[:5]], u.size)
        assert sa[6] == sb[6] and sa[7] == sb[7]
