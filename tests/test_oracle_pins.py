"""Pins of the FP64 CPU oracle against things other than itself: published
known-answer vectors, closed forms, library routines (numpy / scipy / torch
CPU), brute force and the paper's invariants.  No GPU needed."""
import math
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

from oracle import oracle as O
from paper_2510_27117_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_philox_lane_layout_and_uniformity():
    # lane layout: four consecutive indices share one call
    seed = 0x123456789ABCDEF
    lanes = O.philox_lanes(seed, 0, 7, 3, 5, 8)
    for g in range(2):
        ref = O.philox4x32_10([g, 5, 3, 7], [seed & 0xFFFFFFFF, seed >> 32])
        assert list(lanes[4 * g:4 * g + 4]) == list(ref)
    # chi-square on low and high bytes of 2^18 draws
    u = O.philox_lanes(1, 0, 0, 0, 0, 1 << 18)
    for b in (u & 0xFF, u >> 24):
        h = np.bincount(b.astype(np.int64), minlength=256)
        e = u.size / 256
        chi2 = ((h - e) ** 2 / e).sum()
        assert chi2 < 255 + 6 * math.sqrt(2 * 255)


# ---------------------------------------------------------------- Preprocess
def test_power_norm_matches_svd():
    rng = np.random.default_rng(3)
    for (m, n) in [(5, 9), (30, 17), (1, 40)]:
        K = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.5)
        Ks = sp.csr_matrix(K)
        v, it = O.power_norm_K(*O._csr_parts(Ks, np.float64), n, 99, 0)
        assert abs(v - np.linalg.norm(K, 2)) <= 1e-9 * np.linalg.norm(K, 2)
    S = rng.integers(-3, 4, size=(25, 25)).astype(float)
    S = S + S.T
    v, it = O.power_norm_Q(S, 25, 5, 0)
    assert abs(v - np.abs(np.linalg.eigvalsh(S)).max()) <= 1e-9 * v
    v2, _ = O.power_norm_Q(sp.csr_matrix(S), 25, 5, 0)
    assert abs(v - v2) <= 1e-12 * v


def test_preprocess_normalisations():
    inst = W.tiny_bip(n=14, m1=5, m2=2, idx=4)
    S = O.preprocess(inst, 11)
    K = sp.csr_matrix((S.Kv, S.Kc, S.Kp), shape=(S.m, S.n)).toarray()
    # after row scaling and division by ||K||: spectral norm one
    assert abs(np.linalg.norm(K, 2) - 1.0) < 1e-9
    # rows remain parallel to -[A;B] rows, r scaled with the same factor
    Kraw = -np.vstack([inst.A.toarray(), inst.B.toarray()])
    rraw = np.concatenate([inst.b, inst.d])
    for j in range(S.m):
        f = np.linalg.norm(Kraw[j]) * S.s_K
        assert np.allclose(K[j] * f, Kraw[j], atol=1e-12)
        assert abs(S.r[j] * f - rraw[j]) < 1e-9
    # objective scaled by ||Q||_2 + ||c||_2
    Qs = 0.5 * (inst.Q.toarray() + inst.Q.toarray().T)
    s = np.abs(np.linalg.eigvalsh(Qs)).max() + np.linalg.norm(inst.c)
    assert abs(S.s_obj - s) < 1e-9 * s
    assert abs(S.normQ + np.linalg.norm(S.c) - 1.0) < 1e-9


def test_empty_infeasible_row_rejected():
    A = sp.csr_matrix(np.array([[1.0, 1.0], [0.0, 0.0]]))
    inst = W.Instance("bad", 2, np.ones(2), A=A, b=np.array([1.0, 1.0]))
    with pytest.raises(ValueError):
        O.preprocess(inst, 1)
    inst.b = np.array([1.0, -1.0])            # 0 >= -1 holds: fine
    O.preprocess(inst, 1)


def test_step_sizes_and_penalty_schedule():
    t1, t2 = O.step_sizes(0.99, 0.0, 0.0, 0)
    assert abs(t1 * t2 - 0.99) < 1e-15 and abs(t1 - math.sqrt(0.99)) < 1e-15
    t1, t2 = O.step_sizes(0.5, 1.0, 0.3, 1)
    assert abs(t1 - 1 / (4 * 1.3)) < 1e-15 and abs(t1 * t2 - 0.5) < 1e-15
    # closed form with delta = 0 and the growth law of Section 3
    rho = O.rho_update(0, 0.0, 1e-3, 1.0, 20.0, 2.0, 0.0)
    assert rho == 1e-3
    for n in range(1, 200):
        rho = O.rho_update(n, rho, 1e-3, 1.0, 20.0, 2.0, 0.0)
        assert abs(rho - min(1e-3 * (1 + n / 20) ** 2, 1.0)) < 1e-15
    # minimum increment delta dominates a flat schedule; rho_max caps
    rho = 0.1
    for n in range(1, 6):
        rho = O.rho_update(n, rho, 0.1, 0.35, 1e9, 1.0, 0.1)
    assert rho == 0.35


# ---------------------------------------------------------------- PDHG
def _lp_scaled(S, ineq_only=False):
    K = sp.csr_matrix((S.Kv, S.Kc, S.Kp), shape=(S.m, S.n)).toarray()
    m1 = S.m1
    kw = dict(c=S.c, bounds=[(0, 1)] * S.n, method="highs")
    if m1:
        kw.update(A_ub=K[:m1], b_ub=-S.r[:m1])
    if S.m > m1:
        kw.update(A_eq=K[m1:], b_eq=-S.r[m1:])
    res = so.linprog(**kw)
    assert res.status == 0
    y = np.zeros(S.m)
    if m1:
        y[:m1] = -res.ineqlin.marginals
    if S.m > m1:
        y[m1:] = -res.eqlin.marginals
    return res, y


@pytest.mark.parametrize("maker", [
    lambda: W.set_cover(n=60, m=12, density=0.15, idx=1),
    lambda: W.knapsack(40, idx=2),
    lambda: W.tiny_bip(n=16, m1=4, m2=1, idx=6, with_Q=False),
])
def test_pdhg_saddle_point_is_fixed_point(maker):
    """Alg. 2 with rho = 0 maps an LP saddle point (from HiGHS) to itself."""
    inst = maker()
    S = O.preprocess(inst, 5)
    res, y = _lp_scaled(S)
    x = res.x.copy()
    t1, t2 = O.step_sizes(0.99, S.normQ, 0.0, 0)
    x1, xb1, y1, _ = O.pdhg_step(S, t1, t2, 0.0, x, x, y)
    assert np.abs(x1 - x).max() < 1e-7
    assert np.abs(y1 - y).max() < 1e-7
    assert np.abs(xb1 - x).max() < 1e-7


def _lagrangian(S, rho, x, y):
    """L_hat of Eq. (2) evaluated as a scalar function."""
    K = sp.csr_matrix((S.Kv, S.Kc, S.Kp), shape=(S.m, S.n))
    if S.qkind == 1:
        Qx = S.Qd @ x
    elif S.qkind == 2:
        Qx = sp.csr_matrix((S.Qv, S.Qc, S.Qp), shape=(S.n, S.n)) @ x
    else:
        Qx = np.zeros(S.n)
    return x @ Qx + S.c @ x + y @ (K @ x + S.r) + rho * x @ (1 - x)


def test_pdhg_gradient_is_lagrangian_gradient():
    """delta of Alg. 2 equals grad_x L_hat(x_{k-1}; y_k) (Eq. 2) by central
    differences of the scalar Lagrangian."""
    inst = W.tiny_bip(n=12, m1=4, m2=1, idx=8)
    S = O.preprocess(inst, 3)
    rng = np.random.default_rng(0)
    x = rng.random(S.n)
    xb = rng.random(S.n)
    y = rng.random(S.m)
    rho = 0.37
    x1, xb1, y1, delta = O.pdhg_step(S, 0.1, 0.2, rho, x, xb, y)
    h = 1e-6
    for i in range(S.n):
        e = np.zeros(S.n)
        e[i] = h
        fd = (_lagrangian(S, rho, x + e, y1) - _lagrangian(S, rho, x - e, y1)) / (2 * h)
        assert abs(fd - delta[i]) < 1e-7
    # dual step: y_k = Proj(y_{k-1} + tau2 grad_y L_hat(xbar_{k-1}))
    for j in range(S.m):
        e = np.zeros(S.m)
        e[j] = h
        g = (_lagrangian(S, rho, xb, y + e) - _lagrangian(S, rho, xb, y - e)) / (2 * h)
        want = y[j] + 0.2 * g
        if j < S.m1:
            want = max(want, 0.0)
        assert abs(want - y1[j]) < 1e-7
    assert x1.min() >= 0 and x1.max() <= 1 and y1[:S.m1].min() >= 0
    assert np.allclose(xb1, 2 * x1 - x)


def test_knapsack_lp_limit_matches_greedy():
    """With rho = 0 the PDHG iterates reach the fractional-knapsack LP
    optimum, whose closed form is Dantzig's greedy."""
    inst = W.knapsack(30, idx=3)
    S = O.preprocess(inst, 1)
    v, xg = O.knapsack_lp(inst.meta["w"], inst.meta["p"], inst.meta["cap"])
    t1, t2 = O.step_sizes(0.99, 0.0, 0.0, 0)
    x = np.full(S.n, 0.5)
    xb = x.copy()
    y = np.zeros(S.m)
    for _ in range(20000):
        x, xb, y, _ = O.pdhg_step(S, t1, t2, 0.0, x, xb, y)
    obj = -(inst.meta["p"] @ x)
    assert abs(obj - (-v)) <= 1e-6 * abs(v)
    hs = O.halt_stats(S, t1, 0.0, x, x, y)
    assert hs[0] < 1e-6 and hs[1] < 1e-6


def test_knapsack_greedy_matches_linprog():
    for idx in range(3):
        inst = W.knapsack(50, idx=idx)
        w, p, cap = inst.meta["w"], inst.meta["p"], inst.meta["cap"]
        v, x = O.knapsack_lp(w, p, cap)
        res = so.linprog(-p, A_ub=w[None, :], b_ub=[cap], bounds=[(0, 1)] * w.size,
                         method="highs")
        assert abs(v + res.fun) < 1e-9 * v
        assert abs(w @ x - cap) < 1e-9 * cap


def test_dual_bound_is_valid_and_tight():
    """D(y) <= LP* for every y >= 0 (weak duality); equality at the LP dual."""
    inst = W.set_cover(n=80, m=15, density=0.12, idx=2)
    S = O.preprocess(inst, 2)
    res, ystar = _lp_scaled(S)
    rng = np.random.default_rng(1)
    for _ in range(20):
        y = rng.random(S.m) * rng.random()
        hs = O.halt_stats(S, 0.5, 0.0, res.x, res.x, y)
        assert hs[4] <= res.fun + 1e-12
    hs = O.halt_stats(S, 0.5, 0.0, res.x, res.x, ystar)
    assert abs(hs[4] - res.fun) < 1e-8
    assert hs[0] < 1e-9
    assert hs[1] < 1e-8


def test_halt_binary_gap_closed_form():
    inst = W.set_cover(n=30, m=6, density=0.3, idx=0)
    S = O.preprocess(inst, 2)
    x = np.linspace(0, 1, S.n)
    hs = O.halt_stats(S, 0.5, 0.0, x, x, np.zeros(S.m))
    assert abs(hs[2] - np.minimum(x, 1 - x).mean()) < 1e-15


def test_prop2_inequality_holds():
    """Prop. 2 under tau1 tau2 ||K||^2 <= 1/2, tau1 <= 1/(2L), fixed rho."""
    inst = W.tiny_bip(n=14, m1=4, m2=1, idx=11)
    S = O.preprocess(inst, 9)
    rho = 0.2
    L = 2 * (S.normQ + rho)
    t1 = 1 / (2 * L)
    t2 = 0.5 / t1
    x = np.full(S.n, 0.5)
    xb = x.copy()
    y = np.zeros(S.m)

    def phi(x, y):
        return _lagrangian(S, rho, x, y)

    phi0 = phi(x, y)
    sx = sy = sxx = 0.0
    N = 300
    for _ in range(N):
        sxx += x @ x
        x1, xb, y1, _ = O.pdhg_step(S, t1, t2, rho, x, xb, y)
        sx += np.sum((x1 - x) ** 2)
        sy += np.sum((y1 - y) ** 2)
        x, y = x1, y1
    lhs = sx / t1 + sy / t2
    rhs = 4 * (phi0 - phi(x, y)) + 8 / t1 * sxx + 16 * t2 * (S.r @ S.r) * N
    assert lhs <= rhs


# ---------------------------------------------------------------- sampling
def test_bernoulli_threshold_edges_and_means():
    n, k = 64, 4096
    p = np.linspace(0, 1, n).astype(np.float32)
    X = O.bernoulli(p, k, 77, 0, 0)
    assert X[:, 0].sum() == 0 and X[:, -1].sum() == k
    # Prop. 3: E[X] = p; 5 sigma band per variable
    mean = X.mean(axis=0)
    sd = np.sqrt(p * (1 - p) / k) + 1e-12
    assert np.all(np.abs(mean - p) <= 5 * sd + 2 ** -24)


def test_bernoulli_rule_on_explicit_lanes():
    p = np.array([0.25, 0.5, 0.75, 0.1, 0.9], np.float32)
    X = O.bernoulli(p, 3, 1234, 2, 9)
    for s in range(3):
        u = O.philox_lanes(1234, 0, 2, 9, s, p.size)
        t = np.floor(p.astype(np.float64) * 2 ** 24).astype(np.uint64)
        assert list(X[s]) == list(((u >> 8).astype(np.uint64) < t).astype(np.uint8))


def test_single_cover_row_probability():
    """P(row covered) = 1 - prod(1 - p_i) for a single covering row."""
    p = np.array([0.1, 0.2, 0.05, 0.3], np.float32)
    k = 20000
    X = O.bernoulli(p, k, 5, 0, 0)
    hit = (X.sum(axis=1) >= 1).mean()
    q = 1 - np.prod(1 - p.astype(np.float64))
    assert abs(hit - q) <= 5 * math.sqrt(q * (1 - q) / k)


def test_thm4_feasibility_bound():
    """Per-sample infeasibility <= m exp(-2 gamma_+^2 / eta^2) (Thm. 4)."""
    rng = np.random.default_rng(4)
    n, m = 200, 5
    A = (rng.random((m, n)) < 0.5).astype(float)
    p = np.full(n, 0.7, np.float32)
    b = np.floor(A @ p - 12)
    gamma = (A @ p - b).min()
    eta = np.linalg.norm(A, axis=1).max()
    bound = m * math.exp(-2 * gamma ** 2 / eta ** 2)
    X = O.bernoulli(p, 5000, 8, 0, 0)
    bad = ((X @ A.T) < b).any(axis=1).mean()
    assert bad <= bound + 5 * math.sqrt(bound / 5000)


def test_onehot_groups():
    n = 12
    groups = (np.array([0, 4, 9, 12]), np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11]))
    p = np.zeros(n, np.float32)
    p[0:4] = [0.1, 0.2, 0.3, 0.4]
    p[4:9] = [0.5, 0, 0, 0.25, 0.25]
    p[9:12] = 0                                    # W = 0 -> uniform
    k = 20000
    X = O.onehot(p, groups, k, 3, 0, 0)
    for g in range(3):
        sl = slice(groups[0][g], groups[0][g + 1])
        assert np.all(X[:, sl].sum(axis=1) == 1)
    f = X[:, 0:4].mean(axis=0)
    assert np.allclose(f, p[0:4] / p[0:4].sum(), atol=5 * math.sqrt(0.25 / k))
    assert X[:, 5].sum() == 0 and X[:, 6].sum() == 0
    assert np.allclose(X[:, 9:12].mean(axis=0), 1 / 3, atol=5 * math.sqrt(0.25 / k))


def test_axial3d_samples_are_feasible():
    inst = W.assign3d(I=6, idx=0)
    rng = np.random.default_rng(0)
    p = rng.random(inst.n).astype(np.float32)
    X = O.axial3d(p, 6, 50, 9, 0, 4)
    viol, obj = O.Evaluator(inst)(X)
    assert np.all(viol == 0)
    for s in range(50):
        v = np.flatnonzero(X[s])
        i, j, kk = v // 36, (v // 6) % 6, v % 6
        assert sorted(i) == list(range(6)) and sorted(j) == list(range(6)) \
            and sorted(kk) == list(range(6))
        assert obj[s] == inst.c[v].sum()


def test_facility_closure_makes_samples_feasible():
    inst = W.facility_location(nf=5, nc=9, idx=1)
    p = np.random.default_rng(1).random(inst.n).astype(np.float32)
    X = O.sample(inst, p, 40, 3, 0, 0)
    viol, obj = O.Evaluator(inst)(X)
    assert np.all(viol == 0)


# ---------------------------------------------------------------- evaluation
def test_maxcut_objective_is_minus_cut():
    inst = W.max_cut(n=40, idx=3)
    Wm = inst.meta["W"]
    rng = np.random.default_rng(2)
    X = (rng.random((30, 40)) < 0.5).astype(np.uint8)
    viol, obj = O.Evaluator(inst)(X)
    iu = np.triu_indices(40, 1)
    for s in range(30):
        cut = sum(Wm[i, j] for i, j in zip(*iu) if X[s, i] != X[s, j])
        assert obj[s] == -cut and viol[s] == 0


@pytest.mark.parametrize("form", ["csr_dense_graph", "sparse_graph"])
def test_maxcut_csr_objective_is_minus_cut(form):
    """The CSR (sparse-Q) objective path gives minus the cut weight, counted
    edge by edge, with the paper's weights U{-8..10} (negative weights and a
    diagonal that is not zero)."""
    if form == "csr_dense_graph":
        inst = W.max_cut(n=36, idx=4, weights="paper", sparse=True)
        Wm = np.asarray(inst.meta["W"], np.int64)
    else:
        inst = W.max_cut_sparse(n=60, avg_deg=6.0, idx=2)
        Wm = inst.meta["W"].toarray().astype(np.int64)
    n = inst.n
    rng = np.random.default_rng(7)
    X = (rng.random((25, n)) < 0.5).astype(np.uint8)
    viol, obj = O.Evaluator(inst)(X)
    iu, ju = np.nonzero(np.triu(Wm, 1))
    assert len(iu) > 0 and (Wm[iu, ju] < 0).any()
    for s in range(25):
        cut = sum(int(Wm[i, j]) for i, j in zip(iu, ju) if X[s, i] != X[s, j])
        assert obj[s] == -cut and viol[s] == 0


def test_eval_setcover_and_knapsack_semantics():
    inst = W.set_cover(n=50, m=10, density=0.2, idx=5)
    rng = np.random.default_rng(3)
    X = (rng.random((40, 50)) < 0.2).astype(np.uint8)
    viol, obj = O.Evaluator(inst)(X)
    A = inst.A.toarray().astype(bool)
    for s in range(40):
        chosen = set(np.flatnonzero(X[s]))
        uncovered = sum(1 for j in range(10) if not (set(np.flatnonzero(A[j])) & chosen))
        assert viol[s] == uncovered
        assert obj[s] == sum(inst.c[i] for i in chosen)
    kn = W.knapsack(30, idx=1)
    X = (rng.random((40, 30)) < 0.5).astype(np.uint8)
    viol, obj = O.Evaluator(kn)(X)
    for s in range(40):
        wsum = sum(kn.meta["w"][i] for i in np.flatnonzero(X[s]))
        assert viol[s] == (1 if wsum > kn.meta["cap"] else 0)
        assert obj[s] == -sum(kn.meta["p"][i] for i in np.flatnonzero(X[s]))


def _knapsack_dp(w, p, cap):
    w = w.astype(int)
    best = np.zeros(int(cap) + 1)
    for i in range(w.size):
        best[w[i]:] = np.maximum(best[w[i]:], best[:best.size - w[i]] + p[i])
    return best.max()


def test_brute_force_matches_knapsack_dp():
    for idx in range(3):
        kn = W.knapsack(14, idx=20 + idx)
        found, best, bx, nf = O.Evaluator(kn).brute_force()
        assert found
        assert -best == _knapsack_dp(kn.meta["w"], kn.meta["p"], kn.meta["cap"])


def test_incumbent_rule():
    st = dict(found=0, obj=0, round=0, sample=-1)
    viol = np.array([1, 0, 0, 0], np.int32)
    obj = np.array([-100, 5, 3, 3], np.int64)
    assert O.incumbent_update(st, viol, obj, 0) == 2       # earliest of the tie
    assert st["obj"] == 3 and st["sample"] == 2
    assert O.incumbent_update(st, viol, obj, 1) == -1      # equal: not replaced
    assert st["round"] == 0
    obj2 = np.array([0, 2, 9, 9], np.int64)
    assert O.incumbent_update(st, viol, obj2, 2) == 1 and st["obj"] == 2


def test_oracle_run_never_beats_brute_force():
    for idx in range(3):
        inst = W.tiny_bip(n=12, m1=3, m2=1, idx=30 + idx)
        found, best, bx, nf = O.Evaluator(inst).brute_force()
        P = O.Params(k_int=10, k_b=256, seed=100 + idx, x0=0.5)
        sol = O.OracleSolver(inst, P)
        inc = sol.run(400)
        if inc["found"]:
            assert found and inc["obj"] >= best
            v, o = O.Evaluator(inst)(sol.best_x[None, :])
            assert v[0] == 0 and o[0] == inc["obj"]


# ---------------------------------------------------------------- MLP
def _mlp_weights(F=8, H=16, seed=0):
    rng = np.random.default_rng(seed)
    return dict(W1=(rng.standard_normal((H, F)) * 0.4).astype(np.float32),
                b1=(rng.standard_normal(H) * 0.1).astype(np.float32),
                W2=(rng.standard_normal((H, H)) * 0.3).astype(np.float32),
                b2=(rng.standard_normal(H) * 0.1).astype(np.float32),
                w3=(rng.standard_normal(H) * 0.3).astype(np.float32),
                b3=np.array([0.05], np.float32))


def test_bf16_rounding_matches_torch():
    import torch
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(500).astype(np.float32),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -0.0, 65504.0,
                                  1e-40, 3.3895e38], np.float32)])
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    got = O.bf16_round(a)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_mlp_forward_matches_torch_and_grad_matches_fd():
    import torch
    Wt = _mlp_weights()
    rng = np.random.default_rng(1)
    f = rng.standard_normal((37, 8)).astype(np.float32)
    y = (rng.random(37) < 0.4).astype(np.float32)
    z, p = O.mlp_forward(f, Wt, rb=1)
    T = {k: torch.from_numpy(v).double() for k, v in Wt.items()}
    Tb = {k: torch.from_numpy(v).to(torch.bfloat16).double() for k, v in Wt.items()}
    ft = torch.from_numpy(f).double()
    h1 = torch.relu(ft @ Tb["W1"].T + T["b1"])
    h2 = torch.relu(h1 @ Tb["W2"].T + T["b2"])
    zt = h2 @ Tb["w3"] + T["b3"]
    assert np.allclose(z, zt.numpy(), rtol=1e-12, atol=1e-12)
    assert np.allclose(p, np.clip(torch.sigmoid(zt).numpy(), 1e-4, 1 - 1e-4), rtol=1e-12)
    # analytic gradient vs central differences (no rounding -> smooth)
    loss, g = O.mlp_loss_grad(f, y, Wt, rb=0)
    h = 1e-4
    for key in ("W1", "b1", "W2", "w3", "b3"):
        flat = Wt[key].reshape(-1)
        for idx in list(range(min(flat.size, 6))):
            Wp = {k: v.copy() for k, v in Wt.items()}
            Wm = {k: v.copy() for k, v in Wt.items()}
            Wp[key].reshape(-1)[idx] += h
            Wm[key].reshape(-1)[idx] -= h
            dp = (Wp[key].reshape(-1)[idx] - Wm[key].reshape(-1)[idx])
            lp, _ = O.mlp_loss_grad(f, y, Wp, rb=0)
            lm, _ = O.mlp_loss_grad(f, y, Wm, rb=0)
            fd = (lp - lm) / float(dp)
            assert abs(fd - g[key].reshape(-1)[idx]) < 1e-6 + 1e-4 * abs(fd)
    # loss vs torch BCE-with-logits
    zt0, _ = O.mlp_forward(f, Wt, rb=0)
    bce = torch.nn.functional.binary_cross_entropy_with_logits(
        torch.from_numpy(zt0), torch.from_numpy(y).double())
    assert abs(loss - bce.item()) < 1e-12


def test_adam_matches_torch():
    import torch
    rng = np.random.default_rng(2)
    w = rng.standard_normal(20).astype(np.float32)
    wt = torch.nn.Parameter(torch.from_numpy(w.astype(np.float64)))
    opt = torch.optim.Adam([wt], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(20)
    v = np.zeros(20)
    for t in range(1, 6):
        g = rng.standard_normal(20)
        O.adam(w, g, m, v, t, lr=1e-2)
        opt.zero_grad()
        wt.grad = torch.from_numpy(g)
        opt.step()
    assert np.allclose(w, wt.detach().numpy(), rtol=1e-6, atol=1e-7)


# ---------------------------------------------------------------- Algorithm 4
def _assign_of(X, I):
    """(i, j, k) triples of one candidate; None unless a 3D assignment."""
    t = np.argwhere(X.reshape(I, I, I))
    if len(t) != I or len(set(t[:, 0])) != I or len(set(t[:, 1])) != I or \
            len(set(t[:, 2])) != I:
        return None
    return t


def _cost3(t, C):
    return int(sum(C[i, j, k] for i, j, k in t))


def test_alg4_candidates_are_assignments_and_locally_optimal():
    """Every candidate of Algorithm 4 is a 3D assignment; with enough steps
    no pairwise interchange (swap of j or of k between two triples) improves
    it -- checked by enumerating all interchanges here."""
    I = 7
    rng = np.random.default_rng(3)
    p = (rng.random(I ** 3) ** 4).astype(np.float32)
    C = rng.integers(1, 101, size=(I, I, I)).astype(np.int64)
    X = O.assign3d_custom(p, C.ravel(), I, 1, I * I, 40, 11, 0, 2)
    for s in range(40):
        t = _assign_of(X[s], I)
        assert t is not None
        base = _cost3(t, C)
        for a in range(I):
            for b in range(a + 1, I):
                for ax in (1, 2):
                    u = t.copy()
                    u[a, ax], u[b, ax] = t[b, ax], t[a, ax]
                    assert _cost3(u, C) >= base


def test_alg4_partial_assignment_from_top_entries():
    """p concentrated on one assignment (plus noise below it): the top I
    entries are exactly that assignment, the greedy partial assignment is
    complete, and with L = 0 every candidate equals it."""
    I = 6
    rng = np.random.default_rng(4)
    sj, sk = rng.permutation(I), rng.permutation(I)
    p = (0.5 * rng.random(I ** 3)).astype(np.float32)
    target = np.zeros(I ** 3, np.uint8)
    for i in range(I):
        v = (i * I + sj[i]) * I + sk[i]
        p[v] = 0.9
        target[v] = 1
    C = rng.integers(1, 50, size=I ** 3).astype(np.int64)
    X = O.assign3d_custom(p, C, I, 1, 0, 16, 5, 0, 0)
    assert np.all(X == target[None, :])


def test_alg4_random_completion_is_uniform():
    """gamma = 0 (empty partial assignment) and L = 0: the completion pairs
    the i's with two independent uniform permutations, so all (I!)^2 = 36
    assignments of I = 3 appear equally often (chi-square, 36 cells)."""
    I, k = 3, 7200
    p = np.zeros(I ** 3, np.float32)
    C = np.ones(I ** 3, np.int64)
    X = O.assign3d_custom(p, C, I, 0, 0, k, 21, 0, 1)
    counts = {}
    for s in range(k):
        t = _assign_of(X[s], I)
        assert t is not None
        key = tuple(t[:, 1]) + tuple(t[:, 2])
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 36
    e = k / 36
    chi2 = sum((c - e) ** 2 / e for c in counts.values())
    assert chi2 < 80.0                      # 35 dof: p ~ 1e-5 above this


def test_alg4_improvement_never_worsens_and_bounds_optimum():
    """Same candidates with L = 0 and L = 12 (identical completions): the
    improved cost is never higher, and never below the optimum found by
    enumerating all (I!)^2 assignments of I = 4."""
    import itertools
    I = 4
    rng = np.random.default_rng(8)
    p = (rng.random(I ** 3) ** 3).astype(np.float32)
    C = rng.integers(1, 101, size=(I, I, I)).astype(np.int64)
    X0 = O.assign3d_custom(p, C.ravel(), I, 1, 0, 50, 9, 3, 7)
    X1 = O.assign3d_custom(p, C.ravel(), I, 1, 12, 50, 9, 3, 7)
    opt = min(sum(C[i, a[i], b[i]] for i in range(I))
              for a in itertools.permutations(range(I))
              for b in itertools.permutations(range(I)))
    for s in range(50):
        c0 = _cost3(_assign_of(X0[s], I), C)
        c1 = _cost3(_assign_of(X1[s], I), C)
        assert opt <= c1 <= c0


# ---------------------------------------------------------------- CheckHalt
@pytest.mark.parametrize("with_Q", [True, False])
def test_sx_is_thm2_primal_residual(with_Q):
    """||s^x_k|| of orc_halt_stats against Thm. 2's definition, with the two
    gradients of L_hat (Eq. 2) taken by central differences of the scalar
    Lagrangian: s^x = (x_{k-1} - x_k)/tau1 + grad_x L(x_k, y_k) -
    grad_x L(x_{k-1}, y_k).  With Q != 0 the Gap indicator is ||s^x||."""
    inst = W.tiny_bip(n=12, m1=4, m2=1, idx=17, with_Q=with_Q)
    S = O.preprocess(inst, 3)
    assert (S.qkind != 0) == with_Q
    rng = np.random.default_rng(4)
    xp = rng.random(S.n)
    xb = rng.random(S.n)
    y = rng.random(S.m)
    rho, t1, t2 = 0.29, 0.13, 0.4
    x, _, y1, _ = O.pdhg_step(S, t1, t2, rho, xp, xb, y)
    h = 1e-6

    def grad(z):
        g = np.zeros(S.n)
        for i in range(S.n):
            e = np.zeros(S.n)
            e[i] = h
            g[i] = (_lagrangian(S, rho, z + e, y1) - _lagrangian(S, rho, z - e, y1)) / (2 * h)
        return g

    sx = (xp - x) / t1 + grad(x) - grad(xp)
    hs = O.halt_stats(S, t1, rho, x, xp, y1)
    assert np.linalg.norm(x - xp) > 0.1
    assert abs(hs[5] - np.linalg.norm(sx)) <= 1e-6 * np.linalg.norm(sx)
    if with_Q:
        assert hs[1] == hs[5] and math.isnan(hs[4])


def test_halt_tracker_stall_rule():
    """The value-stalling half of CheckHalt on a hand-built sequence: an
    indicator is done when <= tol, or when its best value has not improved
    by more than 1e-3 (relative) for `window` triggers.  Expected decisions
    worked out by hand from that rule."""
    hT = O.HaltTracker(1e-4, 3)
    seq = [(1.0, 5e-5, 0.5),       # t=1: every best set; ind1 <= tol
           (0.9, 5e-5, 0.4996),    # t=2: ind0 improves; ind2 by 0.08% only
           (0.9, 1e-3, 0.4996),    # t=3: ind1 above tol, last improved t=1
           (0.9, 1e-3, 0.4996),    # t=4: ind1, ind2 stalled 3 triggers; ind0 2
           (0.9, 1e-3, 0.4996)]    # t=5: ind0 stalled 3 triggers -> halt
    got = [hT.update(v) for v in seq]
    assert got == [False, False, False, False, True]
    # improvement is measured against the best value so far: 0.2% per
    # trigger resets every trigger, 0.05% every third (0.9995^3 < 0.999), so
    # neither stalls with window 5; 0.01% needs 11 triggers, so the
    # indicators stall at t = 6, five triggers after the best set at t = 1
    for rate, halt_at in ((0.998, None), (0.9995, None), (0.9999, 5)):
        hT = O.HaltTracker(1e-12, 5)
        halted = [hT.update((rate ** t, rate ** t, rate ** t)) for t in range(1, 40)]
        assert (halted.index(True) if any(halted) else None) == halt_at


# ---------------------------------------------------------------- sampling
def test_axial3d_pick_frequencies():
    """Axial 3D picks at I = 3 against the categorical rule: step i = 0 picks
    (j, k) with probability w_0jk / sum w_0 (w = floor(p 2^24)); given that
    pick, step i = 1 picks among the pairs with unused j and k with
    probability proportional to w_1jk; step i = 2 is forced."""
    I, k = 3, 40000
    rng = np.random.default_rng(8)
    p = (0.05 + rng.random(I ** 3)).astype(np.float32)
    w = np.floor(p.astype(np.float64) * 2.0 ** 24).reshape(I, I, I)
    X = O.axial3d(p, I, k, 77, 1, 2).reshape(k, I, I, I)
    first = X[:, 0].reshape(k, I * I)
    f0 = first.mean(axis=0)
    want0 = (w[0] / w[0].sum()).reshape(-1)
    assert np.all(np.abs(f0 - want0) <= 5 * np.sqrt(want0 * (1 - want0) / k))
    j0, k0 = np.unravel_index(np.argmax(want0), (I, I))
    sel = X[first[:, j0 * I + k0] == 1]
    ks = sel.shape[0]
    free = [(j, kk) for j in range(I) for kk in range(I) if j != j0 and kk != k0]
    wf = np.array([w[1, j, kk] for j, kk in free])
    for (j, kk), q in zip(free, wf / wf.sum()):
        f = sel[:, 1, j, kk].mean()
        assert abs(f - q) <= 5 * math.sqrt(q * (1 - q) / ks)
    # every sample is an axial assignment, so step 2 takes the last pair
    assert np.all(X.sum(axis=(2, 3)) == 1) and np.all(X.sum(axis=(1, 3)) == 1)


def test_random_start_vector_from_philox_stream5():
    """x0 < 0: x_0,i = (u_i >> 8) 2^-24 with u_i lane i & 3 of
    Philox4x32-10(counter = (i >> 2, 0, 0, inst | 5 << 28), key = seed),
    built here from explicit generator calls (the generator itself is pinned
    by its published known-answer vectors)."""
    seed, inst_id, n = 0x0123456789ABCDEF, 3, 11
    x0 = O.x0_vector(n, -1.0, seed, inst_id)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    want = np.zeros(n)
    for i in range(n):
        u = O.philox4x32_10([i >> 2, 0, 0, inst_id | (5 << 28)], key)[i & 3]
        want[i] = (int(u) >> 8) * 2.0 ** -24
    assert np.array_equal(x0, want)
    assert np.all((x0 >= 0) & (x0 < 1))
    assert np.all(O.x0_vector(5, 0.25, seed, inst_id) == 0.25)


def test_fp64_evaluator_on_fractional_data():
    """The FP64 evaluator (non-integral data): objective = c^T x + x^T Q x
    (checked against a brute-force sum for every point of {0,1}^8), and a
    row is violated only when it misses its right-hand side by more than
    1e-9 (1 + |rhs|)."""
    n = 8
    rng = np.random.default_rng(6)
    A = sp.csr_matrix(np.array([[0.5, 0.25, 0, 0, 0, 0, 0, 1.0],
                                [0, 0, 1.0, 1.0, 0, 0, 0, 0]]))
    Qd = rng.integers(-3, 4, size=(n, n)).astype(np.float64) * 0.5
    c = rng.random(n) - 0.5
    codes = np.arange(1 << n)
    X = ((codes[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    for eps, kind in ((0.0, "exact"), (0.5e-9, "inside"), (2e-9, "outside")):
        b = np.array([0.75 + eps * 1.75, 1.0])
        inst = W.Instance("frac", n, c, A=A, b=b, Q=Qd)
        ev = O.Evaluator(inst)
        assert not ev.integral
        viol, obj = ev(X)
        xf = X.astype(np.float64)
        assert np.allclose(obj, xf @ c + np.einsum("si,ij,sj->s", xf, Qd, xf), rtol=0,
                           atol=1e-12)
        ax = xf @ A.toarray().T
        want = (ax[:, 0] < 0.75 - 1e-12).astype(int) + (ax[:, 1] < 1.0).astype(int)
        hit = np.isclose(ax[:, 0], 0.75)          # rows exactly at the old rhs
        if kind == "outside":
            want = want + hit
        assert np.array_equal(viol, want)


# ---------------------------------------------------------------- multi-core build
def test_openmp_build_gives_identical_results():
    """The multi-core oracle build (OpenMP over rows and samples, used only
    for the CPU baseline's timing) returns exactly what the single-thread
    reference build returns: PDHG steps, Bernoulli and one-hot sampling,
    closure, repair and evaluation."""
    insts = [W.set_cover(n=300, m=40, density=0.08, idx=2), W.max_cut(n=120, idx=3),
             W.facility_location(nf=7, nc=30, idx=1),
             W.facility_location(nf=9, nc=11, idx=2, relaxed=True)]
    outs = []
    for on in (False, True):
        O.use_threads(on)
        res = []
        for inst in insts:
            S = O.preprocess(inst, 5)
            rng = np.random.default_rng(1)
            x = rng.random(S.n)
            y = rng.random(S.m)
            t1, t2 = O.step_sizes(0.99, S.normQ, 0.1, S.qkind != 0)
            res.append(O.pdhg_step(S, t1, t2, 0.1, x, x, y))
            X = O.sample(inst, x.astype(np.float32), 96, 7, 0, 3)
            res.append((X,) + O.Evaluator(inst)(X))
        outs.append(res)
    O.use_threads(False)
    for a, b in zip(*outs):
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
