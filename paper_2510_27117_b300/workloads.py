"""Seeded synthetic instances of the binary integer program of Eq. (1).

    min  x^T Q x + c^T x   s.t.  A x >= b,  B x = d,  x in {0,1}^n

This module only builds problem data (numpy / scipy.sparse); it holds none of
the solver's arithmetic, so both the CPU oracle and the CUDA path take their
inputs from here.  Every generator is a pure function of its seed (numpy
PCG64).  Shapes follow the five problem classes of Section 4 (set cover,
knapsack, max cut, 3D assignment, facility location); the paper's own
instance generators and seeds are not published, so these are stand-ins with
the stated sizes and distributions.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np
import scipy.sparse as sp

# Seed base per workload family (seed = 1000 * family + instance index).
SC, MC, KN, A3D, FL = 0, 1, 2, 3, 4


@dataclass
class Instance:
    """One BIP in the form of Eq. (1).

    A, B are CSR (float64 values, integral for every generator here); Q is
    None, a dense float64 (n x n) array or a CSR matrix.  ``groups`` lists
    disjoint one-hot groups (each group's variables sum to one in every
    feasible point) as (grp_ptr, grp_idx); ``axial_I`` > 0 marks an axial 3D
    assignment over I^3 variables x_ijk at index (i*I + j)*I + k;
    ``closure`` = (rep_var, rep_ptr, rep_idx) lists monotone repairs
    y <- y OR x_k for k in the list (the facility-location closure);
    ``repair`` = (grp_ptr, grp_idx) lists equality groups relaxed to
    "sum >= 1" whose candidates keep only their least-cost selected member.
    ``repair_rows`` = (row_ptr, row_idx) lists 0/1 equality rows relaxed to
    "sum >= 1" (possibly overlapping) whose candidates are reduced to minimal
    covers by reverse delete in decreasing cost.
    """

    name: str
    n: int
    c: np.ndarray
    A: Optional[sp.csr_matrix] = None
    b: Optional[np.ndarray] = None
    B: Optional[sp.csr_matrix] = None
    d: Optional[np.ndarray] = None
    Q: object = None
    groups: Optional[Tuple[np.ndarray, np.ndarray]] = None
    axial_I: int = 0
    closure: Optional[Tuple[np.ndarray, np.ndarray, np.ndarray]] = None
    repair: Optional[Tuple[np.ndarray, np.ndarray]] = None
    repair_rows: Optional[Tuple[np.ndarray, np.ndarray]] = None
    meta: dict = field(default_factory=dict)

    @property
    def m1(self) -> int:
        return 0 if self.A is None else self.A.shape[0]

    @property
    def m2(self) -> int:
        return 0 if self.B is None else self.B.shape[0]

    def nnz(self) -> int:
        t = 0
        for M in (self.A, self.B):
            if M is not None:
                t += M.nnz
        if isinstance(self.Q, np.ndarray):
            t += int(np.count_nonzero(self.Q))
        elif self.Q is not None:
            t += self.Q.nnz
        return t


def _rng(family: int, idx: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * family + idx))


def _csr(rows, cols, vals, shape) -> sp.csr_matrix:
    M = sp.csr_matrix((np.asarray(vals, np.float64),
                       (np.asarray(rows, np.int64), np.asarray(cols, np.int64))),
                      shape=shape)
    M.sum_duplicates()
    M.sort_indices()
    return M


# --------------------------------------------------------------------------
# Set cover (Section 4.2.1): min c^T x, sum_{i in S_j} x_i >= 1.
# --------------------------------------------------------------------------
def set_cover(n: int = 2000, m: int = 200, density: float = 0.05,
              idx: int = 0, family: int = SC) -> Instance:
    rng = _rng(family, idx)
    mask = rng.random((m, n)) < density
    for j in range(m):
        have = np.flatnonzero(mask[j])
        if have.size < 2:
            free = np.setdiff1d(np.arange(n), have)
            add = rng.choice(free, size=2 - have.size, replace=False)
            mask[j, add] = True
    r, cidx = np.nonzero(mask)
    A = _csr(r, cidx, np.ones(r.size), (m, n))
    c = rng.integers(1, 101, size=n).astype(np.float64)
    return Instance(f"setcover_n{n}_m{m}_s{idx}", n, c, A=A, b=np.ones(m))


# --------------------------------------------------------------------------
# Max cut, QP form (Section 4.2.3) with Q = -L, so x^T Q x = -cut(x).
# --------------------------------------------------------------------------
def max_cut(n: int = 4096, p: float = 0.5, idx: int = 0,
            family: int = MC, weights: str = "pm1", sparse: bool = False) -> Instance:
    """Erdos-Renyi G(n,p); weights +-1 equiprobable ('pm1') or integers
    uniform on [-8, 10] ('int8_10', the paper's range).  Q = W - diag(W 1);
    sparse=True hands Q over as CSR (the sparse-Q path) instead of dense."""
    rng = _rng(family, idx)
    iu = np.triu_indices(n, 1)
    edge = rng.random(iu[0].size) < p
    if weights == "pm1":
        w = np.where(rng.random(iu[0].size) < 0.5, -1.0, 1.0)
    else:
        w = rng.integers(-8, 11, size=iu[0].size).astype(np.float64)
    w = np.where(edge, w, 0.0)
    W = np.zeros((n, n), np.float64)
    W[iu] = w
    W += W.T
    Q = W - np.diag(W.sum(axis=1))
    if sparse:
        Q = sp.csr_matrix(Q)
    inst = Instance(f"maxcut_n{n}_s{idx}" + ("_csr" if sparse else ""), n, np.zeros(n), Q=Q)
    inst.meta["W"] = W
    return inst


def max_cut_sparse(n: int = 65536, avg_deg: float = 32.0, idx: int = 0,
                   family: int = MC, weights: str = "int8_10") -> Instance:
    """Sparse random graph for the sparse-Q path: n * avg_deg / 2 edges drawn
    as uniform pairs i < j (duplicates dropped, zero weights dropped), weights
    as in max_cut.  Q = W - diag(W 1) as CSR; meta["W"] holds W (CSR)."""
    rng = _rng(family, 500 + idx)
    m = int(n * avg_deg / 2)
    i = rng.integers(0, n, size=m)
    j = rng.integers(0, n, size=m)
    keep = i != j
    lo, hi = np.minimum(i, j)[keep], np.maximum(i, j)[keep]
    key = np.unique(lo.astype(np.int64) * n + hi)
    lo, hi = key // n, key % n
    if weights == "pm1":
        w = np.where(rng.random(key.size) < 0.5, -1.0, 1.0)
    else:
        w = rng.integers(-8, 11, size=key.size).astype(np.float64)
    nz = w != 0
    lo, hi, w = lo[nz], hi[nz], w[nz]
    W = sp.csr_matrix((np.concatenate([w, w]), (np.concatenate([lo, hi]),
                                                  np.concatenate([hi, lo]))), shape=(n, n))
    deg = np.asarray(W.sum(axis=1)).ravel()
    Q = (W - sp.diags(deg)).tocsr()
    Q.sum_duplicates()
    Q.sort_indices()
    inst = Instance(f"maxcut_sparse_n{n}_s{idx}", n, np.zeros(n), Q=Q)
    inst.meta["W"] = W
    return inst


# --------------------------------------------------------------------------
# 0-1 knapsack (Section 4.2.2): max p^T x s.t. w^T x <= floor(sum w / 2),
# written as  min (-p)^T x  s.t.  -w^T x >= -cap.
# --------------------------------------------------------------------------
def knapsack(n: int, idx: int = 0, family: int = KN) -> Instance:
    rng = _rng(family, idx)
    w = rng.integers(1, 1001, size=n).astype(np.float64)
    prof = w + rng.integers(0, 101, size=n)
    cap = float(np.floor(0.5 * w.sum()))
    A = _csr(np.zeros(n, np.int64), np.arange(n), -w, (1, n))
    inst = Instance(f"knapsack_n{n}_s{idx}", n, -prof.astype(np.float64),
                    A=A, b=np.array([-cap]))
    inst.meta.update(w=w, p=prof.astype(np.float64), cap=cap)
    return inst


def knapsack_batch(ninst: int = 512, nmin: int = 1000, nmax: int = 100000,
                   idx: int = 0) -> list:
    """Uneven batch: n_i ~ U{nmin..nmax}, instance i seeded 1000*KN + idx*ninst + i."""
    sizes = _rng(KN, 999_000 + idx).integers(nmin, nmax + 1, size=ninst)
    return [knapsack(int(sizes[i]), idx=idx * ninst + i) for i in range(ninst)]


# --------------------------------------------------------------------------
# Axial 3D assignment (Eq. assign3d, Section 2.4.2).
# --------------------------------------------------------------------------
def assign3d(I: int = 64, idx: int = 0, family: int = A3D, sampler: str = "axial",
             gamma: int = 1, L: Optional[int] = None) -> Instance:
    """Axial 3D assignment; sampler 'axial' (one (j,k) per i by p), 'alg4'
    (the paper's customized sampler with gamma*I entries and L steps) or
    'relaxed' (the monotone relaxation of Section 2.4.3: costs are positive,
    so the 3I equality rows become covering rows sum >= 1 of A, candidates
    are plain Bernoulli draws reduced to minimal covers by reverse delete)."""
    rng = _rng(family, idx)
    n = I ** 3
    c = rng.integers(1, 101, size=n).astype(np.float64)
    v = np.arange(n, dtype=np.int64)
    i, j, k = v // (I * I), (v // I) % I, v % I
    rows = np.concatenate([i, I + j, 2 * I + k])
    cols = np.concatenate([v, v, v])
    B = _csr(rows, cols, np.ones(3 * n), (3 * I, n))
    grp_ptr = np.arange(0, n + 1, I * I, dtype=np.int64)      # rows "per i"
    grp_idx = v.copy()
    if sampler == "relaxed":
        inst = Instance(f"assign3d_rel_I{I}_s{idx}", n, c, A=B, b=np.ones(3 * I),
                        repair_rows=(B.indptr.astype(np.int64), B.indices.astype(np.int64)))
        inst.meta.update(sampler="relaxed")
        return inst
    inst = Instance(f"assign3d_I{I}_s{idx}", n, c, B=B, d=np.ones(3 * I),
                    groups=(grp_ptr, grp_idx), axial_I=I)
    if sampler == "alg4":
        inst.meta.update(sampler="alg4", gamma=gamma, L=I if L is None else L)
    return inst


# --------------------------------------------------------------------------
# Uncapacitated facility location (Section 4.2.5).
# Variables: y_i (open facility i) at index i, x_ij (customer j served by i)
# at index nf + j*nf + i.  Rows: sum_i x_ij = 1 (equalities), y_i - x_ij >= 0.
# --------------------------------------------------------------------------
def facility_location(nf: int = 1000, nc: int = 10000, idx: int = 0,
                      family: int = FL, relaxed: bool = False) -> Instance:
    """relaxed=True: the monotone relaxation of Section 2.4.3 (costs are
    nonnegative): the customer rows sum_i x_ij = 1 become sum_i x_ij >= 1
    (appended to A), candidates come from plain Bernoulli draws, and each
    customer's selected facilities are cut to the cheapest one by the repair
    groups before the closure."""
    rng = _rng(family, idx)
    fac = rng.random((nf, 2))
    cus = rng.random((nc, 2))
    f = rng.integers(500, 5001, size=nf).astype(np.float64)
    n = nf + nf * nc
    c = np.empty(n, np.float64)
    c[:nf] = f
    # x index nf + j*nf + i  -> row-major (j, i)
    dist = np.sqrt(((cus[:, None, :] - fac[None, :, :]) ** 2).sum(-1))  # nc x nf
    c[nf:] = np.round(1000.0 * dist).reshape(-1)
    xi = nf + np.arange(nf * nc, dtype=np.int64)
    jj = np.repeat(np.arange(nc, dtype=np.int64), nf)
    ii = np.tile(np.arange(nf, dtype=np.int64), nc)
    B = _csr(jj, xi, np.ones(nf * nc), (nc, n))
    m1 = nf * nc
    rid = np.arange(m1, dtype=np.int64)
    # A rows ordered like x: row r = j*nf + i : y_i - x_ij >= 0
    A_rowptr = np.arange(0, 2 * m1 + 1, 2, dtype=np.int64)
    A_cols = np.empty(2 * m1, np.int64)
    A_vals = np.empty(2 * m1, np.float64)
    A_cols[0::2] = ii
    A_cols[1::2] = xi
    A_vals[0::2] = 1.0
    A_vals[1::2] = -1.0
    A = sp.csr_matrix((A_vals, A_cols.astype(np.int32), A_rowptr), shape=(m1, n))
    del rid
    grp_ptr = np.arange(0, nf * nc + 1, nf, dtype=np.int64)
    grp_idx = xi.copy()
    rep_var = np.arange(nf, dtype=np.int64)
    rep_ptr = np.arange(0, nf * nc + 1, nc, dtype=np.int64)
    rep_idx = (nf + np.arange(nc, dtype=np.int64)[None, :] * nf
               + np.arange(nf, dtype=np.int64)[:, None]).reshape(-1)
    if relaxed:
        A = sp.vstack([A, B]).tocsr()
        inst = Instance(f"facloc_rel_nf{nf}_nc{nc}_s{idx}", n, c, A=A,
                        b=np.concatenate([np.zeros(m1), np.ones(nc)]),
                        repair=(grp_ptr, grp_idx), closure=(rep_var, rep_ptr, rep_idx))
    else:
        inst = Instance(f"facloc_nf{nf}_nc{nc}_s{idx}", n, c, A=A, b=np.zeros(m1),
                        B=B, d=np.ones(nc), groups=(grp_ptr, grp_idx),
                        closure=(rep_var, rep_ptr, rep_idx))
    inst.meta.update(nf=nf, nc=nc)
    return inst


# --------------------------------------------------------------------------
# Tiny random BIPs for brute force (n <= 20): mixed >= rows, one equality
# row, symmetric integer Q, integer c.
# --------------------------------------------------------------------------
def facility_tu_pivots(inst: Instance, nf: int, nc: int):
    """Row and column index sets (J, I) for the TU reformulation (Thm. 5) of
    a facility-location instance: every customer row sum_i x_ij = 1 with the
    customer's cheapest x_ij as its pivot (B_JI is the identity)."""
    cx = np.asarray(inst.c[nf:], np.float64).reshape(nc, nf)
    i0 = cx.argmin(axis=1)
    J = np.arange(nc, dtype=np.int64)
    I = nf + np.arange(nc, dtype=np.int64) * nf + i0
    return J, I


def tiny_bip(n: int = 12, m1: int = 4, m2: int = 1, idx: int = 0,
             with_Q: bool = True, family: int = 9) -> Instance:
    rng = _rng(family, idx)
    Ad = rng.integers(-3, 4, size=(m1, n)) * (rng.random((m1, n)) < 0.6)
    # rhs chosen so that roughly half the cube satisfies each row
    b = np.floor(0.5 * Ad.sum(axis=1)).astype(np.float64) - rng.integers(0, 2, size=m1)
    A = sp.csr_matrix(Ad.astype(np.float64)) if m1 else None
    B = d = None
    if m2:
        Bd = (rng.random((m2, n)) < 0.5).astype(np.float64)
        for r in range(m2):
            if Bd[r].sum() < 2:
                Bd[r, rng.choice(n, 2, replace=False)] = 1.0
        d = np.floor(0.5 * Bd.sum(axis=1))
        B = sp.csr_matrix(Bd)
    Q = None
    if with_Q:
        Qd = rng.integers(-4, 5, size=(n, n)) * (rng.random((n, n)) < 0.3)
        Qd = np.triu(Qd)
        Qd = Qd + np.triu(Qd, 1).T
        Q = sp.csr_matrix(Qd.astype(np.float64))
    c = rng.integers(-10, 11, size=n).astype(np.float64)
    return Instance(f"tiny_n{n}_s{idx}", n, c, A=A, b=(b if m1 else None),
                    B=B, d=d, Q=Q)
