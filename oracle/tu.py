"""TU reformulation of Thm. 5 (Section 2.4.1) in exact arithmetic.

TEST INFRASTRUCTURE ONLY: imported by tests/ and nothing else.  It shares no
code with the CUDA library's host transform.

Given row and column index sets J (rows of B) and I (|J| columns) with B_J
integral and totally unimodular and B_JI invertible, the equalities of J are
removed by substituting  x_I = s + S x_Ibar,  s = B_JI^-1 d_J,
S = -B_JI^-1 B_JIbar,  which is exact for binary x_Ibar once the bounds
0 <= s + S x_Ibar <= 1 are added as constraints (Thm. 5).  The new data, in
the order the theorem defines them:

    Q'  = S^T Q_II S + S^T Q_IIbar + Q_IbarI S + Q_IbarIbar
    A'  = A_.I S + A_.Ibar,            b' = b - A_.I s
    B'  = B_JbarI S + B_JbarIbar,      d' = d_Jbar - B_JbarI s
    c'  = S^T (Q_II + Q_II^T) s + Q_IIbar^T s + Q_IbarI s + S^T c_I + c_Ibar
    c0' = s^T Q_II s + c_I^T s
    S x >= -s,   -S x >= s - 1          (x_I within [0, 1]; a bounds row
                                         that every x in [0, 1] satisfies is
                                         left out)

Q is used as given (not symmetrised), so integral data stay integral; for a
symmetric Q the linear terms reduce to the theorem's 2 S^T Q_II s + 2 Q_IIbar^T s.
B_JI^-1 is computed densely with numpy and rounded (it is integral because
B_J is TU); the rounding is verified exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from paper_2510_27117_b300.workloads import Instance


def _dense(M, shape):
    if M is None:
        return np.zeros(shape)
    return M.toarray() if sp.issparse(M) else np.asarray(M, np.float64)


def tu_reformulate(inst, J, I):
    """Returns (reformulated Instance over x_Ibar, info for tu_recover)."""
    n = inst.n
    J = np.asarray(J, np.int64)
    I = np.asarray(I, np.int64)
    assert J.size == I.size and J.size > 0
    Ibar = np.setdiff1d(np.arange(n), I)
    m2 = inst.m2
    Jbar = np.setdiff1d(np.arange(m2), J)
    B = _dense(inst.B, (m2, n))
    d = np.asarray(inst.d, np.float64)
    BJI = B[np.ix_(J, I)]
    inv = np.rint(np.linalg.inv(BJI))
    assert np.array_equal(BJI @ inv, np.eye(J.size)), "B_JI^-1 not integral"
    s = inv @ d[J]
    S = -inv @ B[np.ix_(J, Ibar)]
    # quadratic and linear terms
    Q = _dense(inst.Q, (n, n)) if inst.Q is not None else None
    c = np.asarray(inst.c, np.float64)
    c_new = S.T @ c[I] + c[Ibar]
    c0 = float(c[I] @ s)
    Q_new = None
    if Q is not None:
        QII = Q[np.ix_(I, I)]
        QIIb = Q[np.ix_(I, Ibar)]
        QIbI = Q[np.ix_(Ibar, I)]
        QIbIb = Q[np.ix_(Ibar, Ibar)]
        Q_new = S.T @ QII @ S + S.T @ QIIb + QIbI @ S + QIbIb
        c_new = c_new + S.T @ (QII + QII.T) @ s + QIIb.T @ s + QIbI @ s
        c0 += float(s @ QII @ s)
    # inequalities: A' x >= b', then the bounds of x_I
    rowsA, rhsA = [], []
    if inst.A is not None and inst.m1:
        A = _dense(inst.A, (inst.m1, n))
        rowsA.append(A[:, I] @ S + A[:, Ibar])
        rhsA.append(np.asarray(inst.b, np.float64) - A[:, I] @ s)
    # bounds rows of x_I, except those every x in [0, 1] satisfies (the
    # row's minimum over the box, sum of its negative coefficients, is at
    # least its right-hand side)
    for M, r in ((S, -s), (-S, s - 1.0)):
        keep = np.minimum(M, 0.0).sum(axis=1) < r
        rowsA.append(M[keep])
        rhsA.append(r[keep])
    A_new = np.vstack(rowsA)
    b_new = np.concatenate(rhsA)
    B_new = d_new = None
    if Jbar.size:
        B_new = B[np.ix_(Jbar, I)] @ S + B[np.ix_(Jbar, Ibar)]
        d_new = d[Jbar] - B[np.ix_(Jbar, I)] @ s
    out = Instance(inst.name + "_tu", int(Ibar.size), c_new,
                   A=sp.csr_matrix(A_new), b=b_new,
                   B=None if B_new is None else sp.csr_matrix(B_new), d=d_new,
                   Q=None if Q_new is None else Q_new)
    info = dict(I=I, Ibar=Ibar, s=s, S=S, c0=c0, n=n)
    return out, info


def tu_recover(info, Xbar):
    """Original candidates (k x n) from reformulated ones (k x |Ibar|)."""
    Xbar = np.asarray(Xbar)
    k = Xbar.shape[0]
    X = np.zeros((k, info["n"]), np.int64)
    X[:, info["Ibar"]] = Xbar
    X[:, info["I"]] = np.rint(info["s"][None, :] + Xbar.astype(np.float64) @ info["S"].T)
    return X
