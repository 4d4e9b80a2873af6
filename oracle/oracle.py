"""ctypes front end of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, the smoke check and the benchmark's CPU-baseline leg import this
module.  It loads oracle/liboracle.so (plain C, FP64, single thread; or,
after use_threads(True), the same source built with OpenMP over rows and
samples, which gives identical results) and strings its routines together in
the order of Alg. 1:

    Preprocess (Section 3) -> loop { UpdatePenalty; FirstOrderStep (Alg. 2);
    every k_int iterations k_r rounds of RandSampleStep (Alg. 3 or the
    customized samplers of Section 2.4.2) + EvalBest; CheckHalt }
    -> EvalBest(round(x_k))

Nothing here imports or calls the CUDA library.  Library primitives used as
steps: scipy.sparse for assembling K = -[A; B] and (Q + Q^T)/2.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.sparse as sp

from . import build as _build

_lib = None
_libs = {}

F64P = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
F32P = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
I32P = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
U32P = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
U8P = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
VP = C.c_void_p
i64, i32, u32, u64, f64 = C.c_int64, C.c_int32, C.c_uint32, C.c_uint64, C.c_double


def use_threads(on: bool) -> int:
    """Select the multi-core build (all host threads, identical results)
    or the single-thread reference build for later calls; returns the
    number of threads the selected build uses."""
    global _lib
    if (on, ) not in _libs:
        _libs[(on, )] = _load(_build.build(omp=on))
    _lib = _libs[(on, )]
    return int(_lib.orc_threads())


def lib():
    if _lib is None:
        use_threads(False)
    return _lib


def _load(path):
    L = C.CDLL(path)
    L.orc_threads.restype = i32
    L.orc_philox4x32_10.argtypes = [U32P, U32P, U32P]
    L.orc_philox_lane.argtypes = [u64, u32, u32, u32, u32, u64]
    L.orc_philox_lane.restype = u32
    L.orc_repair_min.argtypes = [i64, i64, I64P, I64P, I64P, i32, U8P]
    L.orc_repair_rows.argtypes = [i64, i64, I64P, I64P, I64P, i32, U8P]
    L.orc_bernoulli_from.argtypes = [i64, i32, i32, F32P, u64, u32, u32, VP, U8P]
    L.orc_philox_lanes.argtypes = [u64, u32, u32, u32, u32, i64, U32P]
    L.orc_row_normalize.argtypes = [i64, i64, I64P, F64P, F64P, F64P]
    L.orc_row_normalize.restype = i64
    L.orc_power_norm_K.argtypes = [i64, i64, I64P, I32P, F64P, u64, u32, f64, i32,
                                   C.POINTER(i32)]
    L.orc_power_norm_K.restype = f64
    L.orc_power_norm_Q.argtypes = [i32, i64, VP, VP, VP, VP, u64, u32, f64, i32,
                                   C.POINTER(i32)]
    L.orc_power_norm_Q.restype = f64
    L.orc_step_sizes.argtypes = [f64, f64, f64, i32, C.POINTER(f64), C.POINTER(f64)]
    L.orc_rho_update.argtypes = [i64, f64, f64, f64, f64, f64, f64]
    L.orc_rho_update.restype = f64
    L.orc_pdhg_step.argtypes = [i64, i64, i64, I64P, I32P, F64P, F64P, i32, VP, VP,
                                VP, VP, F64P, f64, f64, f64, F64P, F64P, F64P, F64P,
                                F64P, VP]
    L.orc_bernoulli.argtypes = [i64, i32, F32P, u64, u32, u32, VP, U8P]
    L.orc_onehot.argtypes = [i64, i64, I64P, I64P, i32, F32P, u64, u32, u32, U8P]
    L.orc_axial3d.argtypes = [i32, i32, F32P, u64, u32, u32, U8P]
    L.orc_assign3d_custom.argtypes = [i32, i32, i32, i32, F32P, I64P, u64, u32, u32,
                                      U8P]
    L.orc_closure.argtypes = [i64, i64, I64P, I64P, I64P, i32, U8P]
    L.orc_eval_int.argtypes = [i64, i64, I64P, I32P, I64P, I64P, i64, I64P, I32P, I64P,
                               I64P, i32, VP, VP, VP, VP, I64P, i32, U8P, I32P, I64P]
    L.orc_eval_f64.argtypes = [i64, i64, I64P, I32P, F64P, F64P, i64, I64P, I32P, F64P,
                               F64P, i32, VP, VP, VP, VP, F64P, i32, U8P, I32P, F64P]
    L.orc_incumbent_update.argtypes = [i32, I32P, I64P, u32, C.POINTER(i32),
                                       C.POINTER(i64), C.POINTER(u32), C.POINTER(i32)]
    L.orc_incumbent_update.restype = i32
    L.orc_round.argtypes = [i64, F64P, U8P]
    L.orc_halt_stats.argtypes = [i64, i64, i64, I64P, I32P, F64P, F64P, i32, VP, VP, VP,
                                 VP, F64P, f64, f64, F64P, F64P, F64P, F64P]
    L.orc_brute_force.argtypes = [i64, i64, I64P, I32P, I64P, I64P, i64, I64P, I32P,
                                  I64P, I64P, i32, VP, VP, VP, VP, I64P,
                                  C.POINTER(i64), U8P, C.POINTER(i64)]
    L.orc_brute_force.restype = i32
    L.orc_knapsack_lp.argtypes = [i64, F64P, F64P, f64, F64P]
    L.orc_knapsack_lp.restype = f64
    L.orc_bf16_round.argtypes = [C.c_float]
    L.orc_bf16_round.restype = C.c_float
    L.orc_mlp_forward.argtypes = [i64, i32, i32, F32P, F32P, F32P, F32P, F32P, F32P,
                                  F32P, i32, F64P, F64P, VP, VP]
    L.orc_mlp_loss_grad.argtypes = [i64, i32, i32, F32P, F32P, F32P, F32P, F32P, F32P,
                                    F32P, F32P, i32, F64P, F64P, F64P, F64P, F64P, F64P]
    L.orc_mlp_loss_grad.restype = f64
    L.orc_adam.argtypes = [i64, F32P, F64P, F64P, F64P, i64, f64, f64, f64, f64]
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# Philox and sampling
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def philox_lanes(seed, stream, inst, round_id, s, count):
    out = np.zeros(count, np.uint32)
    lib().orc_philox_lanes(seed, stream, inst, round_id, s, count, out)
    return out


def bernoulli(p32, k, seed, inst, round_id, mask=None, first=0):
    """Bernoulli draws of candidates first .. first+k-1 of a round (Alg. 3)."""
    p32 = np.ascontiguousarray(p32, np.float32)
    n = p32.size
    X = np.zeros((k, n), np.uint8)
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    lib().orc_bernoulli_from(n, first, k, p32, seed, inst, round_id, _ptr(m), X)
    return X


def onehot(p32, groups, k, seed, inst, round_id, X=None):
    p32 = np.ascontiguousarray(p32, np.float32)
    n = p32.size
    gp, gi = (np.ascontiguousarray(a, np.int64) for a in groups)
    if X is None:
        X = np.zeros((k, n), np.uint8)
    lib().orc_onehot(n, gp.size - 1, gp, gi, k, p32, seed, inst, round_id, X)
    return X


def axial3d(p32, I, k, seed, inst, round_id):
    p32 = np.ascontiguousarray(p32, np.float32)
    X = np.zeros((k, I ** 3), np.uint8)
    lib().orc_axial3d(I, k, p32, seed, inst, round_id, X)
    return X


def assign3d_custom(p32, cost, I, gamma, L, k, seed, inst, round_id):
    """Algorithm 4: top gamma*I entries, greedy partial assignment, random
    completion and L pairwise-interchange steps per candidate (readings in
    orc_assign3d_custom)."""
    p32 = np.ascontiguousarray(p32, np.float32)
    cost = np.ascontiguousarray(cost, np.int64)
    X = np.zeros((k, I ** 3), np.uint8)
    lib().orc_assign3d_custom(I, gamma, L, k, p32, cost, seed, inst, round_id, X)
    return X


def repair_min(X, groups, cost):
    """Monotone-relaxation repair: per relaxed group keep the selected member
    of least cost (ties to the first listed), clear the others."""
    gp, gi = (np.ascontiguousarray(a, np.int64) for a in groups)
    cost = np.ascontiguousarray(cost, np.int64)
    k, n = X.shape
    lib().orc_repair_min(n, gp.size - 1, gp, gi, cost, k, X)
    return X


def repair_rows(X, rows, cost):
    """General monotone-relaxation repair: each candidate drops its selected
    variables of the relaxed covering rows in decreasing cost (larger index
    first) whenever every such row keeps another selected member."""
    rp, ri = (np.ascontiguousarray(a, np.int64) for a in rows)
    cost = np.ascontiguousarray(cost, np.int64)
    k, n = X.shape
    lib().orc_repair_rows(n, rp.size - 1, rp, ri, cost, k, X)
    return X


def closure(X, clos):
    rv, rp, ri = (np.ascontiguousarray(a, np.int64) for a in clos)
    k, n = X.shape
    lib().orc_closure(n, rv.size, rv, rp, ri, k, X)
    return X


def sample(inst, p32, k, seed, inst_id, round_id, mode=None):
    """RandSampleStep for an Instance: Bernoulli for ungrouped variables,
    one-hot groups (mode 1) or axial 3D picks (mode 2), then closure."""
    if mode is None:
        mode = (3 if inst.meta.get("sampler") == "alg4" else 2) if inst.axial_I else \
            (1 if inst.groups is not None else 0)
    n = inst.n
    if mode == 3:
        I = inst.axial_I
        X = assign3d_custom(p32, np.asarray(inst.c, np.int64), I, inst.meta.get("gamma", 1),
                            inst.meta.get("L", I), k, seed, inst_id, round_id)
    elif mode == 2:
        X = axial3d(p32, inst.axial_I, k, seed, inst_id, round_id)
    else:
        mask = None
        if mode == 1 and inst.groups is not None:
            mask = np.zeros(n, np.uint8)
            mask[inst.groups[1]] = 1
        X = bernoulli(p32, k, seed, inst_id, round_id, mask)
        if mode == 1 and inst.groups is not None:
            onehot(p32, inst.groups, k, seed, inst_id, round_id, X)
    if inst.repair is not None:
        repair_min(X, inst.repair, np.asarray(inst.c, np.int64))
    if getattr(inst, "repair_rows", None) is not None:
        repair_rows(X, inst.repair_rows, np.asarray(inst.c, np.int64))
    if inst.closure is not None:
        closure(X, inst.closure)
    return X


# --------------------------------------------------------------------------
# Evaluation on the original data
# --------------------------------------------------------------------------
def _csr_parts(M, dtype):
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    return (np.ascontiguousarray(M.indptr, np.int64), np.ascontiguousarray(M.indices, np.int32),
            np.ascontiguousarray(M.data.astype(dtype)))


def _empty_csr(dtype):
    return (np.zeros(1, np.int64), np.zeros(1, np.int32), np.zeros(1, dtype))


def is_integral(inst) -> bool:
    arrs = [inst.c]
    for M in (inst.A, inst.B):
        if M is not None:
            arrs.append(M.data)
    for v in (inst.b, inst.d):
        if v is not None:
            arrs.append(v)
    if isinstance(inst.Q, np.ndarray):
        arrs.append(inst.Q.reshape(-1))
    elif inst.Q is not None:
        arrs.append(inst.Q.data)
    return all(np.all(np.floor(a) == a) and np.all(np.abs(a) < 2 ** 31) for a in arrs)


class Evaluator:
    """EvalBest's evaluation on the original data of an Instance."""

    def __init__(self, inst):
        self.inst = inst
        self.integral = is_integral(inst)
        dt = np.int64 if self.integral else np.float64
        self.dt = dt
        self.Ap = _csr_parts(inst.A, dt) if inst.A is not None else _empty_csr(dt)
        self.b = np.ascontiguousarray(inst.b if inst.b is not None else np.zeros(1), dt)
        self.Bp = _csr_parts(inst.B, dt) if inst.B is not None else _empty_csr(dt)
        self.d = np.ascontiguousarray(inst.d if inst.d is not None else np.zeros(1), dt)
        self.c = np.ascontiguousarray(inst.c, dt)
        self.qkind = 0
        self.Qd = self.Qp = self.Qc = self.Qv = None
        if isinstance(inst.Q, np.ndarray):
            self.qkind = 1
            self.Qd = np.ascontiguousarray(inst.Q, dt)
        elif inst.Q is not None:
            self.qkind = 2
            self.Qp, self.Qc, self.Qv = _csr_parts(inst.Q, dt)

    def __call__(self, X):
        X = np.ascontiguousarray(X, np.uint8)
        k = X.shape[0]
        viol = np.zeros(k, np.int32)
        L = lib()
        if self.integral:
            obj = np.zeros(k, np.int64)
            fn = L.orc_eval_int
        else:
            obj = np.zeros(k, np.float64)
            fn = L.orc_eval_f64
        fn(self.inst.n, self.inst.m1, *self.Ap, self.b, self.inst.m2, *self.Bp, self.d,
           self.qkind, _ptr(self.Qd), _ptr(self.Qp), _ptr(self.Qc), _ptr(self.Qv), self.c,
           k, X, viol, obj)
        return viol, obj

    def brute_force(self):
        assert self.integral and self.inst.n <= 24
        best = C.c_int64(0)
        nfeas = C.c_int64(0)
        bx = np.zeros(self.inst.n, np.uint8)
        found = lib().orc_brute_force(
            self.inst.n, self.inst.m1, *self.Ap, self.b, self.inst.m2, *self.Bp, self.d,
            self.qkind, _ptr(self.Qd), _ptr(self.Qp), _ptr(self.Qc), _ptr(self.Qv), self.c,
            C.byref(best), bx, C.byref(nfeas))
        return bool(found), best.value, bx, nfeas.value


def knapsack_lp(w, p, cap):
    w = np.ascontiguousarray(w, np.float64)
    p = np.ascontiguousarray(p, np.float64)
    x = np.zeros(w.size, np.float64)
    v = lib().orc_knapsack_lp(w.size, w, p, float(cap), x)
    return v, x


def incumbent_update(state, viol, obj, round_id):
    found = C.c_int32(state["found"])
    best = C.c_int64(state["obj"])
    br = C.c_uint32(state["round"])
    bs = C.c_int32(state["sample"])
    pick = lib().orc_incumbent_update(viol.size, np.ascontiguousarray(viol, np.int32),
                                      np.ascontiguousarray(obj, np.int64), round_id,
                                      C.byref(found), C.byref(best), C.byref(br), C.byref(bs))
    state.update(found=found.value, obj=best.value, round=br.value, sample=bs.value)
    return pick


# --------------------------------------------------------------------------
# Preprocess (Section 3)
# --------------------------------------------------------------------------
@dataclass
class Scaled:
    n: int
    m: int
    m1: int
    Kp: np.ndarray
    Kc: np.ndarray
    Kv: np.ndarray
    r: np.ndarray
    qkind: int
    Qd: Optional[np.ndarray]
    Qp: Optional[np.ndarray]
    Qc: Optional[np.ndarray]
    Qv: Optional[np.ndarray]
    c: np.ndarray
    normQ: float          # ||Q_hat||_2 after scaling
    s_obj: float
    s_K: float
    normQ_raw: float
    rownorm: np.ndarray
    iters: dict = field(default_factory=dict)


def power_norm_K(Kp, Kc, Kv, n, seed, inst_id, tol=1e-12, maxit=5000):
    it = C.c_int32(0)
    m = Kp.size - 1
    v = lib().orc_power_norm_K(m, n, Kp, Kc, Kv, seed, inst_id, tol, maxit, C.byref(it))
    return v, it.value


def power_norm_Q(Q, n, seed, inst_id, tol=1e-12, maxit=5000):
    it = C.c_int32(0)
    if Q is None:
        return 0.0, 0
    if isinstance(Q, np.ndarray):
        Qd = np.ascontiguousarray(Q, np.float64)
        v = lib().orc_power_norm_Q(1, n, _ptr(Qd), None, None, None, seed, inst_id, tol,
                                   maxit, C.byref(it))
    else:
        Qp, Qc, Qv = _csr_parts(Q, np.float64)
        v = lib().orc_power_norm_Q(2, n, None, _ptr(Qp), _ptr(Qc), _ptr(Qv), seed, inst_id,
                                   tol, maxit, C.byref(it))
    return v, it.value


def build_K(inst):
    """K = -[A; B], r = (b; d) (Eq. 2)."""
    blocks, rhs = [], []
    if inst.A is not None:
        blocks.append(-sp.csr_matrix(inst.A))
        rhs.append(np.asarray(inst.b, np.float64))
    if inst.B is not None:
        blocks.append(-sp.csr_matrix(inst.B))
        rhs.append(np.asarray(inst.d, np.float64))
    if not blocks:
        K = sp.csr_matrix((0, inst.n))
        r = np.zeros(0)
    else:
        K = sp.vstack(blocks, format="csr")
        r = np.concatenate(rhs)
    K.sum_duplicates()
    K.sort_indices()
    return K, r


def sym_Q(Q):
    """Q symmetric WLOG (Eq. 1): the gradient uses (Q + Q^T)/2."""
    if Q is None:
        return None
    if isinstance(Q, np.ndarray):
        return 0.5 * (Q + Q.T)
    S = (0.5 * (sp.csr_matrix(Q) + sp.csr_matrix(Q).T)).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    return S


def preprocess(inst, seed, inst_id=0, tol=1e-12, maxit=5000) -> Scaled:
    K, r = build_K(inst)
    m = K.shape[0]
    Kp, Kc, Kv = _csr_parts(K, np.float64) if m else _empty_csr(np.float64)
    r = np.ascontiguousarray(r, np.float64).copy()
    Kv = Kv.copy()
    rownorm = np.zeros(max(m, 1))
    st = lib().orc_row_normalize(m, inst.m1, Kp, Kv, r if m else np.zeros(1), rownorm)
    if st != 0:
        raise ValueError(f"infeasible empty row {-1 - st}")
    Qs = sym_Q(inst.Q)
    nq, itq = power_norm_Q(Qs, inst.n, seed, inst_id, tol, maxit)
    s_obj = nq + float(np.linalg.norm(inst.c))
    if s_obj == 0.0:
        s_obj = 1.0
    nk, itk = power_norm_K(Kp, Kc, Kv, inst.n, seed, inst_id, tol, maxit) if m else (0.0, 0)
    s_K = nk if nk > 0.0 else 1.0
    Kv = Kv / s_K
    r = r / s_K
    qkind, Qd, Qp, Qc, Qv = 0, None, None, None, None
    if isinstance(Qs, np.ndarray):
        qkind, Qd = 1, np.ascontiguousarray(Qs / s_obj)
    elif Qs is not None:
        qkind = 2
        Qp, Qc, Qv = _csr_parts(Qs, np.float64)
        Qv = Qv / s_obj
    c = np.ascontiguousarray(inst.c / s_obj, np.float64)
    return Scaled(inst.n, m, inst.m1, Kp, Kc, np.ascontiguousarray(Kv), np.ascontiguousarray(r),
                  qkind, Qd, Qp, Qc, Qv, c, nq / s_obj, s_obj, s_K, nq, rownorm[:m],
                  {"Q": itq, "K": itk})


def step_sizes(sigma, normQ, rho, cap):
    t1, t2 = C.c_double(0), C.c_double(0)
    lib().orc_step_sizes(sigma, normQ, rho, int(cap), C.byref(t1), C.byref(t2))
    return t1.value, t2.value


def rho_update(n, rho_prev, rho_min, rho_max, T, p, delta):
    return lib().orc_rho_update(n, rho_prev, rho_min, rho_max, T, p, delta)


def pdhg_step(S: Scaled, tau1, tau2, rho, x_prev, xbar_prev, y):
    """One FirstOrderStep (Alg. 2); returns (x_k, xbar_k, y_k, delta)."""
    x_prev = np.ascontiguousarray(x_prev, np.float64)
    xbar_prev = np.ascontiguousarray(xbar_prev, np.float64)
    y = np.ascontiguousarray(y, np.float64).copy() if S.m else np.zeros(1)
    x = np.zeros(S.n)
    xb = np.zeros(S.n)
    dl = np.zeros(S.n)
    lib().orc_pdhg_step(S.n, S.m, S.m1, S.Kp, S.Kc, S.Kv, S.r if S.m else np.zeros(1),
                        S.qkind, _ptr(S.Qd), _ptr(S.Qp), _ptr(S.Qc), _ptr(S.Qv), S.c, tau1,
                        tau2, rho, x_prev, xbar_prev, y, x, xb, _ptr(dl))
    return x, xb, (y[:S.m] if S.m else np.zeros(0)), dl


def halt_stats(S: Scaled, tau1, rho, x, xp, y):
    out = np.zeros(6)
    lib().orc_halt_stats(S.n, S.m, S.m1, S.Kp, S.Kc, S.Kv, S.r if S.m else np.zeros(1),
                         S.qkind, _ptr(S.Qd), _ptr(S.Qp), _ptr(S.Qc), _ptr(S.Qv), S.c, tau1,
                         rho, np.ascontiguousarray(x, np.float64),
                         np.ascontiguousarray(xp, np.float64),
                         np.ascontiguousarray(y if S.m else np.zeros(1), np.float64), out)
    return out


def x0_vector(n, x0, seed, inst_id):
    """Start point x_0 in [0,1]^n (Alg. 1 leaves it free).  x0 in [0,1]: the
    constant vector; x0 < 0: Philox uniform draws (stream 5) (u >> 8) 2^-24."""
    if x0 >= 0.0:
        return np.full(n, float(np.float32(x0)))
    u = philox_lanes(seed, 5, inst_id, 0, 0, n)
    return (u >> np.uint32(8)).astype(np.float64) * 2.0 ** -24


# --------------------------------------------------------------------------
# Alg. 1 driver
# --------------------------------------------------------------------------
@dataclass
class Params:
    sigma: float = 0.99
    rho_min: float = 1e-3
    rho_max: float = 1.0
    T: float = 20.0
    p: float = 2.0
    delta: float = 0.0
    k_int: int = 50
    k_r: int = 1
    k_b: int = 1024
    tau_cap_by_L: int = -1
    seed: int = 0x5EED0000
    x0: float = 0.5
    halt_tol: float = 1e-4
    stall_window: int = 20
    inst_base: int = 0


class HaltTracker:
    """Value-stalling detector of CheckHalt (Section 3); reading: an indicator
    is done when <= tol, or when its best value has not improved by 1e-3
    (relative) for stall_window triggers."""

    def __init__(self, tol, window):
        self.tol, self.window = tol, window
        self.best = [math.inf] * 3
        self.last = [0] * 3
        self.t = 0

    def update(self, vals):
        self.t += 1
        done = []
        for q in range(3):
            v = vals[q]
            if v < self.best[q] * (1.0 - 1e-3) or self.best[q] == math.inf:
                self.best[q] = v
                self.last[q] = self.t
            done.append(v <= self.tol or (self.t - self.last[q]) >= self.window)
        return all(done)


class OracleSolver:
    def __init__(self, inst, prm: Params, inst_id=None):
        self.inst = inst
        self.prm = prm
        self.inst_id = prm.inst_base if inst_id is None else inst_id
        self.S = preprocess(inst, prm.seed, self.inst_id)
        self.ev = Evaluator(inst)
        cap = prm.tau_cap_by_L
        self.cap = (self.S.qkind != 0) if cap < 0 else bool(cap)
        self.x = x0_vector(inst.n, prm.x0, prm.seed, self.inst_id)
        self.x_prev = self.x.copy()
        self.xbar = self.x.copy()
        self.y = np.zeros(self.S.m)
        self.k = 0
        self.n_rho = 0
        self.rho = rho_update(0, 0.0, prm.rho_min, prm.rho_max, prm.T, prm.p, prm.delta)
        self.inc = dict(found=0, obj=0, round=0, sample=-1)
        self.best_x = None
        self.halt = HaltTracker(prm.halt_tol, prm.stall_window)
        self.trace = []

    def taus(self):
        return step_sizes(self.prm.sigma, self.S.normQ, self.rho, self.cap)

    def step(self):
        """k <- k+1; UpdatePenalty; FirstOrderStep (Alg. 1 body, no sampling)."""
        self.k += 1
        n_rho = (self.k - 1) // self.prm.k_int
        while self.n_rho < n_rho:
            self.n_rho += 1
            P = self.prm
            self.rho = rho_update(self.n_rho, self.rho, P.rho_min, P.rho_max, P.T, P.p, P.delta)
        t1, t2 = self.taus()
        x, xb, y, _ = pdhg_step(self.S, t1, t2, self.rho, self.x, self.xbar, self.y)
        self.x_prev, self.x, self.xbar, self.y = self.x, x, xb, y

    def sample_round(self, round_id, k=None):
        k = self.prm.k_b if k is None else k
        p32 = self.x.astype(np.float32)
        X = sample(self.inst, p32, k, self.prm.seed, self.inst_id, round_id)
        viol, obj = self.ev(X)
        pick = incumbent_update(self.inc, viol, obj.astype(np.int64), round_id) \
            if self.ev.integral else -1
        if pick >= 0:
            self.best_x = X[pick].copy()
        return X, viol, obj

    def run(self, max_iters, halt=True):
        P = self.prm
        while self.k < max_iters:
            self.step()
            if self.k % P.k_int == 0:
                trig = self.k // P.k_int - 1
                for rr in range(P.k_r):
                    self.sample_round(trig * P.k_r + rr)
                t1, _ = self.taus()
                hs = halt_stats(self.S, t1, self.rho, self.x, self.x_prev, self.y)
                self.trace.append((self.k, self.rho, *hs[:3], self.inc["obj"], self.inc["found"]))
                if halt and self.halt.update(hs[:3]):
                    break
        xr = np.zeros(self.inst.n, np.uint8)
        lib().orc_round(self.inst.n, np.ascontiguousarray(self.x), xr)
        viol, obj = self.ev(xr[None, :])
        if self.ev.integral and incumbent_update(self.inc, viol, obj.astype(np.int64),
                                                 0xFFFFFFFF) >= 0:
            self.best_x = xr
        return self.inc


# --------------------------------------------------------------------------
# MLP (learned proposal) reference
# --------------------------------------------------------------------------
def bf16_round(a):
    a = np.asarray(a, np.float32)
    f = np.vectorize(lambda v: lib().orc_bf16_round(float(v)), otypes=[np.float32])
    return f(a) if a.size else a


def mlp_forward(feat, W, rb=1):
    feat = np.ascontiguousarray(feat, np.float32)
    nv, F = feat.shape
    H = W["b1"].size
    z = np.zeros(nv)
    p = np.zeros(nv)
    lib().orc_mlp_forward(nv, F, H, feat, *(np.ascontiguousarray(W[k], np.float32)
                                            for k in ("W1", "b1", "W2", "b2", "w3", "b3")),
                          rb, z, p, None, None)
    return z, p


def mlp_loss_grad(feat, label, W, rb=1):
    feat = np.ascontiguousarray(feat, np.float32)
    label = np.ascontiguousarray(label, np.float32)
    nv, F = feat.shape
    H = W["b1"].size
    g = {k: np.zeros(W[k].shape, np.float64) for k in ("W1", "b1", "W2", "b2", "w3", "b3")}
    loss = lib().orc_mlp_loss_grad(nv, F, H, feat, label,
                                   *(np.ascontiguousarray(W[k], np.float32)
                                     for k in ("W1", "b1", "W2", "b2", "w3", "b3")), rb,
                                   *(g[k] for k in ("W1", "b1", "W2", "b2", "w3", "b3")))
    return loss, g


def adam(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    lib().orc_adam(w.size, w, g, m, v, t, lr, b1, b2, eps)
