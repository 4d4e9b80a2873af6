"""Python binding of libgfors.so: argument marshalling only.

Every call maps one-to-one onto an entry point of include/gfors.h; all
computation runs in the library's CUDA kernels.  Importing this module fails
loudly (ImportError) when the library has not been built, and every solver
call fails (GforsError) on machines without an sm_103a GPU: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgfors.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libgfors.so not built ({LIB_PATH}); run paper_2510_27117_b300/build.py")
_lib = C.CDLL(LIB_PATH)

i32, i64, u32, u64, f64, vp = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double, C.c_void_p

STATUS = {0: "OK", 1: "E_ARG", 2: "E_CUDA", 3: "E_OOM", 4: "E_TIMEOUT", 5: "E_STATE",
          6: "E_UNSUPPORTED"}


class GforsError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class Csr(C.Structure):
    _fields_ = [("rows", i64), ("cols", i64), ("nnz", i64), ("row_ptr", vp),
                ("col_idx", vp), ("val", vp)]


class QMat(C.Structure):
    _fields_ = [("kind", i32), ("dense_rowmajor", vp), ("sparse", Csr)]


class Params(C.Structure):
    _fields_ = [("sigma", f64), ("rho_min", f64), ("rho_max", f64), ("T", f64), ("p", f64),
                ("delta", f64), ("k_int", i32), ("k_r", i32), ("k_b", i32),
                ("tau_cap_by_L", i32), ("seed", u64), ("x0", f64), ("halt_tol", f64),
                ("stall_window", i32), ("inst_base", i32), ("sample_chunk", i32),
                ("eval_mode", i32), ("power_tol", f64), ("power_maxit", i32),
                ("wait_timeout_s", f64), ("pdhg_mode", i32)]


_H = vp
_P = C.POINTER
_lib.gfors_default_params.argtypes = [_P(Params)]
_lib.gfors_version.restype = C.c_char_p
_lib.gfors_last_error.argtypes = [_H]
_lib.gfors_last_error.restype = C.c_char_p
ALLOC_FN = C.CFUNCTYPE(vp, C.c_size_t, vp)
FREE_FN = C.CFUNCTYPE(None, vp, vp)
_lib.gfors_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
_lib.gfors_load.argtypes = [_P(Csr), vp, _P(Csr), vp, _P(QMat), vp, i64, _P(Params), vp,
                            _P(_H)]
_lib.gfors_load_batch.argtypes = [i32, _P(_P(Csr)), _P(vp), _P(_P(Csr)), _P(vp),
                                  _P(_P(QMat)), _P(vp), _P(i64), _P(Params), vp, _P(_H)]
_lib.gfors_set_groups.argtypes = [_H, i32, i32, i64, vp, vp, i32]
_lib.gfors_set_closure.argtypes = [_H, i32, i64, vp, vp, vp]
_lib.gfors_set_repair_groups.argtypes = [_H, i32, i64, vp, vp]
_lib.gfors_set_repair_rows.argtypes = [_H, i32, i64, vp, vp]
_lib.gfors_pdhg_steps.argtypes = [_H, i64]
_lib.gfors_sample_eval.argtypes = [_H, i32, u32, i32]
_lib.gfors_final_round.argtypes = [_H]
_lib.gfors_run.argtypes = [_H, i64, f64, i32, _P(i64)]
_lib.gfors_run_graph.argtypes = [_H, i64, i32, vp, _P(i64), _P(i64)]
_lib.gfors_run_graph_prepare.argtypes = [_H, i32]
_lib.gfors_incumbent.argtypes = [_H, i32, _P(i32), _P(i64), _P(f64), _P(u32), _P(i32), vp]
_lib.gfors_lp_stats.argtypes = [_H, i32, vp]
_lib.gfors_get_scales.argtypes = [_H, i32, vp]
_lib.gfors_get_iterate.argtypes = [_H, i32, vp, vp, vp, vp]
_lib.gfors_set_iterate.argtypes = [_H, i32, vp, vp, vp]
_lib.gfors_set_counters.argtypes = [_H, i64, f64]
_lib.gfors_eval_candidates.argtypes = [_H, i32, i32, vp, vp, vp, vp]
_lib.gfors_get_samples.argtypes = [_H, i32, vp, vp, vp, _P(i32)]
_lib.gfors_mlp_nparams.argtypes = [i32, i32]
_lib.gfors_mlp_nparams.restype = i64
_lib.gfors_set_proposal.argtypes = [_H, vp, i64]
_lib.gfors_get_features.argtypes = [_H, i32, vp]
_lib.gfors_mlp_forward.argtypes = [i32, i32, vp, i64, vp, vp, vp, vp]
_lib.gfors_mlp_loss_grad.argtypes = [i32, i32, vp, i64, vp, vp, vp, vp, vp]
_lib.gfors_mlp_adam.argtypes = [i64, vp, vp, vp, vp, i64, f64, f64, f64, f64, vp]
_lib.gfors_state_export.argtypes = [_H, vp, _P(C.c_size_t)]
_lib.gfors_state_import.argtypes = [_H, vp, C.c_size_t]
_lib.gfors_profile.argtypes = [_H, i32]
_lib.gfors_debug_inject.argtypes = [_H, i32, i32]
_lib.gfors_profile_read.argtypes = [_H, i32, vp, vp]
_lib.gfors_launch_count.argtypes = [_H]
_lib.gfors_launch_count.restype = i64
_lib.gfors_destroy.argtypes = [_H]

EXPORTS = [n for n in dir(_lib) if n.startswith("gfors_")]


def version() -> str:
    return _lib.gfors_version().decode()


def default_params(**kw) -> Params:
    p = Params()
    _lib.gfors_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _check(st, h=None):
    if st != 0:
        msg = _lib.gfors_last_error(h).decode(errors="replace")
        raise GforsError(st, msg)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(vp)


_alloc_keep = []


def set_allocator(alloc=None, free=None):
    """gfors_set_allocator with Python callables alloc(size) -> int device
    address or None, free(ptr); both None restores cudaMalloc / cudaFree."""
    if alloc is None and free is None:
        _alloc_keep[:] = []
        _check(_lib.gfors_set_allocator(ALLOC_FN(0), FREE_FN(0), None))
        return
    fa = ALLOC_FN(lambda size, ctx: alloc(int(size)))
    ff = FREE_FN(lambda ptr, ctx: free(ptr))
    _alloc_keep[:] = [fa, ff]
    _check(_lib.gfors_set_allocator(fa, ff, None))


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through PyTorch's caching
    allocator (device memory comes from torch; the kernels are the library's)."""
    if not enable:
        _check(_lib.gfors_set_allocator(ALLOC_FN(0), FREE_FN(0), None))
        return
    import torch

    def _a(size, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(size))
        except Exception:
            return None

    def _f(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = ALLOC_FN(_a), FREE_FN(_f)
    _alloc_keep[:] = [fa, ff]
    _check(_lib.gfors_set_allocator(fa, ff, None))


class _CsrHold:
    """Keeps the numpy arrays of one CSR alive while the library copies it."""

    def __init__(self, M, n):
        import scipy.sparse as sp
        M = sp.csr_matrix(M)
        self.rp = np.ascontiguousarray(M.indptr, np.int64)
        self.ci = np.ascontiguousarray(M.indices, np.int32)
        self.v = np.ascontiguousarray(M.data, np.float64)
        self.s = Csr(M.shape[0], n, self.v.size, _ptr(self.rp), _ptr(self.ci), _ptr(self.v))


class _InstHold:
    def __init__(self, inst):
        self.n = inst.n
        self.A = _CsrHold(inst.A, inst.n) if inst.A is not None else None
        self.B = _CsrHold(inst.B, inst.n) if inst.B is not None else None
        self.b = np.ascontiguousarray(inst.b, np.float64) if inst.A is not None else None
        self.d = np.ascontiguousarray(inst.d, np.float64) if inst.B is not None else None
        self.c = np.ascontiguousarray(inst.c, np.float64)
        self.Q = None
        self.Qd = None
        self.Qs = None
        if isinstance(inst.Q, np.ndarray):
            self.Qd = np.ascontiguousarray(inst.Q, np.float64)
            self.Q = QMat(1, _ptr(self.Qd), Csr())
        elif inst.Q is not None:
            self.Qs = _CsrHold(inst.Q, inst.n)
            self.Q = QMat(2, None, self.Qs.s)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream      # torch.cuda.Stream


class Handle:
    """One loaded batch (gfors_handle)."""

    def __init__(self, h, insts):
        self.h = vp(h)
        self.insts = insts

    # --- Alg. 1 pieces
    def pdhg_steps(self, nsteps):
        _check(_lib.gfors_pdhg_steps(self.h, nsteps), self.h)

    def sample_eval(self, nrounds, first_round_id, proposal=0):
        _check(_lib.gfors_sample_eval(self.h, nrounds, first_round_id, proposal), self.h)

    def set_assign3d_custom(self, inst, I, gamma=1, L=None):
        """Algorithm 4 sampler for instance inst (L defaults to I steps)."""
        _check(_lib.gfors_set_assign3d_custom(self.h, inst, I, gamma, I if L is None else L),
               self.h)

    def dense_info(self, inst=0):
        """(dense, tensor-core exact, fp8 operands, max|W2|) of instance inst."""
        out = np.zeros(4, np.int64)
        _check(_lib.gfors_dense_info(self.h, inst, _ptr(out)), self.h)
        return dict(dense=bool(out[0]), tc=bool(out[1]), fp8=bool(out[2]), w2max=int(out[3]))

    def pdhg_path(self):
        """Name of the kernels that run this handle's PDHG iterations."""
        v = C.c_int32(0)
        _check(_lib.gfors_pdhg_path(self.h, C.byref(v)), self.h)
        return ("buckets", "one_row", "small", "cooperative", "persistent",
                "cluster")[v.value]

    def sample_eval_range(self, nrounds, first_round_id, proposal, s_begin, s_end):
        _check(_lib.gfors_sample_eval_range(self.h, nrounds, first_round_id, proposal,
                                            s_begin, s_end), self.h)

    def set_iterate_async(self, inst, x, xbar=None, y=None):
        """Enqueue the iterate copies; the arrays must stay alive and unchanged
        until the stream passes them (pinned memory: truly asynchronous)."""
        _check(_lib.gfors_set_iterate_async(self.h, inst, _ptr(x), _ptr(xbar), _ptr(y)), self.h)

    def incumbent_async(self, inst, key_host):
        """Enqueue the copy of (obj, round, sample) into key_host (int64[3],
        pinned); valid after synchronize()."""
        _check(_lib.gfors_incumbent_async(self.h, inst, _ptr(key_host)), self.h)

    def synchronize(self):
        _check(_lib.gfors_synchronize(self.h), self.h)

    def incumbent_key_async(self, inst, key_dev_ptr):
        """Write (obj, round, sample) of instance inst to 3 int64 at a device
        address (e.g. tensor.data_ptr()), on the handle's stream."""
        _check(_lib.gfors_incumbent_key_async(self.h, inst, key_dev_ptr), self.h)

    def final_round(self):
        _check(_lib.gfors_final_round(self.h), self.h)

    def run(self, max_iters, time_budget_s=0.0, proposal=0):
        it = i64(0)
        _check(_lib.gfors_run(self.h, max_iters, time_budget_s, proposal, C.byref(it)), self.h)
        return it.value

    def run_graph(self, max_iters, proposal=0, targets=None):
        """gfors_run_graph: Alg. 1 as one CUDA-graph launch with CheckHalt on
        the device; targets (one int per instance) add the target stop.
        Returns (iterations, triggers run in the graph)."""
        it, tr = i64(0), i64(0)
        t = None if targets is None else np.ascontiguousarray(targets, np.int64)
        _check(_lib.gfors_run_graph(self.h, max_iters, proposal, _ptr(t), C.byref(it),
                                    C.byref(tr)), self.h)
        return it.value, tr.value

    def run_graph_prepare(self, proposal=0):
        """gfors_run_graph_prepare: build the whole-run graph now (set-up)."""
        _check(_lib.gfors_run_graph_prepare(self.h, proposal), self.h)

    # --- results and state
    def incumbent(self, inst=0, want_x=True):
        n = self.insts[inst].n
        f, oi, of, rr, ss = i32(), i64(), f64(), u32(), i32()
        x = np.zeros(n, np.uint8) if want_x else None
        _check(_lib.gfors_incumbent(self.h, inst, C.byref(f), C.byref(oi), C.byref(of),
                                    C.byref(rr), C.byref(ss), _ptr(x)), self.h)
        return dict(found=f.value, obj=oi.value, objf=of.value, round=rr.value,
                    sample=ss.value, x=x)

    def lp_stats(self, inst=0):
        out = np.zeros(8)
        _check(_lib.gfors_lp_stats(self.h, inst, _ptr(out)), self.h)
        return out

    def get_scales(self, inst=0):
        out = np.zeros(8)
        _check(_lib.gfors_get_scales(self.h, inst, _ptr(out)), self.h)
        return out

    def get_iterate(self, inst=0):
        I = self.insts[inst]
        m = I.m1 + I.m2
        x, xb, xp = (np.zeros(I.n, np.float32) for _ in range(3))
        y = np.zeros(max(m, 1), np.float32)
        _check(_lib.gfors_get_iterate(self.h, inst, _ptr(x), _ptr(xb), _ptr(xp), _ptr(y)),
               self.h)
        return x, xb, xp, y[:m]

    def set_iterate(self, inst=0, x=None, xbar=None, y=None):
        a = [None if v is None else np.ascontiguousarray(v, np.float32) for v in (x, xbar, y)]
        _check(_lib.gfors_set_iterate(self.h, inst, *(_ptr(v) for v in a)), self.h)

    def set_counters(self, k, rho=-1.0):
        _check(_lib.gfors_set_counters(self.h, k, rho), self.h)

    def eval_candidates(self, X, inst=0):
        X = np.ascontiguousarray(X, np.uint8)
        k = X.shape[0]
        viol = np.zeros(k, np.int32)
        oi = np.zeros(k, np.int64)
        of = np.zeros(k, np.float64)
        _check(_lib.gfors_eval_candidates(self.h, inst, k, _ptr(X), _ptr(viol), _ptr(oi),
                                          _ptr(of)), self.h)
        return viol, oi

    def get_samples(self, inst=0, want_x=True):
        n = self.insts[inst].n
        cnt = i32()
        _check(_lib.gfors_get_samples(self.h, inst, None, None, None, C.byref(cnt)), self.h)
        k = cnt.value
        X = np.zeros((k, n), np.uint8) if want_x else None
        viol = np.zeros(k, np.int32)
        oi = np.zeros(k, np.int64)
        _check(_lib.gfors_get_samples(self.h, inst, _ptr(X), _ptr(viol), _ptr(oi),
                                      C.byref(cnt)), self.h)
        return X, viol, oi

    def set_groups(self, inst=0, mode=1, groups=None, axial_I=0):
        gp = gi = None
        ng = 0
        if groups is not None:
            gp = np.ascontiguousarray(groups[0], np.int64)
            gi = np.ascontiguousarray(groups[1], np.int64)
            ng = gp.size - 1
        _check(_lib.gfors_set_groups(self.h, inst, mode, ng, _ptr(gp), _ptr(gi), axial_I),
               self.h)

    def set_repair_groups(self, inst, groups):
        gp, gi = (np.ascontiguousarray(a, np.int64) for a in groups)
        _check(_lib.gfors_set_repair_groups(self.h, inst, gp.size - 1, _ptr(gp), _ptr(gi)),
               self.h)

    def set_repair_rows(self, inst, rows):
        """gfors_set_repair_rows: (row_ptr, row_idx) of relaxed covering rows."""
        rp, ri = (np.ascontiguousarray(a, np.int64) for a in rows)
        _check(_lib.gfors_set_repair_rows(self.h, inst, rp.size - 1, _ptr(rp), _ptr(ri)),
               self.h)

    def set_closure(self, inst, closure):
        rv, rp, ri = (np.ascontiguousarray(a, np.int64) for a in closure)
        _check(_lib.gfors_set_closure(self.h, inst, rv.size, _ptr(rv), _ptr(rp), _ptr(ri)),
               self.h)

    def set_proposal(self, W):
        W = np.ascontiguousarray(W, np.float32)
        _check(_lib.gfors_set_proposal(self.h, _ptr(W), W.size), self.h)

    def get_features(self, inst=0):
        n = self.insts[inst].n
        f = np.zeros((n, 8), np.float32)
        _check(_lib.gfors_get_features(self.h, inst, _ptr(f)), self.h)
        return f

    def state_export(self) -> bytes:
        ln = C.c_size_t(0)
        _check(_lib.gfors_state_export(self.h, None, C.byref(ln)), self.h)
        buf = C.create_string_buffer(ln.value)
        _check(_lib.gfors_state_export(self.h, buf, C.byref(ln)), self.h)
        return buf.raw[:ln.value]

    def state_import(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(_lib.gfors_state_import(self.h, buf, len(blob)), self.h)

    # "eval_q" (the sparse-Q objective kernel) is also counted inside "eval"
    PHASES = ("pdhg", "sample", "eval", "dense_score", "incumbent", "fused", "stats",
              "dense_sample", "eval_q")

    def profile(self, enable=True):
        _check(_lib.gfors_profile(self.h, int(enable)), self.h)

    def debug_inject(self, kind, block=0):
        """gfors_debug_inject: kind 1 makes one block of the next cooperative
        PDHG launch skip its first grid-barrier arrival (tests of the
        bounded waits); kind 0 clears it."""
        _check(_lib.gfors_debug_inject(self.h, kind, block), self.h)

    def profile_read(self):
        n = len(self.PHASES)
        ms = np.zeros(n)
        cnt = np.zeros(n, np.int64)
        _check(_lib.gfors_profile_read(self.h, n, _ptr(ms), _ptr(cnt)), self.h)
        return {k: (float(ms[q]), int(cnt[q])) for q, k in enumerate(self.PHASES)}

    def autotune(self, cache_path=None):
        """gfors_autotune; returns (lanes[10], cache hit)."""
        lanes = np.zeros(10, np.int32)
        hit = i32()
        _check(_lib.gfors_autotune(self.h, None if cache_path is None else str(cache_path).encode(),
                                   _ptr(lanes), C.byref(hit)), self.h)
        return lanes, bool(hit.value)

    def set_lanes(self, lanes):
        lanes = np.ascontiguousarray(lanes, np.int32)
        _check(_lib.gfors_set_lanes(self.h, _ptr(lanes)), self.h)

    def get_lanes(self):
        lanes = np.zeros(10, np.int32)
        _check(_lib.gfors_get_lanes(self.h, _ptr(lanes)), self.h)
        return lanes

    def tune_key(self):
        buf = C.create_string_buffer(512)
        _check(_lib.gfors_tune_key(self.h, buf, 512), self.h)
        return buf.value.decode()

    def launch_count(self) -> int:
        return _lib.gfors_launch_count(self.h)

    def destroy(self):
        if self.h:
            _lib.gfors_destroy(self.h)
            self.h = vp(None)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def load(inst, prm: Optional[Params] = None, stream=None, setup=True) -> Handle:
    """gfors_load for one workloads.Instance (plus its groups / closure)."""
    return load_batch([inst], prm, stream, setup)


def load_batch(insts: Sequence, prm: Optional[Params] = None, stream=None,
               setup=True) -> Handle:
    """gfors_load_batch; with setup=True also gfors_set_groups / set_closure
    from each instance's groups, axial size and closure lists."""
    prm = default_params() if prm is None else prm
    holds = [_InstHold(I) for I in insts]
    nb = len(insts)
    A = (_P(Csr) * nb)(*[C.pointer(hd.A.s) if hd.A else _P(Csr)() for hd in holds])
    B = (_P(Csr) * nb)(*[C.pointer(hd.B.s) if hd.B else _P(Csr)() for hd in holds])
    Q = (_P(QMat) * nb)(*[C.pointer(hd.Q) if hd.Q is not None else _P(QMat)() for hd in holds])
    b = (vp * nb)(*[_ptr(hd.b) for hd in holds])
    d = (vp * nb)(*[_ptr(hd.d) for hd in holds])
    c = (vp * nb)(*[_ptr(hd.c) for hd in holds])
    n = (i64 * nb)(*[hd.n for hd in holds])
    h = _H()
    st = _lib.gfors_load_batch(nb, A, b, B, d, Q, c, n, C.byref(prm), _stream_ptr(stream),
                               C.byref(h))
    _check(st, None)
    H = Handle(h.value, list(insts))
    if setup:
        for q, I in enumerate(insts):
            if I.axial_I and I.meta.get("sampler") == "alg4":
                H.set_assign3d_custom(q, I.axial_I, I.meta.get("gamma", 1),
                                      I.meta.get("L", I.axial_I))
            elif I.axial_I:
                H.set_groups(q, 2, None, I.axial_I)
            elif I.groups is not None:
                H.set_groups(q, 1, I.groups)
            if getattr(I, "repair", None) is not None:
                H.set_repair_groups(q, I.repair)
            if getattr(I, "repair_rows", None) is not None:
                H.set_repair_rows(q, I.repair_rows)
            if I.closure is not None:
                H.set_closure(q, I.closure)
    return H


_lib.gfors_sample_eval_range.argtypes = [vp, i32, u32, i32, i32, i32]
_lib.gfors_set_assign3d_custom.argtypes = [vp, i32, i32, i32, i32]
_lib.gfors_dense_info.argtypes = [vp, i32, vp]
_lib.gfors_pdhg_path.argtypes = [vp, vp]
_lib.gfors_set_iterate_async.argtypes = [vp, i32, vp, vp, vp]
_lib.gfors_incumbent_async.argtypes = [vp, i32, vp]
_lib.gfors_synchronize.argtypes = [vp]
_lib.gfors_tu_reformulate.argtypes = [i64, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp]
_lib.gfors_tu_sizes.argtypes = [vp, vp]
_lib.gfors_tu_copy.argtypes = [vp] + [vp] * 14
_lib.gfors_tu_recover.argtypes = [vp, i64, vp, vp]
_lib.gfors_tu_free.argtypes = [vp]
_lib.gfors_tu_free.restype = None
_lib.gfors_incumbent_key_async.argtypes = [vp, i32, vp]
_lib.gfors_autotune.argtypes = [vp, C.c_char_p, vp, vp]
_lib.gfors_set_lanes.argtypes = [vp, vp]
_lib.gfors_get_lanes.argtypes = [vp, vp]
_lib.gfors_tune_key.argtypes = [vp, C.c_char_p, C.c_size_t]
_lib.gfors_tune_cache_lookup.argtypes = [C.c_char_p, C.c_char_p, vp, vp]
_lib.gfors_tune_cache_store.argtypes = [C.c_char_p, C.c_char_p, vp]


class TuReformulation:
    """gfors_tu: a TU-reformulated problem (Thm. 5) and the map back."""

    def __init__(self, t, n, nbar, c0, Ibar):
        self.t = t if isinstance(t, vp) else vp(t)
        self.n, self.nbar, self.c0, self.Ibar = n, nbar, c0, Ibar

    def recover(self, Xbar):
        """Original candidates (k x n uint8) from candidates over x_Ibar."""
        Xbar = np.ascontiguousarray(Xbar, np.uint8).reshape(-1, self.nbar)
        X = np.zeros((Xbar.shape[0], self.n), np.uint8)
        _check(_lib.gfors_tu_recover(self.t, Xbar.shape[0], _ptr(Xbar), _ptr(X)))
        return X

    def __del__(self):
        if getattr(self, "t", None) is not None and self.t.value:
            _lib.gfors_tu_free(self.t)
            self.t = None


def tu_reformulate(inst, J, I):
    """gfors_tu_reformulate on an Instance: returns (Instance over x_Ibar,
    TuReformulation).  The new instance's meta holds the objective constant
    c0' ("tu_c0"); groups, closure and axial marks do not carry over."""
    import scipy.sparse as sp
    from .workloads import Instance
    hd = _InstHold(inst)
    J = np.ascontiguousarray(J, np.int64)
    I = np.ascontiguousarray(I, np.int64)
    out = vp()
    _check(_lib.gfors_tu_reformulate(
        inst.n, C.byref(hd.A.s) if hd.A else None, _ptr(hd.b) if hd.b is not None else None,
        C.byref(hd.B.s) if hd.B else None, _ptr(hd.d) if hd.d is not None else None,
        C.byref(hd.Q) if hd.Q is not None else None, _ptr(hd.c), J.size, _ptr(J), _ptr(I),
        C.byref(out)))
    sz = np.zeros(8, np.int64)
    _check(_lib.gfors_tu_sizes(out, _ptr(sz)))
    nbar, m1, nnzA, m2, nnzB, hasQ, nnzQ = (int(v) for v in sz[:7])
    Ap, Ac, Av = np.zeros(m1 + 1, np.int64), np.zeros(max(nnzA, 1), np.int32), np.zeros(max(nnzA, 1))
    Bp, Bc, Bv = np.zeros(m2 + 1, np.int64), np.zeros(max(nnzB, 1), np.int32), np.zeros(max(nnzB, 1))
    Qp, Qc, Qv = np.zeros(nbar + 1, np.int64), np.zeros(max(nnzQ, 1), np.int32), np.zeros(max(nnzQ, 1))
    b, d, c = np.zeros(max(m1, 1)), np.zeros(max(m2, 1)), np.zeros(nbar)
    c0 = C.c_double(0.0)
    Ibar = np.zeros(nbar, np.int64)
    _check(_lib.gfors_tu_copy(out, _ptr(Ap), _ptr(Ac), _ptr(Av), _ptr(b), _ptr(Bp), _ptr(Bc),
                              _ptr(Bv), _ptr(d), _ptr(Qp), _ptr(Qc), _ptr(Qv), _ptr(c),
                              C.byref(c0), _ptr(Ibar)))
    A = sp.csr_matrix((Av[:nnzA], Ac[:nnzA], Ap), shape=(m1, nbar)) if m1 else None
    B = sp.csr_matrix((Bv[:nnzB], Bc[:nnzB], Bp), shape=(m2, nbar)) if m2 else None
    Q = sp.csr_matrix((Qv[:nnzQ], Qc[:nnzQ], Qp), shape=(nbar, nbar)) if hasQ else None
    new = Instance(inst.name + "_tu", nbar, c, A=A, b=b[:m1] if m1 else None, B=B,
                   d=d[:m2] if m2 else None, Q=Q)
    new.meta["tu_c0"] = c0.value
    return new, TuReformulation(out, inst.n, nbar, c0.value, Ibar)


def tune_cache_lookup(path, key):
    """Lanes stored for key in the tuning cache at path, or None."""
    lanes = np.zeros(10, np.int32)
    found = i32()
    _check(_lib.gfors_tune_cache_lookup(str(path).encode(), key.encode(), _ptr(lanes),
                                        C.byref(found)))
    return lanes if found.value else None


def tune_cache_store(path, key, lanes):
    lanes = np.ascontiguousarray(lanes, np.int32)
    _check(_lib.gfors_tune_cache_store(str(path).encode(), key.encode(), _ptr(lanes)))


NOALLOC_MAX_SAMPLES = 16384
_lib.gfors_fused_eval_noalloc.argtypes = [vp, vp, vp, i64, i64, u64, u32, u32, i32, i32, vp,
                                          vp, vp]


def fused_eval_noalloc(p_dev, a_dev, c_dev, n, rhs, seed, inst_id, round_id, first_sample,
                       nsamples, viol_dev, obj_dev, stream=None):
    """gfors_fused_eval_noalloc on caller-owned device buffers (integer device
    addresses, e.g. torch.Tensor.data_ptr()); allocates nothing."""
    _check(_lib.gfors_fused_eval_noalloc(p_dev, a_dev, c_dev, n, rhs, seed, inst_id, round_id,
                                         first_sample, nsamples, viol_dev, obj_dev,
                                         _stream_ptr(stream)))


def mlp_nparams(F=8, H=128) -> int:
    return _lib.gfors_mlp_nparams(F, H)


def mlp_forward(W_dev, nv, feat_dev, z_dev, p_dev=None, stream=None, F=8, H=128):
    """gfors_mlp_forward on device addresses (e.g. tensor.data_ptr())."""
    _check(_lib.gfors_mlp_forward(F, H, W_dev, nv, feat_dev, z_dev, p_dev, _stream_ptr(stream)))


def mlp_loss_grad(W_dev, nv, feat_dev, label_dev, grad_dev, loss_dev=None, stream=None, F=8,
                  H=128):
    """gfors_mlp_loss_grad on device addresses."""
    _check(_lib.gfors_mlp_loss_grad(F, H, W_dev, nv, feat_dev, label_dev, grad_dev, loss_dev,
                                    _stream_ptr(stream)))


def mlp_adam(np_, W_dev, grad_dev, m_dev, v_dev, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
             stream=None):
    """gfors_mlp_adam on device addresses."""
    _check(_lib.gfors_mlp_adam(np_, W_dev, grad_dev, m_dev, v_dev, t, lr, beta1, beta2, eps,
                               _stream_ptr(stream)))
