"""Failure detection without a GPU fault.

- A bounded device-side wait that runs out: one block of a cooperative PDHG
  launch is told (gfors_debug_inject) to wait at its first grid barrier
  without arriving, so the other blocks' waits expire after wait_timeout_s.
  The next synchronising call reports GFORS_E_TIMEOUT, the handle is failed
  from then on (GFORS_E_STATE), and a new handle on the same device works.
- An allocator hook that returns NULL gives GFORS_E_OOM, with every buffer
  the hook did hand out returned through its free function.
- Malformed input (bad CSR structure, out-of-range or non-finite entries,
  n <= 0, bad parameters) is rejected with GFORS_E_ARG before any device
  work; unsorted CSR rows with duplicates are legal and are merged.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2510_27117_b300 import workloads as W

pytestmark = pytest.mark.gpu
G = pytest.importorskip("paper_2510_27117_b300.gfors")

E_ARG, E_OOM, E_TIMEOUT, E_STATE = 1, 3, 4, 5


@pytest.mark.parametrize("kind,block", [("persistent", 3), ("persistent", 0),
                                        ("cooperative", 7)])
def test_barrier_wait_runs_out(kind, block):
    if kind == "persistent":
        inst, mode, path, x0 = W.max_cut(n=700, idx=6), 0, "persistent", -1.0
    else:
        inst, mode, path, x0 = W.assign3d(I=24, idx=5), 2, "cooperative", 0.5
    prm = G.default_params(k_int=10, k_b=64, x0=x0, pdhg_mode=mode, wait_timeout_s=0.05)
    H = G.load(inst, prm)
    assert H.pdhg_path() == path
    H.pdhg_steps(5)                        # healthy launch first
    x_ok = H.get_iterate(0)[0]
    H.debug_inject(1, block)
    H.pdhg_steps(20)
    with pytest.raises(G.GforsError) as e:
        H.lp_stats(0)
    assert e.value.status == E_TIMEOUT
    with pytest.raises(G.GforsError) as e:
        H.pdhg_steps(1)
    assert e.value.status == E_STATE
    H.destroy()
    # the context is still usable: a fresh handle runs and matches a clean run
    outs = []
    for _ in range(2):
        H2 = G.load(inst, prm)
        H2.pdhg_steps(5)
        outs.append(H2.get_iterate(0)[0])
        H2.destroy()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], x_ok)


def test_injection_is_consumed_and_clearable():
    inst = W.max_cut(n=300, idx=1)
    prm = G.default_params(k_int=10, k_b=64, wait_timeout_s=0.05)
    H = G.load(inst, prm)
    H.debug_inject(1, 2)
    H.debug_inject(0)                      # cleared before any launch
    H.pdhg_steps(12)
    H.lp_stats(0)
    H.debug_inject(1, 10_000)              # beyond the grid: nothing skips
    H.pdhg_steps(12)
    H.lp_stats(0)
    with pytest.raises(G.GforsError) as e:
        H.debug_inject(2, 0)
    assert e.value.status == E_ARG
    H.destroy()


@pytest.mark.parametrize("ok_allocs", [0, 5, 40])
def test_allocator_returning_null_gives_oom(ok_allocs):
    import torch
    torch.cuda.set_device(0)
    live = {}
    calls = [0]

    def alloc(size):
        calls[0] += 1
        if calls[0] > ok_allocs:
            return None
        p = torch.cuda.caching_allocator_alloc(size)
        live[p] = size
        return p

    def free(ptr):
        live.pop(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    inst = W.set_cover(n=500, m=60, density=0.05, idx=3)
    G.set_allocator(alloc, free)
    try:
        with pytest.raises(G.GforsError) as e:
            G.load(inst, G.default_params(k_b=64))
        assert e.value.status == E_OOM
        # a group of buffers may be requested before the group is checked
        assert calls[0] > ok_allocs
        assert not live                    # everything handed out came back
    finally:
        G.set_allocator(None, None)
    H = G.load(inst, G.default_params(k_b=64))   # cudaMalloc again
    H.pdhg_steps(3)
    H.destroy()


def _set_cover_arrays():
    inst = W.set_cover(n=50, m=8, density=0.2, idx=1)
    A = sp.csr_matrix(inst.A)
    return inst, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)


def _load_raw(n, rp, ci, v, b, c, prm=None):
    csr = G.Csr(len(rp) - 1, n, v.size, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    h = G._H()
    st = G._lib.gfors_load(G.C.byref(csr), b.ctypes.data, None, None, None, c.ctypes.data, n,
                           G.C.byref(prm or G.default_params(k_b=64)), None, G.C.byref(h))
    if st == 0:
        G._lib.gfors_destroy(h)
    return st


@pytest.mark.parametrize("defect", ["col_out_of_range", "col_negative", "nan_value",
                                    "inf_rhs", "nan_cost", "rowptr_not_monotone",
                                    "rowptr_start", "nnz_mismatch", "n_zero", "bad_k_b",
                                    "bad_sigma"])
def test_malformed_input_rejected(defect):
    inst, rp, ci, v = _set_cover_arrays()
    n, b, c = inst.n, inst.b.astype(np.float64).copy(), inst.c.astype(np.float64).copy()
    rp, ci, v = rp.copy(), ci.copy(), v.copy()
    prm = G.default_params(k_b=64)
    if defect == "col_out_of_range":
        ci[3] = n
    elif defect == "col_negative":
        ci[0] = -1
    elif defect == "nan_value":
        v[2] = np.nan
    elif defect == "inf_rhs":
        b[1] = np.inf
    elif defect == "nan_cost":
        c[4] = np.nan
    elif defect == "rowptr_not_monotone":
        rp[2], rp[3] = rp[3], rp[2]
    elif defect == "rowptr_start":
        rp = rp + 1
    elif defect == "nnz_mismatch":
        rp[-1] -= 1
    elif defect == "n_zero":
        n = 0
    elif defect == "bad_k_b":
        prm = G.default_params(k_b=48)
    elif defect == "bad_sigma":
        prm = G.default_params(k_b=64, sigma=1.5)
    st = _load_raw(n, rp, ci, v, b, c, prm)
    assert st == E_ARG, G._lib.gfors_last_error(None)


def test_unsorted_rows_with_duplicates_are_merged():
    """Unsorted columns and duplicate entries are legal CSR input: duplicates
    are summed, so the evaluation equals that of the canonical matrix."""
    inst, rp, ci, v = _set_cover_arrays()
    rows = []
    rng = np.random.default_rng(2)
    for j in range(len(rp) - 1):
        cols, vals = list(ci[rp[j]:rp[j + 1]]), list(v[rp[j]:rp[j + 1]])
        # split the first entry into two halves, then shuffle the row
        cols.append(cols[0])
        vals[0] = vals[0] / 2
        vals.append(vals[0])
        perm = rng.permutation(len(cols))
        rows.append((np.array(cols)[perm], np.array(vals)[perm]))
    rp2 = np.cumsum([0] + [len(r[0]) for r in rows]).astype(np.int64)
    ci2 = np.concatenate([r[0] for r in rows]).astype(np.int32)
    v2 = np.concatenate([r[1] for r in rows]).astype(np.float64)
    inst2 = W.Instance("unsorted", inst.n, inst.c, A=sp.csr_matrix((v2, ci2, rp2),
                                                                   shape=inst.A.shape),
                       b=inst.b)
    # the binding hands the duplicates and the column order over unchanged
    assert G._CsrHold(inst2.A, inst.n).v.size == v2.size > v.size
    X = (np.random.default_rng(3).random((64, inst.n)) < 0.3).astype(np.uint8)
    res = []
    for I in (inst, inst2):
        H = G.load(I, G.default_params(k_b=64))
        res.append(H.eval_candidates(X))
        H.destroy()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
