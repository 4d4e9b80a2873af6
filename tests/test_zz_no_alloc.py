"""The allocation-free entry point gfors_fused_eval_noalloc, called through
the C ABI on caller-owned device buffers, returns exactly the violation
flags and objectives of the regular single-row path (gfors_sample_eval on a
loaded knapsack), on two calls in a row (the second call must not see the
first call's scratch).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2510_27117_b300 import workloads as W

pytestmark = pytest.mark.gpu
G = pytest.importorskip("paper_2510_27117_b300.gfors")


def test_noalloc_matches_handle_path_twice():
    import torch
    torch.cuda.set_device(0)
    inst = W.knapsack(6003, idx=21)
    k_b, R, seed = 1024, 17, 0x5EED0042
    prm = G.default_params(k_b=k_b, seed=seed, eval_mode=2, inst_base=5)
    H = G.load(inst, prm)
    rng = np.random.default_rng(9)
    p = rng.random(inst.n).astype(np.float32)
    H.set_iterate(0, p, p, None)
    H.sample_eval(1, R, 0)
    _, viol_ref, obj_ref = H.get_samples(0, want_x=False)
    H.destroy()
    assert viol_ref.size == k_b and 0 < viol_ref.sum() < k_b

    a = np.zeros(inst.n, np.int32)
    a[inst.A.indices] = inst.A.data.astype(np.int32)
    p_t = torch.from_numpy(p).cuda()
    a_t = torch.from_numpy(a).cuda()
    c_t = torch.from_numpy(inst.c.astype(np.int64)).cuda()
    viol_t = torch.full((k_b,), -7, dtype=torch.int32, device="cuda")
    obj_t = torch.full((k_b,), 123, dtype=torch.int64, device="cuda")
    rhs = int(inst.b[0])
    for call in range(2):
        G.fused_eval_noalloc(p_t.data_ptr(), a_t.data_ptr(), c_t.data_ptr(), inst.n, rhs, seed,
                             5, R, 0, k_b, viol_t.data_ptr(), obj_t.data_ptr(), None)
        torch.cuda.synchronize()
        assert np.array_equal(viol_t.cpu().numpy(), viol_ref), f"call {call}"
        assert np.array_equal(obj_t.cpu().numpy(), obj_ref), f"call {call}"


def test_noalloc_rejects_oversize():
    with pytest.raises(G.GforsError):
        G.fused_eval_noalloc(0, 0, 0, 10, 0, 1, 0, 0, 0, G.NOALLOC_MAX_SAMPLES + 1, 0, 0, None)


def test_noalloc_rejects_index_overflow():
    """Candidate indices first_sample + s must stay within int32.  Real
    device buffers are passed, so the call would be harmless even if the
    check were missing; the error text shows which check fired."""
    import torch
    viol_t = torch.zeros(200, dtype=torch.int32, device="cuda")
    obj_t = torch.zeros(200, dtype=torch.int64, device="cuda")
    with pytest.raises(G.GforsError, match="INT32_MAX"):
        G.fused_eval_noalloc(0, 0, 0, 0, 0, 1, 0, 0, 2**31 - 100, 200, viol_t.data_ptr(),
                             obj_t.data_ptr(), None)
