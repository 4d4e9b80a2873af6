"""Several processes (gloo on CPU, world size 2): the candidate-range split
of one round and the incumbent min-reduction reproduce the one-process
incumbent; instance sharding covers a batch once and balances it.  The
candidates are drawn and scored by the oracle (no GPU needed)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2510_27117_b300 import shard as SH
from paper_2510_27117_b300 import workloads as W


def _incumbent(viol, obj, round_id, first_sample):
    """EvalBest over one block of candidates: strictly smaller objective
    among feasible ones; the earliest candidate wins ties."""
    best = None
    for s in range(len(obj)):
        if viol[s] == 0 and (best is None or obj[s] < best[0]):
            best = (int(obj[s]), round_id, first_sample + s)
    return best


def _scores(inst, k_b, nrounds):
    """Plain proposal after a few oracle PDHG steps; viol/obj of every
    candidate of every round (candidate indices global)."""
    P = O.Params(k_int=5, k_b=k_b, seed=0x5EED0000 + 3, x0=0.5)
    sol = O.OracleSolver(inst, P)
    for _ in range(5):
        sol.step()
    p32 = sol.x.astype(np.float32)
    ev = O.Evaluator(inst)
    out = []
    for r in range(nrounds):
        X = O.sample(inst, p32, k_b, P.seed, 0, r)
        viol, obj = ev(X)[:2]
        out.append((np.asarray(viol), np.asarray(obj)))
    return out


def _worker(rank, world, port, k_b, nrounds, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = W.tiny_bip(n=16, m1=3, m2=1, idx=4)
    sc = _scores(inst, k_b, nrounds)
    sb, se = SH.sample_range(k_b, world, rank)
    best = None
    for r, (viol, obj) in enumerate(sc):          # this rank's candidates only
        b = _incumbent(viol[sb:se], obj[sb:se], r, sb)
        if b is not None and (best is None or b[0] < best[0]):
            best = b
    key = torch.tensor(best if best else [SH.INT64_MAX] * 3, dtype=torch.int64)
    g = SH.reduce_incumbent_key(key, rank)
    q.put((rank, g.tolist()))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_candidate_split_and_min_reduction_match_one_process():
    k_b, nrounds, world = 96, 3, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, k_b, nrounds, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # one process over all candidates
    inst = W.tiny_bip(n=16, m1=3, m2=1, idx=4)
    best = None
    for r, (viol, obj) in enumerate(_scores(inst, k_b, nrounds)):
        b = _incumbent(viol, obj, r, 0)
        if b is not None and (best is None or b[0] < best[0]):
            best = b
    assert best is not None
    for rank in range(world):
        assert res[rank][:3] == list(best)
    assert res[0] == res[1]
    assert res[0][3] == (0 if best[2] < SH.sample_range(k_b, world, 0)[1] else 1)


def test_sample_ranges_tile_the_round():
    for k_b in (32, 96, 1024, 8192):
        for world in (1, 2, 3, 8):
            rs = [SH.sample_range(k_b, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == k_b
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert all(a % 32 == 0 and b % 32 == 0 for a, b in rs)
    with pytest.raises(ValueError):
        SH.sample_range(100, 2, 0)


def test_instance_sharding_covers_and_balances():
    sizes = W._rng(W.KN, 999_000).integers(1000, 100001, size=512)
    for world in (1, 2, 4, 8):
        parts = [SH.shard_instances(sizes, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(512))
        loads = [int(sum(sizes[i] for i in p)) for p in parts]
        assert max(loads) - min(loads) <= int(sizes.max())     # LPT bound


def test_min_key_is_lexicographic():
    k = np.array([[5, 2, 9, 1], [5, 1, 30, 0], [7, 0, 0, 2], [5, 1, 3, 3]], np.int64)
    assert SH.min_key(k).tolist() == [5, 1, 3, 3]
    none = np.full((2, 4), SH.INT64_MAX, np.int64)
    none[:, 3] = [0, 1]
    assert SH.min_key(none)[0] == SH.INT64_MAX
