"""Several devices: how the hot path splits, and the one exchange it needs.

The PDHG loop of one instance has no exchange step that a single collective
could serve, so nothing is communicated inside it.  Work splits two ways:

* Instances of a batch are independent (knapsack x512, facility location
  x16): rank r loads its own share, balanced by variable count, and only the
  final incumbents are gathered.
* The candidates of one round split by index: every rank runs the same
  deterministic PDHG iterations and scores candidates
  [s_begin, s_end) of every round (gfors_sample_eval_range keeps the indices
  global, so the union of the ranks' candidates is exactly the one-device
  round).  One all-gather of the 32-byte incumbent key
  (objective, round, candidate, rank) per trigger and a lexicographic minimum
  give the one-device incumbent (strictly better objective wins; the earliest
  round and candidate break ties, as in EvalBest).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

INT64_MAX = np.iinfo(np.int64).max


def shard_instances(sizes: Sequence[int], world: int, rank: int) -> List[int]:
    """Instances of rank `rank`: longest-first assignment to the least loaded
    rank (deterministic; ties to the lower rank)."""
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i)):
        r = min(range(world), key=lambda r: (load[r], r))
        owner[i] = r
        load[r] += int(sizes[i])
    return [i for i in range(len(sizes)) if owner[i] == rank]


def sample_range(k_b: int, world: int, rank: int) -> Tuple[int, int]:
    """Candidate range [s_begin, s_end) of `rank` in a round of k_b
    candidates, in whole 32-candidate words (the bit-packing unit)."""
    if k_b % 32:
        raise ValueError("k_b must be a multiple of 32")
    words = k_b // 32
    a = words * rank // world
    b = words * (rank + 1) // world
    return 32 * a, 32 * b


def min_key(keys: np.ndarray) -> np.ndarray:
    """Lexicographic minimum of rows (objective, round, candidate, rank)."""
    keys = np.asarray(keys, np.int64).reshape(-1, 4)
    order = np.lexsort(keys.T[::-1])
    return keys[order[0]].copy()


def reduce_incumbent_key(key3, rank: int, group=None):
    """All-gather (objective, round, candidate) of every rank -- a torch
    int64 tensor of 3 entries, on the device of the process group's backend
    -- and return the lexicographic minimum with the owning rank appended
    (host numpy int64[4]).  A rank without incumbent passes INT64_MAX."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    mine = torch.cat([key3.reshape(3).to(torch.int64),
                      torch.tensor([rank], dtype=torch.int64, device=key3.device)])
    allk = torch.empty(world * 4, dtype=torch.int64, device=key3.device)
    dist.all_gather_into_tensor(allk, mine, group=group)
    return min_key(allk.cpu().numpy())
