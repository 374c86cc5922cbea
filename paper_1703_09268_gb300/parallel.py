"""Distribution of (source, frequency) pairs over ranks (Sec. 3: the objective
and gradient are sums over the joint source/frequency index set, computed
independently per worker and summed).

* shard(): the pairs a rank evaluates (strided, so every rank gets a spread of
  sources);
* allreduce_sum(): the one exchange step of the path, f and g summed over
  ranks;
* sum_with_deadline(): the paper's proposal for failing workers (Sec. 3):
  wait for each worker's contribution only until a deadline and sum what
  arrived, treating a missing worker as extra stochastic subsampling.
"""
from __future__ import annotations

import datetime
import pickle
from typing import List, Sequence, Tuple

import numpy as np


def shard(n_units: int, rank: int, world: int) -> List[int]:
    """Indices of the units (pairs) owned by `rank`: rank, rank+world, ..."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return list(range(rank, n_units, world))


def allreduce_sum(tensors: Sequence, group=None):
    """In-place sum over ranks of every tensor (torch.distributed, any backend)."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def sum_with_deadline(store, key: str, rank: int, world: int, local: Sequence[np.ndarray],
                      deadline_s: float) -> Tuple[List[np.ndarray], List[int]]:
    """Publish this rank's arrays under `key` and sum the contributions of every
    rank that published before the deadline.  Returns (sums, contributing ranks).

    `store` is a torch.distributed Store (TCPStore / FileStore).  A rank that
    never publishes (crashed, hung, too slow) is left out of the sum."""
    store.set(f"{key}/{rank}", pickle.dumps([np.asarray(a) for a in local]))
    sums = [np.array(a, dtype=np.float64, copy=True) for a in local]
    got = [rank]
    for r in range(world):
        if r == rank:
            continue
        try:
            store.wait([f"{key}/{r}"], datetime.timedelta(seconds=deadline_s))
        except Exception:
            continue
        other = pickle.loads(store.get(f"{key}/{r}"))
        for s, o in zip(sums, other):
            s += o
        got.append(r)
    return sums, sorted(got)
