"""Multi-process helpers (torch.distributed) for runs with one process per GPU.

Rows j of the LOO score are independent, so a sharded evaluation gives each
rank a contiguous row range and exchanges one G1 x G2 block of partial sums,
added in rank order so the result does not depend on arrival order.  The
benchmark runs independent replicas and only needs the max-over-ranks time.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def row_shards(N: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous [start, end) row ranges, sizes differing by at most one."""
    base, rem = divmod(N, world)
    out, s = [], 0
    for r in range(world):
        e = s + base + (1 if r < rem else 0)
        out.append((s, e))
        s = e
    return out


def _tensor(x, dist):
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device=dev)


def max_over_ranks(x: float) -> float:
    import torch.distributed as dist
    t = _tensor([x], dist)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.cpu()[0])


def sum_partials_in_rank_order(part: np.ndarray) -> np.ndarray:
    """All-gather each rank's partial block and add them in rank order."""
    import torch.distributed as dist
    world = dist.get_world_size()
    t = _tensor(part, dist)
    bufs = [t.clone() for _ in range(world)]
    dist.all_gather(bufs, t)
    total = np.zeros_like(np.asarray(part, dtype=np.float64))
    for b in bufs:
        total = total + b.cpu().numpy()
    return total
