"""Path sharding across ranks (one process per GPU) and the merge of caplet
payoff sums.

Paths are independent and each path's Philox counter holds its global index,
so rank r of W simply simulates its own contiguous path range; the only
exchange is one gather of the FP64 sums (n x strikes x 2 values), added in
rank order so the merged result does not depend on arrival order.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def shard_range(total_paths: int, rank: int, world: int) -> Tuple[int, int]:
    """(first_path, count) of rank `rank`: contiguous, sizes differ by <= 1."""
    base, extra = divmod(int(total_paths), int(world))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def merge_sums(s1: np.ndarray, s2: np.ndarray, count: int, group=None):
    """All-gather (sum, sum of squares, path count) and add them in rank order.
    Returns the merged (s1, s2, count) on every rank."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    flat = np.concatenate([np.ravel(s1), np.ravel(s2), [float(count)]]).astype(np.float64)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.from_numpy(flat).to(dev)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    total = np.zeros_like(flat)
    for p in parts:  # fixed rank order
        total += p.cpu().numpy()
    k = s1.size
    return (total[:k].reshape(s1.shape), total[k:2 * k].reshape(s2.shape), int(round(total[-1])))
