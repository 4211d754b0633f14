"""Host-side logic for running on several GPUs of one node.

The solver path does not shard a single chain across GPUs here (every run of this
project has one GPU per process and a chain's iteration would need an all-gather of x
per sweep).  What does shard is independent work: replicas of the same solve, or the
chains of a batch, one subset per rank with no data-path collective.  Only the timing
uses a collective (the max over ranks).
"""
from __future__ import annotations

import numpy as np


def shard_units(sizes, world: int, rank: int):
    """Contiguous slice of units (e.g. chains, by stored entries) for `rank`.

    Boundaries split the prefix sum of `sizes` as evenly as possible, so every rank gets
    about the same total work; every unit lands on exactly one rank.
    """
    sizes = np.asarray(sizes, dtype=np.float64)
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    if sizes.size == 0:
        return 0, 0
    cum = np.concatenate(([0.0], np.cumsum(sizes)))
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(cum, total * r / world, side="left")))
    cuts.append(sizes.size)
    cuts = np.maximum.accumulate(np.clip(cuts, 0, sizes.size))
    return int(cuts[rank]), int(cuts[rank + 1])


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks of the default process group (itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
