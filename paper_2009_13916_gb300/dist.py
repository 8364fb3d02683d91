"""Multi-GPU helpers: independent systems are sharded across ranks (one
process per GPU) with no collective on the data path; only the timing (max
over ranks) and the per-system results are exchanged."""
from __future__ import annotations

import numpy as np


def partition_by_weight(weights, world: int, rank: int):
    """Contiguous range [start, end) of items for `rank`, balancing the summed
    weights (e.g. cells per system) across `world` ranks."""
    w = np.asarray(weights, dtype=np.float64)
    if world <= 1:
        return 0, len(w)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        t = total * r / world
        k = int(np.searchsorted(cum, t, side="left"))
        if k > 0 and (k >= len(cum) or t - cum[k - 1] < cum[k] - t):
            k -= 1  # the cut nearest to the balanced target
        cuts.append(k)
    cuts.append(len(w))
    cuts = np.maximum.accumulate(np.minimum(cuts, len(w)))
    return int(cuts[rank]), int(cuts[rank + 1])


def max_over_ranks(value: float) -> float:
    """Max of a scalar over the ranks of the default process group (identity
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_objects(obj):
    """All ranks' objects in rank order (single-element list without a group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out
