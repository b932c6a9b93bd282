"""Frame sharding across GPUs (one process per GPU).

Frames are independent, so N ranks process N disjoint frame sets and never
exchange frame data; the only collective is the max-over-ranks reduction of
the timing, which a benchmark needs for its whole-job throughput.
"""
from __future__ import annotations

from typing import List


def rank_frame_seeds(rank: int, world: int, per_rank: int, stride: int = 1000) -> List[int]:
    """Seeds of the frames rank `rank` of `world` processes (weak scaling:
    every rank gets `per_rank` frames, disjoint from every other rank's)."""
    if not (0 <= rank < world) or per_rank > stride:
        raise ValueError('rank out of range or per_rank above the seed stride')
    return [stride * rank + i for i in range(per_rank)]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
