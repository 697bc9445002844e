"""Host-side logic of multi-GPU runs: one process per GPU, no collective on the data path.

A single scene does not shard (every solver pass would need a halo exchange), so several
GPUs either run independent replicas of a scene or split a batch of independent scenes
between them.  The only communication is the timing reduction at the end of a measured
region: the slowest rank's time and the sum of the particles all ranks stepped.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def shard_scenes(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Split scenes of the given particle counts between `world` ranks, largest first onto
    the least-loaded rank (longest-processing-time greedy; ties to the lower rank).
    Returns, per rank, the sorted indices of its scenes.  Deterministic, so every rank
    computes the same split without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k))
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += int(sizes[k])
    return [sorted(s) for s in out]


def reduce_timing(ms: float, units: float, world: int, device=None) -> Tuple[float, float]:
    """Whole-job timing of a region every rank timed itself: (max over ranks of the
    milliseconds, sum over ranks of the units processed).  With world == 1 no process
    group is needed."""
    if world == 1:
        return float(ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
