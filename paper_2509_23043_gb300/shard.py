"""Host logic of the multi-GPU path: instances shard across ranks, one process per GPU.

Algorithm 1 runs every instance independently: nothing in a sweep, an exchange or a
proposal reads another instance. Each instance's random streams are keyed by its global
instance id, never by the rank or the slot it occupies. So a batch splits across ranks with
no collective in the data path, and every instance's trajectory is the same whatever the
split. The only cross-rank steps are host-side: a barrier around the timed region and the
max of the ranks' times.
"""
from __future__ import annotations

import heapq
from typing import Sequence


def weak_shard(rank: int, world: int, per_rank: int) -> range:
    """Global instance ids of `rank` when every rank runs `per_rank` instances (weak scaling)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return range(rank * per_rank, (rank + 1) * per_rank)


def balanced_shard(costs: Sequence[float], world: int) -> list[list[int]]:
    """Split a ragged batch (strong scaling) over `world` ranks: longest-processing-time
    greedy on the per-instance cost (spin-flip attempts per sweep, R*N). Deterministic, so
    every rank computes the same split without communicating. Returns the ids per rank,
    ascending."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    heap = [(0.0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for k in order:
        load, r = heapq.heappop(heap)
        out[r].append(k)
        heapq.heappush(heap, (load + float(costs[k]), r))
    return [sorted(v) for v in out]


def job_ms(local_ms: float, dist=None, device=None) -> float:
    """The job's time: the slowest rank's (max over ranks of the device-timed milliseconds)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput in units per ns: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e6)
