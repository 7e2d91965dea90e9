"""Multi-GPU form of the Count Sketch: shard the stream, merge by one sum.

A Count Sketch is linear in its stream (Sec. 1.3), so ranks that sketch
disjoint pieces of one stream with the SAME coefficients (same seed) hold
partial sketches whose element-wise int64 sum is the sketch of the whole
stream.  merge_counters_() performs that single exchange -- an all-reduce of
the t*m counters -- with torch.distributed (NCCL for device tensors, gloo for
host tensors).  Nothing else in the path communicates.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def merge_counters_(counters: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum of an int64 counter tensor over all ranks of `group`.
    Integer addition is exact and order independent, so every rank ends with
    the same counters, equal to those of one sketch over the whole stream."""
    if counters.dtype != torch.int64:
        raise TypeError("counters must be int64")
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(counters, op=dist.ReduceOp.SUM, group=group)
    return counters


def merge_sketch_(sketch, group=None):
    """merge_counters_ on a Sketch's own (device) counters, in place."""
    return merge_counters_(sketch.counters(), group)


def shard_range(n: int, rank: int, world: int) -> tuple:
    """[lo, hi) of rank's contiguous piece of an n-element stream."""
    per = (n + world - 1) // world
    lo = min(n, rank * per)
    return lo, min(n, lo + per)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest value over all ranks (a step's wall time is the slowest rank's)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
