"""Replica bookkeeping for runs on several GPUs (one process per GPU, no data-path collective).

Shots are independent, so N GPUs run N replicas of the same pipeline on disjoint shot ranges.
The only exchanges are at the end of a timed region, on the host side of torch.distributed
(NCCL between GPUs, gloo on CPU): the maximum of the per-rank elapsed times, and sums of
failure and iteration counts.
"""
from __future__ import annotations

import torch


def shot_offset(step: int, rank: int, world: int, p_index: int, n_p: int, shots_per_p: int) -> int:
    """First absolute shot index of (step, rank, p): every (step, rank, p) owns a disjoint range
    of shots_per_p indices, and together they tile 0 .. steps*world*n_p*shots_per_p - 1."""
    return ((step * world + rank) * n_p + p_index) * shots_per_p


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world <= 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(values, world: int, device=None):
    """Element-wise sum of integer counts over the ranks."""
    if world <= 1:
        return [int(v) for v in values]
    t = torch.tensor([int(v) for v in values], dtype=torch.int64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return [int(v) for v in t.tolist()]
