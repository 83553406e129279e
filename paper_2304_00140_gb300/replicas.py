"""Multi-process plumbing of the benchmark (host side only).

A single grid does not exchange data between GPUs here: with N processes
each rank advances its own replica of the grid, and a batch of independent
cases is split across ranks by longest-processing-time on cell counts.  The
only collectives are the timing barrier and the max-over-ranks of the
measured time; there is no data-path collective.
"""
from __future__ import annotations

from typing import List, Sequence


def lpt_partition(weights: Sequence[float], nparts: int) -> List[List[int]]:
    """Longest-processing-time split: items in decreasing weight, each to the
    currently lightest part.  Returns the item indices of every part (each
    part's list in increasing index order)."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0.0] * nparts
    parts: List[List[int]] = [[] for _ in range(nparts)]
    for i in order:
        p = min(range(nparts), key=lambda k: (load[k], k))
        parts[p].append(i)
        load[p] += weights[i]
    return [sorted(p) for p in parts]


def max_over_ranks(value: float, dist, device="cpu") -> float:
    """max of a per-rank float over the process group (identity without one)"""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist, device="cpu") -> float:
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
