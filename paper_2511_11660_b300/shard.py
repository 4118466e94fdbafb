"""Sharding independent designs over ranks (host logic only).

A single design is not split: its levels form a chain of dependent steps.
Independent designs (and their corners) are the unit of work: designs are
assigned to ranks by greedy longest-processing-time on their cost (arcs x
corners), each rank times its own batched context, and only the per-design
reports (WNS/TNS scalars) travel, through a host-side gather -- no
collective on the data path.
"""
from __future__ import annotations

import heapq


def lpt_partition(weights, n_ranks: int) -> list:
    """Assign item i (cost weights[i]) to ranks, heaviest first onto the
    currently lightest rank.  Returns one ascending index list per rank."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    heap = [(0.0, r) for r in range(n_ranks)]
    parts = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(weights[i]), r))
    return [sorted(p) for p in parts]


def gather_reports(local: dict, dist=None) -> dict:
    """Merge {design index: report} dicts of every rank on every rank
    (torch.distributed all_gather_object on the default group; identity when
    not distributed)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return dict(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, local)
    out = {}
    for p in parts:
        out.update(p)
    return out
