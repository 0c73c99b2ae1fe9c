"""Sharding independent segmentation problems across GPUs (one process per GPU).

A single image couples all labels of a pixel (simplex projection) and all
pixels of a filter (FFT), so it is never split; independent images of a batch
are distributed whole.  Images are assigned by longest-processing-time-first
(LPT) greedy on their cost H*W*K*eta*iters; each rank solves its share with no
collective on the data path and the small results (label maps) are gathered at
the end.
"""

from __future__ import annotations

import heapq
from typing import Callable, Sequence


def image_cost(H: int, W: int, K: int, J: int, iters: int = 1) -> int:
    """Work of one image: pixels x labels x filters (eta = 2^(J+2) - 3) x iterations."""
    return H * W * K * ((1 << (J + 2)) - 3) * iters


def lpt_partition(costs: Sequence[float], n_ranks: int) -> list[list[int]]:
    """Assign item indices to n_ranks bins, largest cost first to the least-loaded
    bin (ties: lowest bin index, then lowest item index).  Deterministic."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(n_ranks)]
    heapq.heapify(heap)
    bins: list[list[int]] = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        bins[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    for b in bins:
        b.sort()
    return bins


def solve_sharded(shapes: Sequence[tuple], solve_one: Callable[[int], object], rank: int, world: int,
                  gather: bool = True):
    """Solve the images assigned to `rank` with solve_one(index) and, when
    gather is set and torch.distributed is initialised with world > 1, collect
    {index: result} from every rank on all ranks (results only; no image data
    moves between ranks).  shapes: (H, W, K, J[, iters]) per image."""
    costs = [image_cost(*s) for s in shapes]
    mine = lpt_partition(costs, world)[rank]
    local = {i: solve_one(i) for i in mine}
    if not gather or world == 1:
        return local
    import torch.distributed as dist

    parts: list = [None] * world
    dist.all_gather_object(parts, local)
    merged = {}
    for p in parts:
        merged.update(p)
    return merged
