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


def share(shapes: Sequence[tuple], rank: int, world: int) -> list[int]:
    """Indices of the images rank `rank` of `world` solves: its LPT bin of the
    costs image_cost(H, W, K, J[, iters])."""
    return lpt_partition([image_cost(*s) for s in shapes], world)[rank]


def gather_results(local: dict, world: int) -> dict:
    """{index: result} of every rank on every rank (torch.distributed object
    all-gather; the identity for one rank)."""
    if world == 1:
        return dict(local)
    import torch.distributed as dist

    parts: list = [None] * world
    dist.all_gather_object(parts, local)
    merged = {}
    for p in parts:
        merged.update(p)
    return merged


def batch_solver(images, codebooks, Lambdas, gammas, iters: int, tune: bool = False):
    """The GPU solver of a rank's share: solver(indices) builds one
    ShearletBatch (one CUDA graph per iteration over the share's images) on
    the current device from the host images [C, H, W] (or [H, W]), runs
    `iters` iterations and returns {index: label map (int32 numpy)}."""

    def solve(indices):
        if not indices:
            return {}
        import numpy as np
        import torch

        from .api import ShearletBatch

        imgs = [torch.as_tensor(np.ascontiguousarray(images[i], dtype=np.float32)).cuda() for i in indices]
        g = gammas if isinstance(gammas, (int, float)) else [gammas[i] for i in indices]
        batch = ShearletBatch(imgs, [codebooks[i] for i in indices], [Lambdas[i] for i in indices], g)
        try:
            if tune:
                batch.tune(5)
            batch.step(iters)
            batch.synchronize()
            return {i: batch.image(j).labels().cpu().numpy() for j, i in enumerate(indices)}
        finally:
            batch.close()

    return solve


def solve_batch_sharded(shapes: Sequence[tuple], solver: Callable[[list], dict], rank: int, world: int,
                        gather: bool = True) -> dict:
    """The sharded batched solve: rank `rank` solves its LPT share with
    solver(indices) -> {index: result} (batch_solver on a GPU) and, with
    gather, every rank receives every result.  No image data moves between
    ranks; only the results are gathered."""
    local = solver(share(shapes, rank, world))
    return gather_results(local, world) if gather else local


def solve_sharded(shapes: Sequence[tuple], solve_one: Callable[[int], object], rank: int, world: int,
                  gather: bool = True):
    """Solve the images assigned to `rank` with solve_one(index) and, when
    gather is set and torch.distributed is initialised with world > 1, collect
    {index: result} from every rank on all ranks (results only; no image data
    moves between ranks).  shapes: (H, W, K, J[, iters]) per image."""
    local = {i: solve_one(i) for i in share(shapes, rank, world)}
    return gather_results(local, world) if gather else local
