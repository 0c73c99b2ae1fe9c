"""Image sharding across ranks (host logic; world size 2 over gloo on CPU)."""

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1112_1805_gb300 import shard, synth


def test_lpt_is_a_partition_and_balanced():
    shapes = synth.batch_shapes()
    costs = [shard.image_cost(H, W, K, J) for H, W, K, J in shapes]
    for n in (1, 2, 3, 4, 8):
        bins = shard.lpt_partition(costs, n)
        flat = sorted(i for b in bins for i in b)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in b) for b in bins]
        # LPT bound: makespan <= 4/3 of the optimum, and the optimum >= max(mean, largest item)
        assert max(loads) <= (4 / 3) * max(sum(costs) / n, max(costs)) + 1e-9


def test_lpt_deterministic_and_small_cases():
    assert shard.lpt_partition([5, 5, 5], 2) == [[0, 2], [1]]
    assert shard.lpt_partition([], 3) == [[], [], []]
    assert shard.lpt_partition([1, 2, 3, 4], 1) == [[0, 1, 2, 3]]
    with pytest.raises(ValueError):
        shard.lpt_partition([1], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, shapes, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    solved_here = []

    def solve_one(i):  # stands in for a GPU solve: records where each image ran
        solved_here.append(i)
        H, W, K, J = shapes[i]
        return (i, H * W, rank)

    res = shard.solve_sharded(shapes, solve_one, rank, world)
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([[k, v[1], v[2]] for k, v in sorted(res.items())], dtype=np.int64))
    np.save(os.path.join(out_dir, f"here{rank}.npy"), np.array(sorted(solved_here), dtype=np.int64))
    dist.barrier()
    dist.destroy_process_group()


def test_solve_sharded_gloo_world2(tmp_path):
    shapes = synth.batch_shapes(n=11)
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, shapes, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0, r1 = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    assert np.array_equal(r0, r1)  # every rank sees all results
    assert list(r0[:, 0]) == list(range(11))
    assert all(r0[i, 1] == shapes[i][0] * shapes[i][1] for i in range(11))
    h0, h1 = np.load(tmp_path / "here0.npy"), np.load(tmp_path / "here1.npy")
    assert set(h0).isdisjoint(set(h1)) and sorted(list(h0) + list(h1)) == list(range(11))
    costs = [shard.image_cost(*s) for s in shapes]
    assert [list(h0), list(h1)] == shard.lpt_partition(costs, 2)
    assert all(r0[i, 2] == (0 if i in set(h0) else 1) for i in range(11))


def _problem_set(n=6):
    """Small seeded images of uneven sizes (host arrays) with their codebooks and weights."""
    rng = np.random.default_rng(synth.seed_for(3, 900))
    sides = [(16, 24), (24, 16), (32, 32), (16, 16), (20, 30), (24, 24), (18, 28), (28, 20)]
    shapes, images, cbs, lams = [], [], [], []
    for i in range(n):
        H, W = sides[i % len(sides)]
        K, J = 2 + i % 3, 1 + i % 2
        cb = np.array([[0.2 + 0.6 * k / (K - 1)] for k in range(K)])
        img, _ = synth.ellipse_image(H, W, cb, rng, n_ellipses=3)
        shapes.append((H, W, K, J))
        images.append(img.astype(np.float32))
        cbs.append(cb)
        lams.append(synth.scale_weights(0.1, J))
    return shapes, images, cbs, lams


def _oracle_solver(images, cbs, lams, iters):
    """CPU stand-in for shard.batch_solver with the same signature: each
    image of the share solved by the FP64 oracle; returns label maps."""
    import oracle

    def solve(indices):
        out = {}
        for i in indices:
            o = oracle.admm_run(images[i].astype(np.float64), cbs[i], len(lams[i]) - 1, lams[i], 1.0, iters)
            out[i] = o["labels"]
        return out

    return solve


def _batch_worker(rank, world, port, n, iters, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shapes, images, cbs, lams = _problem_set(n)
    res = shard.solve_batch_sharded(shapes, _oracle_solver(images, cbs, lams, iters), rank, world)
    for i, lab in res.items():
        np.save(os.path.join(out_dir, f"r{rank}_{i}.npy"), lab)
    np.save(os.path.join(out_dir, f"share{rank}.npy"), np.array(shard.share(shapes, rank, world), dtype=np.int64))
    dist.barrier()
    dist.destroy_process_group()


def test_solve_batch_sharded_gloo_world2_real_solves(tmp_path, oracle_mod):
    # the product's sharded batched solve over two gloo ranks on CPU, each rank
    # solving its LPT share for real (the oracle standing in for the GPU
    # batch); every rank gets every label map, equal to a one-process solve
    n, iters = 6, 8
    port = _free_port()
    mp.start_processes(_batch_worker, args=(2, port, n, iters, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    shapes, images, cbs, lams = _problem_set(n)
    ref = _oracle_solver(images, cbs, lams, iters)(list(range(n)))
    for rank in (0, 1):
        for i in range(n):
            assert np.array_equal(np.load(tmp_path / f"r{rank}_{i}.npy"), ref[i]), (rank, i)
    s0, s1 = np.load(tmp_path / "share0.npy"), np.load(tmp_path / "share1.npy")
    assert len(s0) and len(s1) and set(s0).isdisjoint(set(s1)) and sorted(list(s0) + list(s1)) == list(range(n))
