"""GPU: batched solves of independent images of uneven sizes (one CUDA graph
per iteration, one branch per image) against single-image runs and the oracle."""

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth
from tests.gpu_util import labels_agree, need_cuda

pytestmark = pytest.mark.gpu


def _images(shapes, seed):
    rng = np.random.default_rng(seed)
    out = []
    for H, W, K, J, C in shapes:
        if C == 1:
            cb = np.array([[0.2 + 0.6 * k / (K - 1)] for k in range(K)])
        else:
            cb = np.array([[a, b, c] for a in (0.2, 0.8) for b in (0.2, 0.8) for c in (0.2, 0.8)])[:K]
        img, lab = synth.ellipse_image(H, W, cb, rng, n_ellipses=4)
        out.append((img.astype(np.float32), cb, synth.scale_weights(0.1, J)))
    return out


def _single(torch, img, cb, Lam, T):
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    fb = FilterBank(img.shape[1], img.shape[2], len(Lam) - 1)
    seg = ShearletSegmenter(fb, torch.tensor(img, device="cuda"), cb, Lam, 1.0)
    seg.step(T)
    seg.synchronize()
    out = {k: seg.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bv")}
    seg.close()
    fb.close()
    return out


def test_batch_equals_single_runs_and_oracle(oracle_mod):
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import ShearletBatch

    shapes = [(64, 96, 2, 2, 1), (48, 80, 3, 1, 1), (32, 32, 4, 2, 1), (40, 64, 3, 2, 3), (30, 50, 5, 2, 1)]
    data = _images(shapes, 42)
    T = 25
    batch = ShearletBatch([torch.tensor(d[0], device="cuda") for d in data], [d[1] for d in data],
                          [d[2] for d in data], 1.0)
    batch.step(T)
    batch.synchronize()
    for i, (img, cb, Lam) in enumerate(data):
        view = batch.image(i)
        got = {k: view.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bv")}
        ref = _single(torch, img, cb, Lam, T)
        for k in got:  # same kernels in the same order: bit-identical
            assert np.array_equal(got[k], ref[k]), (i, k)
        o = oracle_mod.admm_run(img.astype(np.float64), cb.astype(np.float32).astype(np.float64), len(Lam) - 1,
                                Lam.astype(np.float32).astype(np.float64), 1.0, T)
        assert np.abs(got["u"] - o["u"]).max() <= 1e-4, i
        lab = view.labels().cpu().numpy()
        assert labels_agree(lab, o["labels"], o["gap"]), i
    assert int(batch.image(0).get(B.SEG_ITER)) == T
    batch.close()


def test_uneven_batch_shapes_first_iterations():
    # the uneven batch of the batched workload (384 x 640 first, sides from
    # 128 to 1024, K from 2 to 6, J = floor(log2(min side)/2)), first 12 images
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import ShearletBatch

    shp = synth.batch_shapes()[:12]
    data = _images([(H, W, K, J, 1) for H, W, K, J in shp], synth.seed_for(3))
    T = 3
    batch = ShearletBatch([torch.tensor(d[0], device="cuda") for d in data], [d[1] for d in data],
                          [d[2] for d in data], 1.0)
    batch.step(T)
    batch.synchronize()
    for i in (0, 1, 5, 11):
        img, cb, Lam = data[i]
        ref = _single(torch, img, cb, Lam, T)
        got = batch.image(i).get(B.SEG_U).cpu().numpy()
        assert np.array_equal(got, ref["u"]), i
    for i in range(len(data)):
        w = batch.image(i).get(B.SEG_W)
        assert float(w.min()) >= 0 and float((w.sum(0) - 1).abs().max()) < 1e-5
    batch.close()


def test_lanes_give_the_same_bits():
    # the images chained into two or three lanes run the same kernels on the
    # same buffers as with every image in a lane of its own
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import ShearletBatch

    data = _images([(64, 96, 2, 2, 1), (48, 80, 3, 1, 1), (32, 32, 4, 2, 1), (40, 64, 3, 2, 3), (96, 128, 3, 2, 1)], 9)
    res = []
    for lanes in (0, 2, 3, 7):
        batch = ShearletBatch([torch.tensor(d[0], device="cuda") for d in data], [d[1] for d in data],
                              [d[2] for d in data], 1.0)
        batch.lanes = lanes
        assert batch.lanes == lanes
        batch.step(4)
        if lanes == 2:  # a change between steps: the graph is captured again
            batch.lanes = 1
        batch.step(4)
        batch.synchronize()
        res.append([{k: batch.image(i).get(getattr(B, "SEG_" + k)).cpu().numpy() for k in ("U", "BV")}
                    for i in range(len(data))])
        if lanes == 7:
            with pytest.raises(B.ShearsegError) as e:
                batch.lanes = -1
            assert e.value.code == B.SHF_ERR_ARG
        batch.close()
    for r in res[1:]:
        for i in range(len(data)):
            for k in ("U", "BV"):
                assert np.array_equal(res[0][i][k], r[i][k]), (i, k)


def test_sharded_batch_solver_on_one_rank(oracle_mod):
    # the product's sharded batched solve (shard.solve_batch_sharded with the
    # GPU batch solver) on one rank: the label maps of every image, against
    # the oracle's after the same number of iterations
    need_cuda()
    from paper_1112_1805_gb300 import shard

    shapes5 = [(64, 96, 2, 2, 1), (48, 80, 3, 1, 1), (32, 32, 4, 2, 1), (30, 50, 5, 2, 1), (40, 64, 3, 2, 1)]
    data = _images(shapes5, 77)
    T = 20
    shapes = [(H, W, K, J) for H, W, K, J, _ in shapes5]
    solver = shard.batch_solver([d[0] for d in data], [d[1] for d in data], [d[2] for d in data], 1.0, T)
    res = shard.solve_batch_sharded(shapes, solver, 0, 1)
    assert sorted(res) == list(range(len(shapes)))
    for i, (img, cb, Lam) in enumerate(data):
        o = oracle_mod.admm_run(img.astype(np.float64), cb.astype(np.float32).astype(np.float64), len(Lam) - 1,
                                Lam.astype(np.float32).astype(np.float64), 1.0, T)
        assert labels_agree(res[i], o["labels"], o["gap"]), i


def test_member_plan_change_rebuilds_the_batch_graphs():
    # a new plan for one image reallocates its work buffers: the batch's
    # graphs (which hold the old ones) are rebuilt before the next step, and
    # the results equal a batch that ran the same plans throughout
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import ShearletBatch

    data = _images([(64, 128, 3, 2, 1), (48, 64, 2, 2, 1)], 7)

    def make():
        return ShearletBatch([torch.tensor(d[0], device="cuda") for d in data], [d[1] for d in data],
                             [d[2] for d in data], 1.0)

    a = make()
    a.step(12)
    p = B.seg_admm_get_plan(a.image(0).handle)
    assert p["fast"] == 1
    p["wave_mib"] = 1  # one filter per wave
    B.seg_admm_set_plan(a.image(0).handle, p)
    a.step(13)
    a.synchronize()
    b = make()
    B.seg_admm_set_plan(b.image(0).handle, p)
    b.step(12)
    b.step(13)
    b.synchronize()
    for i in range(2):
        ua = a.image(i).get(B.SEG_U).cpu().numpy()
        ub = b.image(i).get(B.SEG_U).cpu().numpy()
        assert np.abs(ua - ub).max() <= 1e-5, i  # plans group the sums differently for 12 iterations
        assert np.isfinite(ua).all()
    a.close()
    b.close()
