"""GPU: work plans and the autotuner.

Every plan computes the iteration of Sec. 3; plans differ only in how the
FP32 synthesis sums are grouped, so each one must meet the oracle bars
(max |u - u_oracle| <= 1e-4, relative energy <= 1e-5) and be bitwise
reproducible.  The tuner must leave the iterate exactly as it found it."""

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth
from tests.gpu_util import labels_agree, need_cuda

pytestmark = pytest.mark.gpu

U_TOL = 1e-4
E_TOL = 1e-5


@pytest.fixture(scope="module")
def torch_mod():
    return need_cuda()


def _problem(H, W, K, J, seed):
    rng = np.random.default_rng(seed)
    cb = np.array([[0.2 + 0.6 * k / (K - 1)] for k in range(K)])
    img, _ = synth.ellipse_image(H, W, cb, rng)
    Lam = synth.scale_weights(0.1, J)
    return img.astype(np.float32), cb, Lam.astype(np.float32)


def _run(torch, img, cb, J, Lam, T, plan=None):
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    C, H, W = img.shape
    fb = FilterBank(H, W, J)
    seg = ShearletSegmenter(fb, torch.tensor(img, device="cuda"), cb, Lam.tolist(), 1.0)
    if plan is not None:
        seg.set_plan(plan)
    got_plan = seg.plan()
    seg.step(T)
    seg.synchronize()
    out = {k: seg.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bv", "labels")}
    out["energy"] = seg.energy()
    out["plan"] = got_plan
    seg.close()
    fb.close()
    return out


def _oracle(O, img, cb, J, Lam, T):
    return O.admm_run(img.astype(np.float64), cb.astype(np.float64), J, Lam.astype(np.float64), 1.0, T)


def _check(o, g):
    assert np.abs(g["u"] - o["u"]).max() <= U_TOL
    assert np.abs(g["w"] - o["w"]).max() <= U_TOL
    assert np.abs(g["bv"] - o["bv"]).max() <= U_TOL
    assert abs(g["energy"] - o["energy"]) / abs(o["energy"]) <= E_TOL
    assert labels_agree(g["labels"], o["labels"], o["gap"])


FAST_PLANS = [dict(wave_mib=1, col_ctas_per_sm=1), dict(wave_mib=1, col_ctas_per_sm=0),
              dict(wave_mib=2, col_ctas_per_sm=3), dict(wave_mib=64, col_ctas_per_sm=2),
              dict(wave_mib=4096, col_ctas_per_sm=32),
              dict(wave_mib=64, col_ctas_per_sm=0, sms=40)]  # grids sized for 40 SMs


def test_fast_plans_match_oracle(torch_mod, oracle_mod):
    # 128 x 256, J = 3 (29 filters, 0.13 MiB of spectra per filter): 1 MiB
    # waves give 5 waves per label, 2 MiB 2 waves per label, 64 MiB and 4096
    # MiB one wave of all three labels
    img, cb, Lam = _problem(128, 256, 3, 3, 31)
    T = 12
    o = _oracle(oracle_mod, img, cb, 3, Lam, T)
    for p in FAST_PLANS:
        g = _run(torch_mod, img, cb, 3, Lam, T, p)
        assert g["plan"]["fast"] == 1
        assert g["plan"]["wave_mib"] == p["wave_mib"] and g["plan"]["col_ctas_per_sm"] == p["col_ctas_per_sm"]
        assert g["plan"]["sms"] == p.get("sms", 0)
        _check(o, g)


def test_uneven_label_groups_match_oracle(torch_mod, oracle_mod):
    # 64 x 64, J = 2 (13 filters, 20 KiB of spectra per filter), K = 5: a 1 MiB
    # wave holds 51 planes, i.e. three whole labels, and the labels split into
    # waves of 3 and 2; 4096 MiB puts all five in one wave
    img, cb, Lam = _problem(64, 64, 5, 2, 35)
    T = 15
    o = _oracle(oracle_mod, img, cb, 2, Lam, T)
    for p in (dict(wave_mib=1, col_ctas_per_sm=0), dict(wave_mib=4096, col_ctas_per_sm=1)):
        g = _run(torch_mod, img, cb, 2, Lam, T, p)
        assert g["plan"]["fast"] == 1 and g["plan"]["wave_mib"] == p["wave_mib"]
        _check(o, g)


def test_plan_is_bitwise_reproducible(torch_mod):
    img, cb, Lam = _problem(128, 256, 3, 3, 32)
    for p in (FAST_PLANS[0], FAST_PLANS[2]):
        a = _run(torch_mod, img, cb, 3, Lam, 6, p)
        b = _run(torch_mod, img, cb, 3, Lam, 6, p)
        assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["bv"], b["bv"])


def test_serial_launches_give_the_same_bits(torch_mod):
    # serial = 1 drops programmatic dependent launch: the same kernels in the
    # same order, so the same bits; changing only it recaptures the graphs
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    # the second: 32 values per thread at L = 1024
    for H, W, K, J, extra in ((128, 256, 3, 3, {}), (64, 2048, 2, 1, {"row_kernel": 4})):
        img, cb, Lam = _problem(H, W, K, J, 35)
        fb = FilterBank(H, W, J)
        res = []
        for serial in (0, 1, 2):
            seg = ShearletSegmenter(fb, torch_mod.tensor(img, device="cuda"), cb, Lam.tolist(), 1.0)
            seg.set_plan(dict(seg.plan(), **extra))
            if serial < 2:
                seg.set_plan(dict(seg.plan(), serial=serial))
                assert seg.plan()["serial"] == serial
                seg.step(5)
            else:  # serial from the third iteration on
                seg.step(2)
                seg.set_plan(dict(seg.plan(), serial=1))
                seg.step(3)
                with pytest.raises(B.ShearsegError) as e:
                    seg.set_plan(dict(seg.plan(), serial=2))
                assert e.value.code == B.SHF_ERR_ARG and seg.plan()["serial"] == 1
            seg.synchronize()
            res.append({k: seg.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bv")})
            seg.close()
        fb.close()
        for r in res[1:]:
            for k in ("u", "w", "bv"):
                assert np.array_equal(res[0][k], r[k]), (H, W, k)


def test_general_plans_match_oracle(torch_mod, oracle_mod):
    # 72 x 120 (72 = 9 * 8) is not a register-FFT size: the general kernels
    img, cb, Lam = _problem(72, 120, 3, 2, 33)
    T = 12
    o = _oracle(oracle_mod, img, cb, 2, Lam, T)
    base = _run(torch_mod, img, cb, 2, Lam, T)
    assert base["plan"]["fast"] == 0
    _check(o, base)
    rb = base["plan"]["tile_rows"]
    for p in (dict(tile_cols=4, tile_rows=rb, groups=1), dict(tile_cols=16, tile_rows=max(1, rb // 2), groups=13),
              dict(tile_cols=32, tile_rows=min(72, 2 * rb), groups=5)):
        g = _run(torch_mod, img, cb, 2, Lam, T, p)
        assert g["plan"]["tile_cols"] == p["tile_cols"] and g["plan"]["tile_rows"] == p["tile_rows"]
        _check(o, g)


def test_bad_plans_are_rejected_and_keep_the_old_plan(torch_mod):
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    for H, W, bad in ((64, 64, dict(wave_mib=64, col_ctas_per_sm=-1)), (64, 64, dict(wave_mib=0, col_ctas_per_sm=0)),
                      (64, 64, dict(wave_mib=64, col_ctas_per_sm=33)), (64, 64, dict(sms=-1)),
                      (72, 120, dict(tile_cols=0, tile_rows=1, groups=1)),
                      (72, 120, dict(tile_cols=8, tile_rows=10000, groups=1))):
        img, cb, Lam = _problem(H, W, 3, 2, 34)
        fb = FilterBank(H, W, 2)
        seg = ShearletSegmenter(fb, torch_mod.tensor(img, device="cuda"), cb, Lam.tolist(), 1.0)
        before = seg.plan()
        with pytest.raises(B.ShearsegError):
            seg.set_plan(dict(before, **bad))
        assert seg.plan() == before
        seg.step(2)
        seg.synchronize()
        seg.close()
        fb.close()


@pytest.mark.parametrize("H,W,J", [(256, 256, 3), (96, 160, 2), (72, 120, 2)])
def test_tune_restores_the_iterate_and_keeps_parity(torch_mod, oracle_mod, H, W, J):
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    img, cb, Lam = _problem(H, W, 3, J, 35)
    fb = FilterBank(H, W, J)
    seg = ShearletSegmenter(fb, torch_mod.tensor(img, device="cuda"), cb, Lam.tolist(), 1.0)
    seg.step(4)
    seg.synchronize()
    snap = {k: seg.get(k).cpu().numpy() for k in (B.SEG_BV, B.SEG_W, B.SEG_BW, B.SEG_U)}
    best = seg.tune(2)
    assert best["us_per_iter"] > 0 and np.isfinite(best["us_per_iter"])
    plan = seg.plan()
    for k in ("fast", "wave_mib", "col_ctas_per_sm", "tile_cols", "tile_rows", "groups"):
        assert plan[k] == best[k]
    for k, v in snap.items():
        assert np.array_equal(seg.get(k).cpu().numpy(), v)
    assert int(seg.get(B.SEG_ITER)) == 4
    seg.step(8)
    seg.synchronize()
    u = seg.get(B.SEG_U).cpu().numpy()
    times = B.seg_admm_kernel_times(seg.handle)
    assert all(ms >= 0 for ms, _ in times.values()) and sum(n for _, n in times.values()) > 0
    seg.close()
    fb.close()
    o = _oracle(oracle_mod, img, cb, J, Lam, 12)
    assert np.abs(u - o["u"]).max() <= U_TOL


def test_batch_tune(torch_mod, oracle_mod):
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import ShearletBatch

    shapes = [(64, 64), (72, 120), (64, 64), (96, 160)]
    probs = [_problem(H, W, 3, 2, 40 + i) for i, (H, W) in enumerate(shapes)]
    batch = ShearletBatch([torch_mod.tensor(p[0], device="cuda") for p in probs], [p[1] for p in probs],
                          [p[2].tolist() for p in probs])
    batch.step(3)
    batch.synchronize()
    snap = [{k: batch.image(i).get(k).cpu().numpy() for k in (B.SEG_BV, B.SEG_U)} for i in range(4)]
    batch.tune(2)  # per shape, then the batch-wide SM share: the iterates come back as they were
    plans = [batch.image(i).plan() for i in range(4)]
    assert [p["fast"] for p in plans] == [1, 0, 1, 1]
    assert plans[0] == plans[2]
    assert len({p["sms"] for p in plans if p["fast"]}) == 1
    for i in range(4):
        assert int(batch.image(i).get(B.SEG_ITER)) == 3
        for k, v in snap[i].items():
            assert np.array_equal(batch.image(i).get(k).cpu().numpy(), v), (i, k)
    batch.step(7)
    batch.synchronize()
    for i, p in enumerate(probs):
        u = batch.image(i).get(B.SEG_U).cpu().numpy()
        o = _oracle(oracle_mod, p[0], p[1], 2, p[2], 10)
        assert np.abs(u - o["u"]).max() <= U_TOL
    batch.close()


@pytest.mark.parametrize("H,W,K,J,T", [(512, 128, 3, 2, 6),   # v-step: 8 values, 16 values, pairs (L = 64); columns 8 / 16
                                      (512, 256, 2, 3, 5),   # L = 128: all three row kernels; H = 512: both columns
                                      (1024, 512, 2, 2, 4),  # L = 256: 8 / 16 values; H = 1024: both columns
                                      (96, 384, 3, 2, 12),   # L = 192: 8 / 12 values; H = 96: 8 / 12 values
                                      (64, 640, 2, 2, 6),    # L = 320: 8 / 20 values
                                      (320, 192, 2, 2, 6),   # H = 320: 8 / 20 values; L = 96: 8 / 12 values
                                      (1280, 64, 2, 2, 5),   # H = 1280: columns of 4, 8 / 20 values
                                      (1536, 48, 2, 1, 5),   # H = 1536: 8 / 12 values (128 threads a column)
                                      (48, 2048, 2, 1, 4)])  # L = 1024: 8 / 16 / 32 values; H = 48: 8 / 12 values
def test_every_fft_kernel_variant_meets_the_bars(torch_mod, oracle_mod, H, W, K, J, T):
    # the plan's FFT kernels (row_kernel: 1 eight values per thread, 2 sixteen,
    # 3 pairs of rows, 4 twelve, twenty or thirty-two; col_kernel: 1 eight, 2 sixteen, 3
    # twelve or twenty)
    # change only the order of
    # the FFT arithmetic: each one meets the oracle bars, and the sizes without
    # a variant refuse it
    from paper_1112_1805_gb300 import binding as B

    img, cb, Lam = _problem(H, W, K, J, H + 3 * W)
    o = _oracle(oracle_mod, img, cb, J, Lam, T)
    L = W // 2
    rows = ([1] + ([2] if L in (64, 128, 256, 512, 1024) else []) + ([3] if L in (64, 128) else [])
            + ([4] if L in (24, 40, 48, 80, 96, 160, 192, 320, 384, 640, 1024) else []))
    cols = ([1] + ([2] if H in (512, 1024, 2048) else [])
            + ([3] if H in (24, 40, 48, 80, 96, 160, 192, 320, 384, 640, 768, 1280, 1536) else []))
    seen = set()
    for rk in rows:
        for ck in cols:
            g = _run(torch_mod, img, cb, J, Lam, T, plan={"wave_mib": 64, "col_ctas_per_sm": 0, "row_kernel": rk,
                                                          "col_kernel": ck})
            assert (g["plan"]["row_kernel"], g["plan"]["col_kernel"]) == (rk, ck)
            _check(o, g)
            seen.add((rk, ck))
    assert len(seen) == len(rows) * len(cols)
    for bad in ({"row_kernel": 3} if 3 not in rows else {}, {"row_kernel": 4} if 4 not in rows else {},
                {"col_kernel": 2} if 2 not in cols else {}, {"col_kernel": 3} if 3 not in cols else {},
                {"row_kernel": 7}, {"col_kernel": -1}):
        if not bad:
            continue
        with pytest.raises(B.ShearsegError) as e:
            _run(torch_mod, img, cb, J, Lam, 1, plan=dict({"wave_mib": 64, "col_ctas_per_sm": 0}, **bad))
        assert e.value.code == B.SHF_ERR_ARG
