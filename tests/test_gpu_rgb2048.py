"""GPU: the 2048 x 2048 RGB workload (K = 8 colours {0.2, 0.8}^3, J = 5, 125
filters, 16.8 GB of b_v in HBM).

A full-size FP64 oracle run does not fit (33 GB of host state, about a minute
per iteration), so, as planned for this workload: oracle parity on crops with
the same K, J and colours (a register-FFT size and a general-path size), and
at full size what holds exactly or at any size: the data term, the first
iterate u = -gamma s / 2 (bitwise), simplex feasibility of w, |b_v| <= gamma
Lambda_j per filter, finite iterates -- with the default plan and with the
one the benchmark's tuner picks (32-value rows, plain launches), whose
iterates agree with the default's to rounding.  Oracle parity of the 32-value
rows themselves: the kernel-variant test at 48 x 2048 (test_gpu_plan.py)."""

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth
from tests.gpu_util import labels_agree, need_cuda

pytestmark = pytest.mark.gpu

U_TOL = 1e-4
E_TOL = 1e-5


@pytest.mark.parametrize("H,W,T", [(256, 256, 15), (72, 120, 10)])
def test_rgb_crop_matches_oracle(oracle_mod, H, W, T):
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    wl = synth.WORKLOADS["rgb2048"]
    cb = wl.codebook()
    rng = np.random.default_rng(synth.seed_for(wl.index, 1))
    img, _ = synth.bezier_texture_image(H, W, cb, rng)
    img = img.astype(np.float32)
    Lam = wl.Lambda().astype(np.float32)
    fb = FilterBank(H, W, wl.J)
    seg = ShearletSegmenter(fb, torch.tensor(img, device="cuda"), cb, Lam.tolist(), wl.gamma)
    assert seg.plan()["fast"] == (1 if H == 256 else 0)
    seg.step(T)
    seg.synchronize()
    g = {k: seg.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "labels")}
    energy = seg.energy()
    seg.close()
    fb.close()
    o = oracle_mod.admm_run(img.astype(np.float64), cb.astype(np.float64), wl.J, Lam.astype(np.float64), wl.gamma, T)
    assert np.abs(g["u"] - o["u"]).max() <= U_TOL
    assert np.abs(g["w"] - o["w"]).max() <= U_TOL
    assert abs(energy - o["energy"]) / abs(o["energy"]) <= E_TOL
    assert labels_agree(g["labels"], o["labels"], o["gap"])


# the default plan, and the one the tuner picks for this image on a GB300 (rows
# of 32 values per thread at half width 1024, plain stream order)
@pytest.mark.parametrize("plan", [{}, {"row_kernel": 4, "serial": 1}])
def test_rgb2048_full_size_properties(plan):
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    img, lab, wl = synth.make_workload_image("rgb2048")
    img = np.ascontiguousarray(img, dtype=np.float32)
    cb = wl.codebook()
    Lam = wl.Lambda()
    fb = FilterBank(wl.H, wl.W, wl.J)
    f = torch.tensor(img, device="cuda")
    seg = ShearletSegmenter(fb, f, cb, Lam.tolist(), wl.gamma)
    assert seg.plan()["fast"] == 1  # H = 2048: register FFTs with column batches of 4
    if plan:
        seg.set_plan(dict(seg.plan(), **plan))
    # data term at sampled pixels
    s = seg.get(B.SEG_S)
    rng = np.random.default_rng(3)
    ys, xs = rng.integers(0, wl.H, 64), rng.integers(0, wl.W, 64)
    s_h = s[:, ys, xs].cpu().numpy().astype(np.float64)
    f_h = img[:, ys, xs].astype(np.float64)
    ref = ((f_h[None, :, :] - cb[:, :, None]) ** 2).sum(axis=1)
    assert np.abs(s_h - ref).max() <= 1e-5
    # first iterate from zero: u = -gamma s / 2, exactly
    seg.step(1)
    seg.synchronize()
    u = seg.get(B.SEG_U)
    assert torch.equal(u, -0.5 * wl.gamma * s)
    seg.step(2)
    seg.synchronize()
    w = seg.get(B.SEG_W)
    assert bool(torch.isfinite(w).all()) and float(w.min()) >= 0.0
    assert float((w.sum(0) - 1.0).abs().max()) <= 1e-5
    u = seg.get(B.SEG_U)
    assert bool(torch.isfinite(u).all())
    bv = seg.get(B.SEG_BV)  # [K][eta][H][W], 16.8 GB on the device
    amax = bv.abs().amax(dim=(0, 2, 3)).cpu().numpy()
    del bv
    # filter f belongs to scale j(f) (f = 0 low-pass): |b_v| <= gamma Lambda_j(f)
    eta = fb.eta
    scale_of = [0]
    for j in range(wl.J):
        n = 2 * (2 * 2**j - 1) + 2
        scale_of += [j + 1] * n
    assert len(scale_of) == eta
    bound = np.array([wl.gamma * Lam[scale_of[f]] for f in range(eta)])
    assert np.all(amax <= bound * (1 + 1e-6) + 1e-12)
    labels = seg.labels().cpu().numpy()
    assert labels.shape == (wl.H, wl.W) and labels.min() >= 0 and labels.max() < wl.K
    seg.close()
    fb.close()


def test_rgb2048_full_size_row_kernels_agree():
    # the 16- and 32-value row transforms at half width 1024 on the full image:
    # the same iteration up to the order of the FP32 FFT arithmetic
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    img, _, wl = synth.make_workload_image("rgb2048")
    f = torch.tensor(np.ascontiguousarray(img, dtype=np.float32), device="cuda")
    fb = FilterBank(wl.H, wl.W, wl.J)
    us = []
    for rk in (2, 4):
        seg = ShearletSegmenter(fb, f, wl.codebook(), wl.Lambda().tolist(), wl.gamma)
        seg.set_plan(dict(seg.plan(), row_kernel=rk))
        seg.step(3)
        seg.synchronize()
        us.append(seg.get(B.SEG_U).clone())
        seg.close()
    fb.close()
    assert float((us[0] - us[1]).abs().max()) <= 1e-5
