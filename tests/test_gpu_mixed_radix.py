"""GPU: the register-FFT path at heights and half widths 3 * 2^a and 5 * 2^a
against the oracle's trajectory (bars: max |u - u_oracle| <= 1e-4, relative
energy <= 1e-5, labels equal except at top-two gaps below 1e-4).

These sizes cover every radix-R first pass (R = 3, 5) of both the column
transforms (height H) and the packed row transforms (L = W/2), the row-group
layouts (L/8 threads that divide a warp, span whole warps, or are packed
across warps), the mixed spans of the later passes, and heights above 1024
(column batches of 4)."""

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth
from tests.gpu_util import labels_agree, need_cuda

pytestmark = pytest.mark.gpu

U_TOL = 1e-4
E_TOL = 1e-5


def _problem(H, W, K, J, seed, C=1):
    rng = np.random.default_rng(seed)
    if C == 1:
        cb = np.array([[0.2 + 0.6 * k / (K - 1)] for k in range(K)])
    else:
        cb = np.array([[0.2, 0.2, 0.8], [0.8, 0.2, 0.2], [0.2, 0.8, 0.5], [0.7, 0.7, 0.2], [0.5, 0.5, 0.5]])[:K]
    img, _ = synth.ellipse_image(H, W, cb, rng)
    return img.astype(np.float32), cb, synth.scale_weights(0.1, J).astype(np.float32)


def _run(torch, img, cb, J, Lam, T):
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    C, H, W = img.shape
    fb = FilterBank(H, W, J)
    seg = ShearletSegmenter(fb, torch.tensor(img, device="cuda"), cb, Lam.tolist(), 1.0)
    plan = seg.plan()
    seg.step(T)
    seg.synchronize()
    out = {k: seg.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bv", "labels")}
    out["energy"] = seg.energy()
    seg.close()
    fb.close()
    return plan, out


SHAPES = [
    # H, W, K, J, C, T
    (24, 48, 3, 1, 1, 10),     # H = 3*8, L = 24 = 3*8 (3-thread row groups)
    (40, 80, 4, 2, 1, 10),     # H = 5*8, L = 40 = 5*8 (5-thread row groups)
    (96, 160, 3, 2, 1, 10),    # H = 3*32, L = 80 = 5*16
    (160, 96, 2, 2, 3, 8),     # H = 5*32, L = 48 = 3*16, RGB
    (192, 384, 5, 3, 1, 5),    # H = 3*64, L = 192 = 3*64 (24-thread groups)
    (320, 640, 4, 3, 1, 3),    # H = 5*64, L = 320 = 5*64 (40-thread groups over 2 warps)
    (384, 768, 3, 3, 1, 3),    # H = 3*128, L = 384 (48-thread groups)
    (128, 1536, 2, 3, 1, 3),   # L = 768 = 3*256 (96-thread groups over 3 warps)
    (640, 80, 6, 2, 1, 4),     # H = 5*128, K = 6
    (2048, 64, 2, 2, 1, 3),    # H = 2048: column batches of 4
    (1536, 80, 3, 2, 1, 3),    # H = 3*512, batches of 4
    (1280, 48, 2, 1, 3, 4),    # H = 5*256, batches of 4, RGB
]


@pytest.mark.parametrize("H,W,K,J,C,T", SHAPES)
def test_mixed_radix_matches_oracle(oracle_mod, H, W, K, J, C, T):
    torch = need_cuda()
    img, cb, Lam = _problem(H, W, K, J, H * 7 + W, C)
    plan, g = _run(torch, img, cb, J, Lam, T)
    assert plan["fast"] == 1
    o = oracle_mod.admm_run(img.astype(np.float64), cb.astype(np.float64), J, Lam.astype(np.float64), 1.0, T)
    assert np.abs(g["u"] - o["u"]).max() <= U_TOL
    assert np.abs(g["w"] - o["w"]).max() <= U_TOL
    assert np.abs(g["bv"] - o["bv"]).max() <= U_TOL
    assert abs(g["energy"] - o["energy"]) / abs(o["energy"]) <= E_TOL
    assert labels_agree(g["labels"], o["labels"], o["gap"])


def test_unsupported_sizes_take_the_general_path():
    torch = need_cuda()
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    for H, W in ((72, 120), (30, 50), (1152, 64)):
        img, cb, Lam = _problem(H, W, 3, 2, 5)
        fb = FilterBank(H, W, 2)
        seg = ShearletSegmenter(fb, torch.tensor(img, device="cuda"), cb, Lam.tolist(), 1.0)
        assert seg.plan()["fast"] == 0
        seg.close()
        fb.close()
