"""GPU parity: the TV-regularised model of Sec. 4 (eq. TVreg) through the C
ABI against the oracle's trajectory.

Bars as for the shearlet model: max |u - u_oracle| <= 1e-4 (also w, b_w and
b_v), relative energy error <= 1e-5, labels equal wherever the oracle's
top-two gap is at least 1e-4."""

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth
from tests.gpu_util import labels_agree, need_cuda

pytestmark = pytest.mark.gpu

U_TOL = 1e-4
E_TOL = 1e-5


def _r32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _gpu(torch, img, cb, lam, gamma, T, per_label=False, chunks=None):
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import TVSegmenter

    seg = TVSegmenter(torch.tensor(img, dtype=torch.float32, device="cuda"), cb, lam, gamma, per_label)
    for n in chunks or [T]:
        seg.step(n)
    seg.synchronize()
    out = {k: seg.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bw", "bv", "labels")}
    out["energy"] = seg.energy()
    out["iters"] = int(seg.get(B.SEG_ITER))
    seg.close()
    return out


def _check(o, g):
    for k in ("u", "w", "bw", "bv"):
        assert np.abs(g[k] - o[k]).max() <= U_TOL, k
    assert abs(g["energy"] - o["energy"]) / abs(o["energy"]) <= E_TOL
    assert labels_agree(g["labels"], o["labels"], o["gap"])


@pytest.mark.parametrize("H,W,K,C,T,lam,per_label", [
    (64, 64, 3, 1, 200, 0.1, False),   # the 64 x 64 ellipse workload's shape
    (30, 50, 5, 1, 60, 0.08, False),   # radix-3/5 transforms, ragged tiles
    (40, 64, 8, 3, 40, 0.1, False),    # RGB data term, K = 8
    (15, 16, 3, 1, 50, 0.1, False),    # odd H
    (128, 96, 4, 1, 80, 0.1, True),    # per-label groups
    (48, 80, 2, 1, 60, 0.0, False),    # lambda = 0
    (16, 16, 16, 1, 30, 0.05, False),  # K = 16
    # register-FFT u-step (H in 512, 1024, 2048; W/2 in 64..1024): every row
    # group geometry (T = 4 .. 64 threads) and column height
    (512, 128, 3, 1, 30, 0.1, False),
    (1024, 256, 2, 1, 20, 0.1, True),
    (2048, 512, 2, 1, 8, 0.1, False),
    (512, 2048, 2, 1, 8, 0.1, False),
    (512, 1024, 3, 3, 10, 0.08, False),
])
def test_tv_trajectory_matches_oracle(oracle_mod, H, W, K, C, T, lam, per_label):
    torch = need_cuda()
    rng = np.random.default_rng(H * W + K + 3)
    if C == 1:
        cb = np.linspace(0.1, 0.9, K)[:, None]
    else:
        cb = np.array([[a, b, c] for a in (0.2, 0.8) for b in (0.2, 0.8) for c in (0.2, 0.8)])[:K]
    img, _ = synth.ellipse_image(H, W, cb, rng, n_ellipses=4)
    img = img.astype(np.float32)
    lam32 = float(np.float32(lam))
    o = oracle_mod.tv_admm_run(img.astype(np.float64), _r32(cb), lam32, 1.0, T, per_label)
    g = _gpu(torch, img, cb, lam32, 1.0, T, per_label, chunks=[1, T - 1])
    assert g["iters"] == T
    _check(o, g)


def test_tv_one_iteration_from_given_state(oracle_mod):
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import TVSegmenter

    O = oracle_mod
    H, W, K = 24, 40, 3
    rng = np.random.default_rng(17)
    cb = np.array([[0.1], [0.5], [0.9]])
    img = rng.uniform(0, 1, size=(1, H, W)).astype(np.float32)
    lam, gamma = 0.15, 0.7
    st = O.tv_zero_state(K, H, W)
    for key in ("v", "bv", "w", "bw"):
        st[key][...] = (rng.standard_normal(st[key].shape) * 0.3).astype(np.float32)
    s = O.data_term(img.astype(np.float64), _r32(cb))
    seg = TVSegmenter(torch.tensor(img, device="cuda"), cb, lam, gamma)
    seg.set(B.SEG_BV, torch.tensor(st["bv"], dtype=torch.float32))
    seg.set(B.SEG_V, torch.tensor(st["v"], dtype=torch.float32))
    seg.set(B.SEG_W, torch.tensor(st["w"], dtype=torch.float32))
    seg.set(B.SEG_BW, torch.tensor(st["bw"], dtype=torch.float32))
    assert np.abs(seg.get(B.SEG_V).cpu().numpy() - st["v"]).max() <= 1e-6
    for n in (1, 2):
        O.tv_admm_iterate(st, s, float(np.float32(lam)), float(np.float32(gamma)), n)
        seg.step(n)
        seg.synchronize()
        for key, sel in (("u", B.SEG_U), ("w", B.SEG_W), ("bw", B.SEG_BW), ("bv", B.SEG_BV), ("v", B.SEG_V)):
            got = seg.get(sel).cpu().numpy()
            assert np.abs(got - st[key]).max() <= 1e-5, (n, key)
    seg.close()


def test_tv_textured_512_full_run(oracle_mod):
    # the 512 x 512 Bezier/grating image (K = 4) with the TV weights of the
    # paper's stripes and fish runs (gamma = 1, lambda = 1/12, 100 iterations)
    torch = need_cuda()
    img, lab, wl = synth.make_workload_image("bezier512")
    img = img.astype(np.float32)
    cb = wl.codebook()
    lam = float(np.float32(1.0 / 12.0))
    T = 100
    o = oracle_mod.tv_admm_run(img.astype(np.float64), _r32(cb), lam, 1.0, T)
    g = _gpu(torch, img, cb, lam, 1.0, T)
    _check(o, g)
    assert (g["labels"] != lab).mean() < 0.05


def test_tv_reset_repeats_bitwise_and_kernel_times():
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import TVSegmenter

    rng = np.random.default_rng(5)
    cb = np.array([[0.2], [0.5], [0.8]])
    img, _ = synth.ellipse_image(96, 128, cb, rng)
    f = torch.tensor(img.astype(np.float32), device="cuda")
    seg = TVSegmenter(f, cb, 0.1)
    seg.step(25)
    u1 = seg.get(B.SEG_U)
    seg.reset(f)
    seg.step(25)
    assert torch.equal(u1, seg.get(B.SEG_U))
    times = seg.kernel_times(3)
    assert set(times) == {"tv_row_fwd", "tv_col_solve", "tv_row_inv", "tv_prox", "tv_rhs"}
    assert all(v >= 0 for v in times.values()) and times["tv_prox"] > 0 and times["tv_row_fwd"] > 0
    assert int(seg.get(B.SEG_ITER)) == 28
    # a host image through reset gives the same data term
    seg.reset(img.astype(np.float32))
    assert int(seg.get(B.SEG_ITER)) == 0
    seg.close()


def test_tv_argument_errors():
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import TVSegmenter

    f = torch.zeros((1, 32, 32), device="cuda")
    with pytest.raises(B.ShearsegError) as e:
        TVSegmenter(f, np.array([[0.5]]), 0.1)  # K = 1
    assert e.value.code == B.SHF_ERR_ARG
    with pytest.raises(B.ShearsegError) as e:
        TVSegmenter(torch.zeros((1, 32, 14), device="cuda"), np.array([[0.2], [0.8]]), 0.1)  # W/2 = 7
    assert e.value.code == B.SHF_ERR_SIZE
    with pytest.raises(B.ShearsegError) as e:
        TVSegmenter(f, np.array([[0.2], [0.8]]), -1.0)
    assert e.value.code == B.SHF_ERR_ARG
    bad = f.clone()
    bad[0, 3, 3] = float("nan")
    with pytest.raises(B.ShearsegError) as e:
        TVSegmenter(bad, np.array([[0.2], [0.8]]), 0.1)
    assert e.value.code == B.SHF_ERR_NONFINITE
