"""GPU parity: the ADMM through the C ABI vs the oracle's trajectory.

Bars (stated for the FP32 path against the FP64 oracle): max |u - u_oracle|
<= 1e-4, relative energy error <= 1e-5, and label maps equal except at pixels
whose top-two gap in the oracle is below 1e-4."""

import os

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth
from tests.gpu_util import labels_agree, need_cuda, rel_max_err

pytestmark = pytest.mark.gpu

U_TOL = 1e-4
E_TOL = 1e-5


@pytest.fixture(scope="module")
def torch_mod():
    return need_cuda()


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _gpu_run(torch, img, cb, J, Lam, gamma, T, chunks=None):
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    C, H, W = img.shape
    fb = FilterBank(H, W, J)
    seg = ShearletSegmenter(fb, torch.tensor(img, dtype=torch.float32, device="cuda"), cb, Lam, gamma)
    for n in chunks or [T]:
        seg.step(n)
    seg.synchronize()
    out = {k: seg.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bw", "bv", "labels", "gap")}
    out["energy"] = seg.energy()
    seg.close()
    fb.close()
    return out


def _check_against(o, g, check_bv=True):
    assert np.abs(g["u"] - o["u"]).max() <= U_TOL
    assert np.abs(g["w"] - o["w"]).max() <= U_TOL
    assert np.abs(g["bw"] - o["bw"]).max() <= U_TOL
    if check_bv:
        assert np.abs(g["bv"] - o["bv"]).max() <= U_TOL
    assert abs(g["energy"] - o["energy"]) / abs(o["energy"]) <= E_TOL
    assert labels_agree(g["labels"], o["labels"], o["gap"])


def test_ellipses64_full_trajectory(torch_mod, O):
    # 64 x 64, K = 3, codebook {0.2, 0.5, 0.8}, J = 2, 200 iterations.
    img, lab, wl = synth.make_workload_image("ellipses64")
    cb = wl.codebook()
    o = O.admm_run(img.astype(np.float32).astype(np.float64), cb.astype(np.float32).astype(np.float64), wl.J,
                   wl.Lambda().astype(np.float32).astype(np.float64), wl.gamma, wl.iters)
    g = _gpu_run(torch_mod, img, cb, wl.J, wl.Lambda(), wl.gamma, wl.iters, chunks=[1, 49, 150])
    _check_against(o, g)
    assert (g["labels"] != lab).mean() < 0.02


@pytest.mark.parametrize("H,W,K,J,C,T", [(48, 80, 2, 1, 1, 40), (30, 50, 5, 2, 1, 30), (40, 64, 8, 2, 3, 25),
                                        (16, 16, 16, 1, 1, 20), (96, 96, 4, 3, 1, 15), (15, 16, 3, 1, 1, 20),
                                        (8, 16, 3, 1, 1, 20), (32, 256, 4, 2, 1, 15), (256, 64, 3, 3, 1, 10),
                                        (128, 128, 6, 3, 3, 10)])
def test_edge_shapes(torch_mod, O, H, W, K, J, C, T):
    # ragged tiles (odd H, W/2 not a multiple of the tile), K from 2 to 16, RGB;
    # power-of-two shapes take the register-FFT path (8 <= H <= 1024, W <= 2048).
    rng = np.random.default_rng(H * W + K)
    if C == 1:
        cb = np.linspace(0.1, 0.9, K)[:, None]
        img, lab = synth.ellipse_image(H, W, cb, rng)
    else:
        cb = np.array([[a, b, c] for a in (0.2, 0.8) for b in (0.2, 0.8) for c in (0.2, 0.8)])[:K]
        img, lab = synth.ellipse_image(H, W, cb, rng, n_ellipses=4)
    Lam = synth.scale_weights(0.1, J)
    img32 = img.astype(np.float32)
    o = O.admm_run(img32.astype(np.float64), cb.astype(np.float32).astype(np.float64), J,
                   Lam.astype(np.float32).astype(np.float64), 1.0, T)
    g = _gpu_run(torch_mod, img32, cb, J, Lam, 1.0, T)
    _check_against(o, g)


@pytest.mark.parametrize("H,W,K,J,T", [(16, 128, 3, 1, 12), (24, 256, 4, 2, 12), (16, 512, 3, 2, 10),
                                      (8, 1024, 2, 1, 10), (16, 2048, 3, 1, 8), (40, 2048, 2, 2, 6)])
def test_radix16_row_widths(torch_mod, O, H, W, K, J, T):
    # half widths L = 64 .. 1024 take the v-step with 16 values per thread
    # (L = 1024: row groups of two warps with a named barrier); a ragged
    # number of rows per launch leaves some row groups without a row
    rng = np.random.default_rng(H * W + 7 * K)
    cb = np.linspace(0.15, 0.85, K)[:, None]
    img, lab = synth.ellipse_image(H, W, cb, rng, n_ellipses=3)
    Lam = synth.scale_weights(0.1, J)
    img32 = img.astype(np.float32)
    o = O.admm_run(img32.astype(np.float64), cb.astype(np.float32).astype(np.float64), J,
                   Lam.astype(np.float32).astype(np.float64), 1.0, T)
    g = _gpu_run(torch_mod, img32, cb, J, Lam, 1.0, T)
    _check_against(o, g)


def test_one_iteration_from_given_state(torch_mod, O):
    # Start both sides from the same arbitrary (v, b_v, w, b_w): every term of the
    # u-, v-, w- and b-updates is exercised from the first iteration on.
    torch = torch_mod
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    H, W, K, J = 40, 48, 3, 2
    rng = np.random.default_rng(21)
    cb = np.array([[0.1], [0.5], [0.9]])
    img = rng.uniform(0, 1, size=(1, H, W)).astype(np.float32)
    Lam = np.array([0.05, 0.1, 0.2], dtype=np.float32)
    gamma = 0.8
    st = O.zero_state(K, J, H, W)
    for key in ("v", "bv", "w", "bw"):
        st[key][...] = (rng.standard_normal(st[key].shape) * 0.3).astype(np.float32)
    s = O.data_term(img.astype(np.float64), cb.astype(np.float32).astype(np.float64))
    fb = FilterBank(H, W, J)
    seg = ShearletSegmenter(fb, torch.tensor(img, device="cuda"), cb, Lam, gamma)
    seg.set(B.SEG_BV, torch.tensor(st["bv"], dtype=torch.float32))
    seg.set(B.SEG_V, torch.tensor(st["v"], dtype=torch.float32))
    seg.set(B.SEG_W, torch.tensor(st["w"], dtype=torch.float32))
    seg.set(B.SEG_BW, torch.tensor(st["bw"], dtype=torch.float32))
    for n in (1, 2):
        O.admm_iterate(st, s, J, Lam.astype(np.float64), gamma, n)
        seg.step(n)
        seg.synchronize()
        for key, sel in (("u", B.SEG_U), ("w", B.SEG_W), ("bw", B.SEG_BW), ("bv", B.SEG_BV)):
            got = seg.get(sel).cpu().numpy()
            assert np.abs(got - st[key]).max() <= 1e-5, (n, key)
        # the carried synthesis S^T(v - b_v)
        stv = seg.get(B.SEG_STV).cpu().numpy()
        assert np.abs(stv - O.synthesize(st["v"] - st["bv"], J)).max() <= 1e-5


def test_bezier512_first_iterations(torch_mod, O):
    # Full-size workload (512 x 512, K = 4, J = 4, eta = 61) in the benchmark's
    # launch configuration: the first 3 iterations element by element.
    img, lab, wl = synth.make_workload_image("bezier512")
    cb = wl.codebook()
    T = 3
    img32 = img.astype(np.float32)
    o = O.admm_run(img32.astype(np.float64), cb.astype(np.float32).astype(np.float64), wl.J,
                   wl.Lambda().astype(np.float32).astype(np.float64), wl.gamma, T)
    g = _gpu_run(torch_mod, img32, cb, wl.J, wl.Lambda(), wl.gamma, T)
    _check_against(o, g)


def test_large_multiwave_first_iterations(torch_mod, O):
    # 1024 x 1024, J = 3: the filters of a label are processed in several waves
    # whose partial sums accumulate; first 2 iterations element by element.
    H = W = 1024
    K, J, T = 2, 3, 2
    rng = np.random.default_rng(77)
    cb = np.array([[0.3], [0.7]])
    img, lab = synth.ellipse_image(H, W, cb, rng)
    Lam = synth.scale_weights(0.1, J)
    img32 = img.astype(np.float32)
    o = O.admm_run(img32.astype(np.float64), cb.astype(np.float64), J, Lam.astype(np.float32).astype(np.float64),
                   1.0, T)
    g = _gpu_run(torch_mod, img32, cb, J, Lam, 1.0, T)
    _check_against(o, g)


def test_bezier512_full_run_properties(torch_mod, O):
    # 500 iterations at full size: properties that hold at any iteration count.
    torch = torch_mod
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    img, lab, wl = synth.make_workload_image("bezier512")
    cb = wl.codebook()
    fb = FilterBank(wl.H, wl.W, wl.J)
    seg = ShearletSegmenter(fb, torch.tensor(img, dtype=torch.float32, device="cuda"), cb, wl.Lambda(), wl.gamma)
    seg.step(1)
    e1 = seg.energy()
    seg.step(wl.iters - 1)
    seg.synchronize()
    w = seg.get(B.SEG_W)
    assert float(w.min()) >= 0.0
    assert float((w.sum(0) - 1).abs().max()) < 1e-5
    bv = seg.get(B.SEG_BV)
    thr = torch.tensor(O.thresholds(wl.J, wl.Lambda(), wl.gamma), dtype=torch.float32, device="cuda")
    assert bool((bv.abs() <= thr[None, :, None, None] * (1 + 1e-6)).all())
    e = seg.energy()
    assert e < e1
    # the ADMM residual u - w has become small
    assert float((seg.get(B.SEG_U) - w).abs().max()) < 0.05
    labels = seg.labels().cpu().numpy()
    assert (labels != lab).mean() < 0.05
    assert np.isfinite(e)


def test_checkpoint_resume_bitwise(torch_mod, tmp_path):
    torch = torch_mod
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    img, lab, wl = synth.make_workload_image("ellipses64")
    fb = FilterBank(wl.H, wl.W, wl.J)
    f = torch.tensor(img, dtype=torch.float32, device="cuda")
    a = ShearletSegmenter(fb, f, wl.codebook(), wl.Lambda(), wl.gamma)
    a.step(30)
    path = os.path.join(str(tmp_path), "ck.bin")
    a.save(path)
    a.step(20)
    b = ShearletSegmenter(fb, f, wl.codebook(), wl.Lambda(), wl.gamma)
    b.load(path)
    assert int(b.get(B.SEG_ITER)) == 30
    b.step(20)
    for sel in (B.SEG_U, B.SEG_W, B.SEG_BW, B.SEG_BV):
        assert torch.equal(a.get(sel), b.get(sel))


def test_deterministic_and_reset(torch_mod):
    torch = torch_mod
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    img, lab, wl = synth.make_workload_image("ellipses64")
    fb = FilterBank(wl.H, wl.W, wl.J)
    f = torch.tensor(img, dtype=torch.float32, device="cuda")
    a = ShearletSegmenter(fb, f, wl.codebook(), wl.Lambda(), wl.gamma)
    a.step(40)
    u1 = a.get(B.SEG_U)
    a.reset(img.astype(np.float32))  # host image
    a.step(40)
    assert torch.equal(u1, a.get(B.SEG_U))
    assert int(a.get(B.SEG_ITER)) == 40


def test_solve_stops_on_tolerance(torch_mod):
    torch = torch_mod
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    img, lab, wl = synth.make_workload_image("ellipses64")
    fb = FilterBank(wl.H, wl.W, wl.J)
    seg = ShearletSegmenter(fb, torch.tensor(img, dtype=torch.float32, device="cuda"), wl.codebook(), wl.Lambda(),
                            wl.gamma, max_iters=400, tol=1e-3, check_every=10)
    it, res = seg.solve()
    assert it < 400 and res < 1e-3 and it % 10 == 0


def test_nonfinite_and_bad_arguments(torch_mod):
    torch = torch_mod
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    fb = FilterBank(32, 32, 2)
    f = torch.rand((1, 32, 32), device="cuda")
    f[0, 3, 4] = float("nan")
    with pytest.raises(B.ShearsegError) as ei:
        ShearletSegmenter(fb, f, [[0.2], [0.8]], [0, 0.01, 0.02])
    assert ei.value.code == B.SHF_ERR_NONFINITE
    with pytest.raises(B.ShearsegError) as ei:
        ShearletSegmenter(fb, torch.rand((1, 32, 32), device="cuda"), [[0.2]], [0, 0.01, 0.02])  # K = 1
    assert ei.value.code == B.SHF_ERR_ARG
    params, keep = B.make_params(1.0, 3, [0, 0.01, 0.02, 0.04])  # J = 3 against a J = 2 bank
    g = torch.rand((1, 32, 32), device="cuda")
    with pytest.raises(B.ShearsegError) as ei:
        B.seg_admm_init(fb.handle, g.data_ptr(), 1, [0.2, 0.8], 2, params)
    assert ei.value.code == B.SHF_ERR_STATE
    with pytest.raises(ValueError):
        B.make_params(1.0, 2, [0, 0.01])
