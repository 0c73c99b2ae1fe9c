"""GPU parity: the NL-means-regularised model of Sec. 4 through the C ABI
against the oracle.

The neighbour graph is integer work decided by floating point: both sides
compute the patch distances in FP64 with every operation rounded separately
and the same order, so the graphs must be identical.  The iterations: max
|u - u_oracle| <= 1e-4 (also w, b_w and b_v), relative energy error <= 1e-5,
labels equal wherever the oracle's top-two gap is at least 1e-4 (the oracle
solves the u-step exactly by conjugate gradients, the GPU by Chebyshev
iterations to a relative error of 1e-7)."""

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth
from tests.gpu_util import labels_agree, need_cuda

pytestmark = pytest.mark.gpu

U_TOL = 1e-4
E_TOL = 1e-5


def _r32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _image(H, W, K, C, seed, sigma=0.05):
    rng = np.random.default_rng(seed)
    if C == 1:
        cb = np.linspace(0.15, 0.85, K)[:, None]
    else:
        cb = np.array([[a, b, c] for a in (0.2, 0.8) for b in (0.2, 0.8) for c in (0.2, 0.8)])[:K]
    img, lab = synth.ellipse_image(H, W, cb, rng, sigma=sigma, n_ellipses=4)
    return img.astype(np.float32), cb, lab


@pytest.mark.parametrize("H,W,K,C,prm", [
    (64, 64, 3, 1, {}),                                   # the paper's p = 5, varpi = 15, a = 2, mt = 5
    (30, 50, 4, 1, {}),
    (40, 64, 5, 3, {}),                                   # RGB distances
    (24, 36, 3, 1, {"patch": 3, "window": 7, "a": 1.0, "neighbours": 3}),
])
def test_nl_graph_identical_to_oracle(oracle_mod, H, W, K, C, prm):
    torch = need_cuda()
    from paper_1112_1805_gb300.api import NLSegmenter

    img, cb, _ = _image(H, W, K, C, H * W + C)
    seg = NLSegmenter(torch.tensor(img, device="cuda"), cb, 0.05, 0.2, **prm)
    nbr, deg, steps = seg.graph()
    seg.close()
    onbr, odeg = oracle_mod.nl_graph(img.astype(np.float64), p=prm.get("patch", 5), win=prm.get("window", 15),
                                     a=prm.get("a", 2.0), mt=prm.get("neighbours", 5))
    assert np.array_equal(deg, odeg)
    assert np.array_equal(nbr, onbr)
    assert steps > 0 and steps % 2 == 0


@pytest.mark.parametrize("H,W,K,C,T,lam,gamma", [
    (64, 64, 3, 1, 100, 1 / 32, 0.2),     # the paper's fish weights: gamma = 1/5, lambda = 1/32, 100 iterations
    (30, 50, 4, 1, 60, 1 / 16, 0.2),
    (40, 64, 5, 3, 40, 1 / 32, 0.2),
    (48, 48, 2, 1, 50, 0.0, 0.5),         # lambda = 0
    (16, 24, 16, 1, 25, 1 / 32, 0.2),     # K = 16
])
def test_nl_trajectory_matches_oracle(oracle_mod, H, W, K, C, T, lam, gamma):
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import NLSegmenter

    img, cb, _ = _image(H, W, K, C, 7 * H + W + K)
    lam32, g32 = float(np.float32(lam)), float(np.float32(gamma))
    seg = NLSegmenter(torch.tensor(img, device="cuda"), cb, lam32, g32)
    seg.step(1)
    seg.step(T - 1)
    seg.synchronize()
    got = {k: seg.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bw", "bv", "labels")}
    energy = seg.energy()
    assert int(seg.get(B.SEG_ITER)) == T
    seg.close()
    o = oracle_mod.nl_admm_run(img.astype(np.float64), _r32(cb), lam32, g32, T)
    for k in ("u", "w", "bw", "bv"):
        assert np.abs(got[k] - o[k]).max() <= U_TOL, k
    assert abs(energy - o["energy"]) / abs(o["energy"]) <= E_TOL
    assert labels_agree(got["labels"], o["labels"], o["gap"])


def test_nl_one_iteration_from_given_state(oracle_mod):
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import NLSegmenter

    O = oracle_mod
    H, W, K = 20, 28, 3
    img, cb, _ = _image(H, W, K, 1, 31)
    rng = np.random.default_rng(32)
    lam, gamma = 0.1, 0.5
    seg = NLSegmenter(torch.tensor(img, device="cuda"), cb, lam, gamma)
    nbr, deg, _ = seg.graph()
    st = O.nl_zero_state(K, 10, H, W)
    for key in ("v", "bv", "w", "bw"):
        st[key][...] = (rng.standard_normal(st[key].shape) * 0.3).astype(np.float32)
    # zero rows of D keep zero duals in both codes
    for i in range(H * W):
        st["v"][:, deg[i]:, i // W, i % W] = 0.0
        st["bv"][:, deg[i]:, i // W, i % W] = 0.0
    s = O.data_term(img.astype(np.float64), _r32(cb))
    seg.set(B.SEG_BV, torch.tensor(st["bv"], dtype=torch.float32))
    seg.set(B.SEG_V, torch.tensor(st["v"], dtype=torch.float32))
    seg.set(B.SEG_W, torch.tensor(st["w"], dtype=torch.float32))
    seg.set(B.SEG_BW, torch.tensor(st["bw"], dtype=torch.float32))
    for n in (1, 2):
        O.nl_admm_iterate(st, s, nbr, float(np.float32(lam)), float(np.float32(gamma)), n)
        seg.step(n)
        seg.synchronize()
        for key, sel in (("u", B.SEG_U), ("w", B.SEG_W), ("bw", B.SEG_BW), ("bv", B.SEG_BV), ("v", B.SEG_V)):
            got = seg.get(sel).cpu().numpy()
            assert np.abs(got - st[key]).max() <= 2e-5, (n, key)
    seg.close()


def test_nl_reset_and_kernel_times(oracle_mod):
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import NLSegmenter

    img, cb, _ = _image(48, 64, 3, 1, 41)
    img2, _, _ = _image(48, 64, 3, 1, 42)
    f = torch.tensor(img, device="cuda")
    seg = NLSegmenter(f, cb, 1 / 32, 0.2)
    seg.step(10)
    u1 = seg.get(B.SEG_U)
    seg.reset(torch.tensor(img2, device="cuda"))  # a new image: a new graph
    nbr2, _, _ = seg.graph()
    assert np.array_equal(nbr2, oracle_mod.nl_graph(img2.astype(np.float64))[0])
    seg.reset(img)  # host image, the first graph again
    seg.step(10)
    assert torch.equal(u1, seg.get(B.SEG_U))
    t = seg.kernel_times(2)
    assert set(t) == {"nl_solve", "nl_prox", "nl_rhs"} and all(v > 0 for v in t.values())
    seg.close()


def test_nl_argument_errors():
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import NLSegmenter

    f = torch.zeros((1, 32, 32), device="cuda")
    cb = np.array([[0.2], [0.8]])
    for kw in ({"window": 14}, {"window": 17}, {"patch": 11}, {"neighbours": 9}, {"a": 0.0}):
        with pytest.raises(B.ShearsegError) as e:
            NLSegmenter(f, cb, 0.1, 0.2, **kw)
        assert e.value.code == B.SHF_ERR_ARG, kw
    bad = f.clone()
    bad[0, 1, 1] = float("inf")
    with pytest.raises(B.ShearsegError) as e:
        NLSegmenter(bad, cb, 0.1, 0.2)
    assert e.value.code == B.SHF_ERR_NONFINITE


def test_nl_textured_512_graph_and_first_iterations(oracle_mod):
    # the 512 x 512 textured image of the NL-means benchmark leg (K = 4, the
    # paper's p = 5, varpi = 15, a = 2, mt = 5, gamma = 1/5, lambda = 1/32): the
    # graph equal to the oracle's at full size, and five iterations at the bars
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import NLSegmenter

    img, _, wl = synth.make_workload_image("bezier512")
    img = img.astype(np.float32)
    cb = wl.codebook()
    lam32, g32 = float(np.float32(1 / 32)), float(np.float32(0.2))
    T = 5
    seg = NLSegmenter(torch.tensor(img, device="cuda"), cb, lam32, g32)
    nbr, deg, _ = seg.graph()
    seg.step(T)
    seg.synchronize()
    got = {k: seg.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bw", "bv", "labels")}
    energy = seg.energy()
    seg.close()
    onbr, odeg = oracle_mod.nl_graph(img.astype(np.float64))
    assert np.array_equal(deg, odeg)
    assert np.array_equal(nbr, onbr)
    o = oracle_mod.nl_admm_run(img.astype(np.float64), _r32(cb), lam32, g32, T)
    for k in ("u", "w", "bw", "bv"):
        assert np.abs(got[k] - o[k]).max() <= U_TOL, k
    assert abs(energy - o["energy"]) / abs(o["energy"]) <= E_TOL
    assert labels_agree(got["labels"], o["labels"], o["gap"])


def test_nl_barrier_wait_gives_up_and_state_stays_usable():
    # the grid barrier of the Chebyshev solve waits at most one second: a
    # barrier that cannot complete reports SHF_ERR_TIMEOUT (no fault, no
    # hang), and the state then iterates on as before
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import NLSegmenter

    img, cb, _ = _image(32, 48, 3, 1, 77)
    f = torch.tensor(img, device="cuda")
    seg = NLSegmenter(f, cb, 1 / 32, 0.2)
    seg.step(3)
    seg.synchronize()
    u3 = seg.get(B.SEG_U)
    with pytest.raises(B.ShearsegError) as e:
        B.nl_admm_barrier_selftest(seg.handle)
    assert e.value.code == B.SHF_ERR_TIMEOUT
    seg.synchronize()  # the flag was cleared
    assert torch.equal(seg.get(B.SEG_U), u3)
    seg.reset(f)
    seg.step(3)
    seg.synchronize()
    assert torch.equal(seg.get(B.SEG_U), u3)
    seg.close()
