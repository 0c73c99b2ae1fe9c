"""GPU: reverse mode of the unrolled ADMM through the C ABI against the
oracle's FP64 reverse mode (itself pinned by finite differences).

FP32 forward and adjoint over T iterations: gradients must agree with the
oracle to 1e-3 of the largest component (plus 1e-6), losses to 1e-5."""

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth
from tests.gpu_util import need_cuda

pytestmark = pytest.mark.gpu


def _problem(seed, H, W, K, J, C=1):
    rng = np.random.default_rng(seed)
    if C == 1:
        cb = np.array([[0.2 + 0.6 * k / (K - 1)] for k in range(K)])
    else:
        cb = np.array([[0.2, 0.2, 0.8], [0.8, 0.2, 0.2], [0.2, 0.8, 0.5], [0.7, 0.7, 0.2]])[:K]
    img, lab = synth.ellipse_image(H, W, cb, rng, n_ellipses=4)
    Lam = synth.scale_weights(0.1, J) + np.r_[0.003, np.zeros(J)]
    return img.astype(np.float32), lab, cb.astype(np.float32), Lam.astype(np.float32)


def _gpu_grads(torch, img, lab, cb, Lam, J, T, ck):
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    import oracle as O

    fb = FilterBank(img.shape[1], img.shape[2], J)
    seg = ShearletSegmenter(fb, torch.tensor(img, device="cuda"), cb.astype(np.float64), Lam.tolist(), 1.0)
    B.seg_admm_unrolled_fwd(seg.handle, T, ck)
    w = seg.get(B.SEG_W).cpu().numpy()
    loss, wbar = O.ce_loss(w.astype(np.float64), lab)
    wb = torch.tensor(wbar, dtype=torch.float32, device="cuda")
    fbar = torch.empty(img.shape, dtype=torch.float32, device="cuda")
    sbar = torch.empty((cb.shape[0],) + img.shape[1:], dtype=torch.float32, device="cuda")
    dc, dl = B.seg_admm_unrolled_bwd(seg.handle, wb.data_ptr(), cb.shape[0], cb.shape[1], J, fbar.data_ptr(),
                                     sbar.data_ptr())
    out = {"loss": loss, "w": w, "codebook": np.array(dc).reshape(cb.shape), "Lambda": np.array(dl),
           "f": fbar.cpu().numpy(), "sbar": sbar.cpu().numpy()}
    seg.close()
    fb.close()
    return out


def _close(a, b, rel=1e-3, abs_=1e-6):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() <= rel * np.abs(b).max() + abs_


# register-FFT sizes (24 x 32, 64 x 64, 32 x 48, 40 x 80) take the fused fast
# reverse sweep; 30 x 50 takes the general kernels
@pytest.mark.parametrize("H,W,K,J,C,T,ck", [(24, 32, 3, 2, 1, 8, 3), (24, 32, 3, 2, 3, 8, 8), (64, 64, 3, 2, 1, 20, 5),
                                            (32, 48, 4, 1, 1, 12, 1), (40, 80, 5, 2, 1, 10, 4),
                                            (30, 50, 3, 2, 1, 8, 3)])
def test_gradients_match_oracle(oracle_mod, H, W, K, J, C, T, ck):
    torch = need_cuda()
    img, lab, cb, Lam = _problem(H * W + K, H, W, K, J, C)
    g = _gpu_grads(torch, img, lab, cb, Lam, J, T, ck)
    o = oracle_mod.unrolled_grads(img.astype(np.float64), cb.astype(np.float64), J, Lam.astype(np.float64), 1.0,
                                  T, lab)
    assert np.abs(g["w"] - o["w"]).max() <= 1e-4
    assert abs(g["loss"] - o["loss"]) <= 1e-5 * abs(o["loss"])
    assert _close(g["codebook"], o["codebook"])
    assert _close(g["Lambda"], o["Lambda"])
    assert _close(g["f"], o["f"])
    assert _close(g["sbar"], o["sbar"])


def test_checkpoint_spacing_does_not_change_gradients():
    torch = need_cuda()
    img, lab, cb, Lam = _problem(5, 32, 32, 3, 2)
    ref = _gpu_grads(torch, img, lab, cb, Lam, 2, 9, 9)
    for ck in (1, 2, 4):
        g = _gpu_grads(torch, img, lab, cb, Lam, 2, 9, ck)
        for key in ("codebook", "Lambda", "f"):
            assert np.array_equal(g[key], ref[key]), (ck, key)


def test_autograd_function_and_descent_step():
    torch = need_cuda()
    from paper_1112_1805_gb300.api import FilterBank, unrolled_segmentation

    img, lab, cb, Lam = _problem(11, 48, 48, 3, 2)
    fb = FilterBank(48, 48, 2)
    f = torch.tensor(img, device="cuda", requires_grad=True)
    c = torch.tensor(cb, dtype=torch.float64, requires_grad=True)
    L = torch.tensor(Lam, dtype=torch.float64, requires_grad=True)
    lab_t = torch.tensor(lab, dtype=torch.int64, device="cuda")

    def loss_of(w):
        wl = torch.gather(w, 0, lab_t[None])[0]
        return -torch.log(torch.clamp(wl, min=1e-6)).mean()

    w = unrolled_segmentation(f, c, L, fb, 1.0, 10, 5)
    loss = loss_of(w)
    loss.backward()
    ref = _gpu_grads(torch, img, lab, cb, Lam, 2, 10, 5)
    assert np.allclose(c.grad.numpy(), ref["codebook"], rtol=1e-5, atol=1e-7)
    assert np.allclose(L.grad.numpy(), ref["Lambda"], rtol=1e-5, atol=1e-7)
    assert np.allclose(f.grad.cpu().numpy(), ref["f"], rtol=1e-5, atol=1e-7)
    # a small step against the codebook gradient lowers the loss
    with torch.no_grad():
        c2 = c - 1e-2 * c.grad / c.grad.abs().max()
    loss2 = loss_of(unrolled_segmentation(f.detach(), c2, L.detach(), fb, 1.0, 10, 5))
    assert loss2.item() < loss.detach().item()


def test_unrolled_workload_shape():
    # the differentiable workload's per-image shape: 256 x 256, K = 4, J = 3,
    # 50 unrolled iterations, checkpoint every 10
    torch = need_cuda()
    img, lab, wl = synth.make_workload_image("unrolled256")
    cb = wl.codebook().astype(np.float32)
    Lam = wl.Lambda().astype(np.float32)
    g = _gpu_grads(torch, img.astype(np.float32), lab, cb, Lam, wl.J, wl.iters, 10)
    for key in ("codebook", "Lambda", "f"):
        assert np.all(np.isfinite(g[key]))
    assert np.abs(g["codebook"]).max() > 0 and np.abs(g["Lambda"][1:]).max() > 0


def test_enqueued_sweeps_on_concurrent_states_equal_the_synchronous_call():
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    probs = [_problem(40 + i, 64, 64, 3, 2) for i in range(3)]
    fb = FilterBank(64, 64, 2)
    segs = [ShearletSegmenter(fb, torch.tensor(p[0], device="cuda"), p[2].astype(np.float64), p[3].tolist(), 1.0)
            for p in probs]
    cots = [torch.full((3, 64, 64), 1e-3 * (i + 1), device="cuda") for i in range(3)]
    ref = []
    for sg, c in zip(segs, cots):
        B.seg_admm_unrolled_fwd(sg.handle, 9, 4)
        ref.append(B.seg_admm_unrolled_bwd(sg.handle, c.data_ptr(), 3, 1, 2))
    for sg, c in zip(segs, cots):
        B.seg_admm_unrolled_fwd(sg.handle, 9, 4)
        B.seg_admm_unrolled_bwd_enqueue(sg.handle, c.data_ptr())
    got = [B.seg_admm_unrolled_grads(sg.handle, 3, 1, 2) for sg in segs]
    assert got == ref
    with pytest.raises(B.ShearsegError):
        fresh = ShearletSegmenter(fb, torch.tensor(probs[0][0], device="cuda"), probs[0][2].astype(np.float64),
                                  probs[0][3].tolist(), 1.0)
        B.seg_admm_unrolled_grads(fresh.handle, 3, 1, 2)
    for sg in segs:
        sg.close()
    fb.close()
