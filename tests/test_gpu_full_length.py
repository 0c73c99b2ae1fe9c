"""GPU parity over whole runs of the benchmark workloads.

The ADMM of Sec. 3 (eqs. ADMM_u, ADMM_vw, ADMM_b) through the C ABI, run for
the workload's full iteration count, against oracle trajectories stored by
tests/golden/make_oracle_refs.py (FP64 oracle only, FP32-rounded inputs):

* the 512 x 512 Bezier/grating image (K = 4, J = 4, 61 filters), all 500
  iterations, with the default work plan and with the plan the autotuner picks
  (the benchmark's launch configuration);
* a seeded 256 x 256 image with the colours, K = 8 and J = 5 of the 2048 x 2048
  RGB workload, all 1000 iterations;
* one 256 x 256 image of the differentiable workload: 50 unrolled iterations,
  checkpoints every 10, gradients of the cross-entropy loss.

And the first four images of the uneven 64-image batch (384 x 640 with radix-3
and radix-5 transforms, 1024 x 160, 768 x 160, 384 x 192), solved inside the
tuned batch for 30 iterations, against the oracle run here.

Bars (FP32 path against the FP64 oracle): max |u - u_oracle| <= 1e-4 (also w
and b_w), relative energy error <= 1e-5, labels equal wherever the oracle's
top-two gap is at least 1e-4; gradients within 1e-3 of the largest oracle
component (+1e-6)."""

import os

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth
from tests.gpu_util import labels_agree, need_cuda

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U_TOL = 1e-4
E_TOL = 1e-5


def _ref(name):
    return dict(np.load(os.path.join(GOLDEN, name)))


def _solve(torch, img, ref, tune=False):
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    C, H, W = img.shape
    J = int(ref["J"])
    fb = FilterBank(H, W, J)
    seg = ShearletSegmenter(fb, torch.tensor(img, device="cuda"), ref["codebook"].astype(np.float64),
                            ref["Lambda"].tolist(), float(ref["gamma"]))
    if tune:
        seg.tune(10)  # restores the zero iterate after its trials
    seg.step(int(ref["T"]))
    seg.synchronize()
    out = {k: seg.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bw", "labels")}
    out["energy"] = seg.energy()
    out["iters"] = int(seg.get(B.SEG_ITER))
    out["plan"] = seg.plan()
    seg.close()
    fb.close()
    return out


def _check(g, ref):
    H, W = g["labels"].shape
    assert g["iters"] == int(ref["T"])
    errs = {k: float(np.abs(g[k] - ref[k]).max()) for k in ("u", "w", "bw")}
    assert max(errs.values()) <= U_TOL, errs
    e_rel = abs(g["energy"] - float(ref["energy"])) / abs(float(ref["energy"]))
    assert e_rel <= E_TOL, e_rel
    clear = np.unpackbits(ref["clear"])[: H * W].reshape(H, W).astype(bool)
    assert np.array_equal(g["labels"][clear], ref["labels"].astype(np.int32)[clear])


@pytest.mark.parametrize("tune", [False, True])
def test_bezier512_all_500_iterations(tune):
    torch = need_cuda()
    ref = _ref("ref_bezier512_T500.npz")
    img, _, wl = synth.make_workload_image("bezier512")
    g = _solve(torch, img.astype(np.float32), ref, tune=tune)
    assert g["plan"]["fast"] == 1
    _check(g, ref)


def test_rgb_crop_all_1000_iterations():
    torch = need_cuda()
    ref = _ref("ref_rgbcrop256_T1000.npz")
    wl = synth.WORKLOADS["rgb2048"]
    rng = np.random.default_rng(synth.seed_for(wl.index, 1))
    img, _ = synth.bezier_texture_image(256, 256, wl.codebook(), rng)
    g = _solve(torch, img.astype(np.float32), ref)
    _check(g, ref)


def test_unrolled256_gradients_at_50_iterations(oracle_mod):
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    ref = _ref("ref_unrolled256_T50.npz")
    img, lab, wl = synth.make_workload_image("unrolled256")
    img = img.astype(np.float32)
    cb = wl.codebook().astype(np.float32)
    Lam = wl.Lambda().astype(np.float32)
    fb = FilterBank(wl.H, wl.W, wl.J)
    seg = ShearletSegmenter(fb, torch.tensor(img, device="cuda"), cb.astype(np.float64), Lam.tolist(), wl.gamma)
    B.seg_admm_unrolled_fwd(seg.handle, wl.iters, 10)
    w = seg.get(B.SEG_W).cpu().numpy()
    loss, wbar = oracle_mod.ce_loss(w.astype(np.float64), lab)
    wb = torch.tensor(wbar, dtype=torch.float32, device="cuda")
    fbar = torch.empty(img.shape, dtype=torch.float32, device="cuda")
    dc, dl = B.seg_admm_unrolled_bwd(seg.handle, wb.data_ptr(), wl.K, 1, wl.J, fbar.data_ptr())
    seg.close()
    fb.close()

    def close(a, b, rel=1e-3, abs_=1e-6):
        a, b = np.asarray(a, float), np.asarray(b, float)
        return float(np.abs(a - b).max()), rel * float(np.abs(b).max()) + abs_

    assert np.abs(w - ref["w"]).max() <= U_TOL
    assert abs(loss - float(ref["loss"])) <= 1e-5 * abs(float(ref["loss"]))
    for name, got in (("codebook_grad", np.array(dc).reshape(wl.K, 1)), ("Lambda_grad", np.array(dl)),
                      ("f_grad", fbar.cpu().numpy())):
        err, bar = close(got, ref[name].reshape(np.shape(got)))
        assert err <= bar, (name, err, bar)


def test_uneven_batch_first_images_against_oracle(oracle_mod):
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import ShearletBatch

    # the batched workload exactly as generated for the benchmark
    shapes = synth.batch_shapes()
    rng = np.random.default_rng(synth.seed_for(3))
    imgs, cbs, lams = [], [], []
    for H, W, K, J in shapes:
        cb = np.array([[0.2 + 0.6 * k / (K - 1)] for k in range(K)])
        img, _ = synth.ellipse_image(H, W, cb, rng)
        imgs.append(img.astype(np.float32))
        cbs.append(cb)
        lams.append(synth.scale_weights(0.1, J))
    T = 30
    batch = ShearletBatch([torch.tensor(x, device="cuda") for x in imgs], cbs, lams, 1.0)
    batch.tune(5)
    batch.step(T)
    batch.synchronize()
    for i in range(4):
        view = batch.image(i)
        got = {k: view.get(getattr(B, "SEG_" + k.upper())).cpu().numpy() for k in ("u", "w", "bw")}
        o = oracle_mod.admm_run(imgs[i].astype(np.float64), cbs[i].astype(np.float32).astype(np.float64),
                                shapes[i][3], lams[i].astype(np.float32).astype(np.float64), 1.0, T)
        for k in got:
            assert np.abs(got[k] - o[k]).max() <= U_TOL, (i, shapes[i], k)
        assert labels_agree(view.labels().cpu().numpy(), o["labels"], o["gap"]), i
        e = view.energy()
        assert abs(e - o["energy"]) / abs(o["energy"]) <= E_TOL, i
    batch.close()
