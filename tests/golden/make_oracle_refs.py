"""Write the stored oracle references for the full-length parity tests.

Calls only the FP64 oracle (``oracle/``) and the seeded input generators
(``paper_1112_1805_gb300/synth.py``, no method arithmetic).  Each reference is
the trajectory of the ADMM of Sec. 3 (eqs. ADMM_u, ADMM_vw, ADMM_b) from the
zero state, run for the workload's full iteration count on the FP32-rounded
inputs that the CUDA path receives:

* ``ref_bezier512_T500.npz`` -- the 512 x 512 Bezier/grating image, K = 4,
  J = 4 (61 filters), 500 iterations;
* ``ref_rgbcrop256_T1000.npz`` -- a seeded 256 x 256 crop-sized image of the
  2048 x 2048 RGB workload (K = 8 colours {0.2, 0.8}^3, J = 5, 125 filters),
  1000 iterations (the full-size run does not fit the host);
* ``ref_unrolled256_T50.npz`` -- one 256 x 256 image of the differentiable
  workload (K = 4, J = 3): w after 50 iterations, the cross-entropy loss
  against the generator's label map and its gradients with respect to the
  codebook, Lambda and the image, by the oracle's reverse mode.

Stored arrays are FP32 (rounding error <= 6e-8 relative, far below the 1e-4
parity bar); the labels with a mask of the pixels whose top-two gap is at
least 1e-4; energies and losses in FP64.

Usage: ``python tests/golden/make_oracle_refs.py [bezier512] [rgbcrop] [unrolled]``
(all three by default; hours on a few host cores).
"""

from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1112_1805_gb300 import synth  # noqa: E402

TIE = 1e-4


def _f32(a):
    return np.asarray(a, dtype=np.float32)


def _r64(a):
    """The FP32 value the CUDA path sees, widened for the oracle."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _save(name, **arrays):
    path = os.path.join(HERE, name)
    tmp = path + ".tmp.npz"
    np.savez_compressed(tmp, **arrays)
    os.replace(tmp, path)
    print(f"wrote {path} ({os.path.getsize(path) / 1e6:.2f} MB)", flush=True)


def _admm_ref(img, cb, J, Lam, gamma, T):
    o = O.admm_run(_r64(img), _r64(cb), J, _r64(Lam), gamma, T)
    return dict(u=_f32(o["u"]), w=_f32(o["w"]), bw=_f32(o["bw"]), labels=o["labels"].astype(np.int8),
                clear=np.packbits(o["gap"] >= TIE), energy=np.float64(o["energy"]),
                fp_res=o["fp_res"].astype(np.float64), T=np.int32(T), J=np.int32(J), gamma=np.float64(gamma),
                Lambda=_f32(Lam), codebook=_f32(cb))


def bezier512():
    img, _, wl = synth.make_workload_image("bezier512")
    ref = _admm_ref(img, wl.codebook(), wl.J, wl.Lambda(), wl.gamma, wl.iters)
    _save("ref_bezier512_T500.npz", **ref)


def rgbcrop_image():
    """The seeded 256 x 256 image with the RGB workload's colours and texture."""
    wl = synth.WORKLOADS["rgb2048"]
    rng = np.random.default_rng(synth.seed_for(wl.index, 1))
    img, _ = synth.bezier_texture_image(256, 256, wl.codebook(), rng)
    return img.astype(np.float32), wl


def rgbcrop():
    img, wl = rgbcrop_image()
    ref = _admm_ref(img, wl.codebook(), wl.J, wl.Lambda(), wl.gamma, wl.iters)
    _save("ref_rgbcrop256_T1000.npz", **ref)


def unrolled():
    img, lab, wl = synth.make_workload_image("unrolled256")
    g = O.unrolled_grads(_r64(img), _r64(wl.codebook()), wl.J, _r64(wl.Lambda()), wl.gamma, wl.iters, lab)
    _save("ref_unrolled256_T50.npz", w=_f32(g["w"]), loss=np.float64(g["loss"]), codebook_grad=g["codebook"],
          Lambda_grad=g["Lambda"], f_grad=_f32(g["f"]), T=np.int32(wl.iters), J=np.int32(wl.J))


JOBS = {"unrolled": unrolled, "bezier512": bezier512, "rgbcrop": rgbcrop}

if __name__ == "__main__":
    for name in sys.argv[1:] or list(JOBS):
        t0 = time.time()
        JOBS[name]()
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)
