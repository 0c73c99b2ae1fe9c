"""Pins for the oracle's reverse mode of the unrolled ADMM (gradients of a loss
of w_T with respect to the codebook, the weights Lambda and the image),
checked against central finite differences of the oracle's own forward in FP64."""

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _problem(seed=3, H=24, W=32, K=3, J=2, C=1):
    rng = np.random.default_rng(seed)
    if C == 1:
        cb = np.array([[0.2 + 0.6 * k / (K - 1)] for k in range(K)])
    else:
        cb = np.array([[0.2, 0.2, 0.8], [0.8, 0.2, 0.2], [0.2, 0.8, 0.5]])[:K]
    img, lab = synth.ellipse_image(H, W, cb, rng, n_ellipses=3)
    Lam = synth.scale_weights(0.1, J) + np.r_[0.003, np.zeros(J)]
    return img, lab, cb, Lam


def _loss(O, img, lab, cb, Lam, J, T, gamma=1.0):
    s = O.data_term(img, cb)
    st = O.zero_state(cb.shape[0], J, img.shape[-2], img.shape[-1])
    O.admm_iterate(st, s, J, Lam, gamma, T)
    return O.ce_loss(st["w"], lab)[0]


@pytest.mark.parametrize("C", [1, 3])
def test_codebook_and_lambda_gradients_match_finite_differences(O, C):
    J, T = 2, 8
    img, lab, cb, Lam = _problem(C=C)
    g = O.unrolled_grads(img, cb, J, Lam, 1.0, T, lab)
    h = 1e-6
    for k in range(cb.shape[0]):
        for ch in range(cb.shape[1]):
            p, m = cb.copy(), cb.copy()
            p[k, ch] += h
            m[k, ch] -= h
            fd = (_loss(O, img, lab, p, Lam, J, T) - _loss(O, img, lab, m, Lam, J, T)) / (2 * h)
            assert abs(fd - g["codebook"][k, ch]) <= 1e-6 + 1e-5 * abs(fd), (k, ch)
    for j in range(J + 1):
        p, m = Lam.copy(), Lam.copy()
        p[j] += h
        m[j] -= h
        fd = (_loss(O, img, lab, cb, p, J, T) - _loss(O, img, lab, cb, m, J, T)) / (2 * h)
        assert abs(fd - g["Lambda"][j]) <= 1e-6 + 1e-4 * abs(fd), j


def test_image_gradient_matches_finite_differences(O):
    J, T = 2, 6
    img, lab, cb, Lam = _problem(seed=8)
    g = O.unrolled_grads(img, cb, J, Lam, 1.0, T, lab)
    h = 1e-6
    for (y, x) in [(3, 4), (10, 20), (23, 31)]:
        p, m = img.copy(), img.copy()
        p[0, y, x] += h
        m[0, y, x] -= h
        fd = (_loss(O, p, lab, cb, Lam, J, T) - _loss(O, m, lab, cb, Lam, J, T)) / (2 * h)
        assert abs(fd - g["f"][0, y, x]) <= 1e-7 + 1e-5 * abs(fd)


def test_vjp_of_a_linear_functional(O):
    # for L = <a, w_T> with an arbitrary a, sbar and Lambar must give the
    # directional derivatives of L along s and Lambda
    J, T = 1, 5
    rng = np.random.default_rng(1)
    K, H, W = 3, 16, 20
    s = rng.uniform(0, 1, size=(K, H, W))
    Lam = np.array([0.01, 0.03])
    a = rng.standard_normal((K, H, W))
    wT, sbar, lbar = O.unrolled_vjp(s, J, Lam, 0.7, T, a)

    def L(s_, Lam_):
        st = O.zero_state(K, J, H, W)
        O.admm_iterate(st, s_, J, Lam_, 0.7, T)
        return (a * st["w"]).sum()

    assert np.abs(wT - (lambda st: (O.admm_iterate(st, s, J, Lam, 0.7, T), st["w"])[1])(O.zero_state(K, J, H, W))).max() < 1e-12
    d = rng.standard_normal((K, H, W))
    h = 1e-6
    fd = (L(s + h * d, Lam) - L(s - h * d, Lam)) / (2 * h)
    assert abs(fd - (sbar * d).sum()) <= 1e-6 + 1e-5 * abs(fd)
    for j in range(J + 1):
        e = np.zeros(J + 1)
        e[j] = h
        fd = (L(s, Lam + e) - L(s, Lam - e)) / (2 * h)
        assert abs(fd - lbar[j]) <= 1e-6 + 1e-4 * abs(fd)
