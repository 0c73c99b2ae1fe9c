"""Pins for the oracle's TV-regularised segmentation, the comparison model of
Sec. 4 (eq. TVreg: the labels' gradients coupled per pixel), solved by the
ADMM of Sec. 3 with S replaced by the periodic forward-difference gradient.

Hand values and closed forms pin the pieces (the gradient and its adjoint,
the u-step's linear solve against the explicit 5-point stencil and a dense
solve, the group shrinkage against its optimality conditions, the energy of a
stripe image); the iteration is pinned through the stationarity of its
u-subproblem, the monotone fixed-point residual, KKT at convergence and the
special cases with known minimisers."""

import math

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _stencil(u):
    """(I + grad^T grad) u for periodic forward differences: 5 u minus the
    four neighbours (the 5-point Laplacian with the identity added)."""
    return (5 * u - np.roll(u, 1, axis=-2) - np.roll(u, -1, axis=-2) - np.roll(u, 1, axis=-1)
            - np.roll(u, -1, axis=-1))


def test_gradient_hand_values(O):
    u = np.array([[[1.0, 2.0, 4.0], [0.0, 3.0, 3.0]]])  # K = 1, H = 2, W = 3
    g = O.tv_grad(u)
    # along rows (next row minus this row, wrapping) and along columns
    assert g[0, 0].tolist() == [[-1.0, 1.0, -1.0], [1.0, -1.0, 1.0]]
    assert g[0, 1].tolist() == [[1.0, 2.0, -3.0], [3.0, 0.0, -3.0]]
    assert np.abs(O.tv_grad(np.full((2, 5, 7), 0.3))).max() == 0.0
    # adjoint of a constant field: zero divergence
    assert np.abs(O.tv_grad_adj(np.full((2, 2, 5, 7), 1.7))).max() < 1e-15


def test_gradient_adjoint(O):
    rng = np.random.default_rng(3)
    u = rng.standard_normal((3, 9, 14))
    p = rng.standard_normal((3, 2, 9, 14))
    assert abs((O.tv_grad(u) * p).sum() - (u * O.tv_grad_adj(p)).sum()) < 1e-11


@pytest.mark.parametrize("H,W", [(8, 8), (15, 24), (30, 50), (12, 7)])
def test_solve_inverts_the_stencil(O, H, W):
    rng = np.random.default_rng(H * W)
    rhs = rng.standard_normal((2, H, W))
    u = O.tv_solve(rhs)
    assert np.abs(_stencil(u) - rhs).max() < 1e-12
    # and (I + grad^T grad) built from the gradient itself
    assert np.abs(u + O.tv_grad_adj(O.tv_grad(u)) - rhs).max() < 1e-12


def test_solve_against_dense_matrix(O):
    # the matrix of I + grad^T grad assembled column by column from tv_grad and
    # tv_grad_adj (no FFT), solved densely
    H, W = 4, 6
    n = H * W
    M = np.zeros((n, n))
    for i in range(n):
        e = np.zeros((1, H, W))
        e.flat[i] = 1.0
        M[:, i] = (e + O.tv_grad_adj(O.tv_grad(e))).ravel()
    rng = np.random.default_rng(0)
    rhs = rng.standard_normal((1, H, W))
    assert np.abs(O.tv_solve(rhs).ravel() - np.linalg.solve(M, rhs.ravel())).max() < 1e-12


def test_group_shrinkage(O):
    rng = np.random.default_rng(5)
    K, H, W, t = 3, 4, 5, 0.7
    g = rng.standard_normal((K, 2, H, W)) * 0.6
    v = O.tv_shrink(g, t)
    # closed form on one pixel: g (1 - t/|g|)_+ over its 2K values
    gx = g[:, :, 1, 2].ravel()
    n = np.linalg.norm(gx)
    assert np.allclose(v[:, :, 1, 2].ravel(), gx * max(0.0, 1 - t / n), atol=1e-15)
    # optimality of the prox of t |.|_2 per pixel: g - v = t v/|v| where v != 0, |g| <= t where v = 0
    for y in range(H):
        for x in range(W):
            gp, vp = g[:, :, y, x].ravel(), v[:, :, y, x].ravel()
            nv = np.linalg.norm(vp)
            if nv > 0:
                assert np.abs((gp - vp) - t * vp / nv).max() < 1e-12
            else:
                assert np.linalg.norm(gp) <= t + 1e-12
            # and no random perturbation lowers the objective
            f0 = t * nv + 0.5 * np.sum((vp - gp) ** 2)
            for _ in range(5):
                d = vp + 1e-3 * rng.standard_normal(vp.shape)
                assert t * np.linalg.norm(d) + 0.5 * np.sum((d - gp) ** 2) >= f0 - 1e-12
    # per-label groups: each label's two values shrink on their own
    vl = O.tv_shrink(g, t, per_label=True)
    gk = g[1, :, 2, 3]
    assert np.allclose(vl[1, :, 2, 3], gk * max(0.0, 1 - t / np.linalg.norm(gk)), atol=1e-15)


def test_energy_of_a_stripe(O):
    # K = 2, a vertical stripe of label 1 (columns 2..4) on label 0: the two
    # one-hot planes change at 2 H pixels, where both labels step by 1, so the
    # coupled TV is 2 H sqrt(2) (and 2 * 2 H for the per-label sum).
    H, W, lam = 8, 10, 0.3
    x = np.zeros((2, H, W))
    x[0] = 1.0
    x[0, :, 2:5] = 0.0
    x[1, :, 2:5] = 1.0
    s = np.stack([np.full((H, W), 0.1), np.full((H, W), 0.4)])
    data = 0.1 * H * (W - 3) + 0.4 * H * 3
    assert abs(O.tv_energy(x, s, lam) - (data + lam * 2 * H * math.sqrt(2))) < 1e-12
    assert abs(O.tv_energy(x, s, lam, per_label=True) - (data + lam * 4 * H)) < 1e-12


def test_one_iteration_matches_subproblem_optimality(O):
    # u minimises <u,s> + 1/(2 gamma) (||grad u + b_v - v||^2 + ||u + b_w - w||^2):
    # gamma s + grad^T(grad u + b_v - v) + (u + b_w - w) = 0, checked with the stencil
    rng = np.random.default_rng(8)
    K, H, W, lam, gamma = 3, 12, 18, 0.2, 0.6
    s = rng.uniform(0, 1, (K, H, W))
    st = O.tv_zero_state(K, H, W)
    for key in ("v", "bv", "w", "bw"):
        st[key][...] = rng.standard_normal(st[key].shape) * 0.3
    old = {k: v.copy() for k, v in st.items()}
    O.tv_admm_iterate(st, s, lam, gamma, 1)
    u = st["u"]
    r = gamma * s + (_stencil(u) - u) + O.tv_grad_adj(old["bv"] - old["v"]) + (u + old["bw"] - old["w"])
    assert np.abs(r).max() < 1e-11
    gv = old["bv"] + O.tv_grad(u)
    assert np.abs(st["v"] - O.tv_shrink(gv, gamma * lam)).max() < 1e-15
    assert np.abs(st["bv"] - (gv - st["v"])).max() < 1e-15
    gw = old["bw"] + u
    wp = O.project_simplex(gw.transpose(1, 2, 0).reshape(-1, K)).reshape(H, W, K).transpose(2, 0, 1)
    assert np.abs(st["w"] - wp).max() < 1e-15


def test_first_iterate_from_zero(O):
    # v = b_v = w = b_w = 0: (I + grad^T grad) u = -gamma s
    rng = np.random.default_rng(2)
    s = rng.uniform(0, 1, (2, 10, 16))
    st = O.tv_zero_state(2, 10, 16)
    O.tv_admm_iterate(st, s, 0.1, 0.5, 1)
    assert np.abs(_stencil(st["u"]) + 0.5 * s).max() < 1e-13


def test_fixed_point_residual_non_increasing(O):
    img, lab, wl = synth.make_workload_image("ellipses64")
    s = O.data_term(img, wl.codebook())
    st = O.tv_zero_state(wl.K, wl.H, wl.W)
    r = O.tv_admm_iterate(st, s, 0.1, 1.0, 150, record_residual=True)
    assert np.all(np.diff(r) <= 1e-12 * r[:-1] + 1e-14)
    assert r[-1] < 1e-2 * r[0]


def test_kkt_at_convergence(O):
    # fixed point: grad u = v, u = w, gamma s + grad^T b_v + b_w = 0, and the
    # duals in their balls: |b_v(x)| <= gamma lambda over the 2K values of x
    rng = np.random.default_rng(1)
    H = W = 32
    lab = np.zeros((H, W), int)
    lab[8:20, 5:25] = 1
    lab[22:30, 10:30] = 2
    cb = np.array([0.2, 0.5, 0.8])
    f = cb[lab] + 0.05 * rng.standard_normal((H, W))
    lam, gamma = 0.05, 1.0
    st = O.tv_admm_run(f, cb, lam, gamma, 2000)
    assert np.abs(gamma * st["s"] + O.tv_grad_adj(st["bv"]) + st["bw"]).max() < 1e-3
    assert np.abs(st["u"] - st["w"]).max() < 1e-3
    assert np.abs(O.tv_grad(st["u"]) - st["v"]).max() < 1e-3
    nb = np.sqrt((st["bv"] ** 2).sum(axis=(0, 1)))
    assert nb.max() <= gamma * lam * (1 + 1e-12)
    assert (st["labels"] != lab).mean() < 0.01


def test_zero_regulariser_gives_nearest_codebook(O):
    # lambda = 0: min <u, s> over C separates per pixel (vertex of the smallest
    # cost).  The u-step still couples pixels through (I + grad^T grad)^-1,
    # which damps an isolated pixel's update up to ninefold, so pixels whose
    # two smallest costs differ by little converge slowly: checked where the
    # difference is at least 0.02.
    img, lab, wl = synth.make_workload_image("ellipses64")
    st = O.tv_admm_run(img, wl.codebook(), 0.0, 1.0, 300)
    s = st["s"]
    srt = np.sort(s, axis=0)
    clear = (srt[1] - srt[0]) > 0.02
    assert np.array_equal(st["labels"][clear], s.argmin(0)[clear])


def test_constant_image_single_label(O):
    cb = np.array([0.1, 0.45, 0.9, 0.6])
    f = np.full((20, 24), cb[1])
    st = O.tv_admm_run(f, cb, 0.5, 1.0, 80)
    assert np.all(st["labels"] == 1)
    assert np.abs(st["w"][1] - 1.0).max() < 1e-6


def test_energy_decreases_and_beats_nearest_codebook_on_noise(O):
    # on a noisy piecewise-constant image the TV model removes isolated
    # nearest-codebook errors, and its energy falls from the first iterate
    rng = np.random.default_rng(synth.seed_for(0, 11))
    cb = np.array([0.2, 0.5, 0.8])
    img, lab = synth.ellipse_image(64, 64, cb[:, None], rng, sigma=0.12)
    s = O.data_term(img, cb)
    st = O.tv_zero_state(3, 64, 64)
    O.tv_admm_iterate(st, s, 0.05, 1.0, 1)
    e1 = O.tv_energy(st["w"], s, 0.05)
    O.tv_admm_iterate(st, s, 0.05, 1.0, 299)
    assert O.tv_energy(st["w"], s, 0.05) < e1
    labels, _ = O.labels(st["w"])
    assert (labels != lab).mean() < 0.5 * (s.argmin(0) != lab).mean()
