"""Pins for the oracle's ADMM (Sec. 3, "Alternating Direction Method of
Multipliers": eq. ADMM_u, ADMM_vw, ADMM_b and the closed forms after them).

The iteration has no printed worked example; it is pinned through properties
that a dropped term, a wrong sign or a swapped operand would break: the
stationarity of the u-subproblem, the prox characterisations of the v- and
w-steps, the monotone fixed-point residual of ADMM, KKT stationarity at
convergence, and the special cases with known minimisers."""

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _random_state(O, K, J, H, W, rng):
    st = O.zero_state(K, J, H, W)
    for key in ("v", "bv", "w", "bw"):
        st[key][...] = rng.standard_normal(st[key].shape) * 0.3
    return st


def test_one_iteration_matches_subproblem_optimality(O):
    # From an arbitrary state: (i) u minimises <u,s> + 1/(2 gamma) ||b + A u - (v,w)||^2,
    # i.e. s + gamma^-1 A^T (A u + b - (v,w)) = 0 with A = (S; I);
    # (ii) v+ = argmin ||Lambda v||_1 + 1/(2 gamma)||v - g_v||^2 (checked via the prox
    # inequality), (iii) w+ is the projection of g_w, (iv) b updates per eq. ADMM_b.
    rng = np.random.default_rng(4)
    K, J, H, W = 3, 2, 24, 40
    gamma = 0.7
    Lam = np.array([0.05, 0.1, 0.2])
    s = rng.uniform(0, 1, size=(K, H, W))
    st = _random_state(O, K, J, H, W, rng)
    old = {k: v.copy() for k, v in st.items()}
    O.admm_iterate(st, s, J, Lam, gamma, 1)
    u = st["u"]
    Su = O.analyze(u, J)
    grad = s + (O.synthesize(Su + old["bv"] - old["v"], J) + (u + old["bw"] - old["w"])) / gamma
    assert np.abs(grad).max() < 1e-11
    gv = old["bv"] + Su
    thr = O.thresholds(J, Lam, gamma)[None, :, None, None]
    v = st["v"]
    # prox optimality of the l1 step: (g_v - v)/gamma in Lambda * subdifferential of |v|
    r = gv - v
    assert np.all(np.abs(r) <= thr + 1e-12)
    nz = v != 0
    assert np.abs((r - thr * np.sign(v))[nz]).max() < 1e-12
    assert np.abs(st["bv"] - (old["bv"] + Su - v)).max() < 1e-12
    gw = old["bw"] + u
    wproj = O.project_simplex(gw.transpose(1, 2, 0).reshape(-1, K)).reshape(H, W, K).transpose(2, 0, 1)
    assert np.abs(st["w"] - wproj).max() < 1e-14
    assert np.abs(st["bw"] - (old["bw"] + u - st["w"])).max() < 1e-14


def test_first_iteration_from_zero_state(O):
    # With v = b_v = w = b_w = 0 the u-step gives u = -gamma s / 2.
    rng = np.random.default_rng(9)
    K, J, H, W = 2, 1, 16, 16
    s = rng.uniform(0, 1, size=(K, H, W))
    st = O.zero_state(K, J, H, W)
    O.admm_iterate(st, s, J, [0.1, 0.1], 0.5, 1)
    assert np.abs(st["u"] + 0.25 * s).max() < 1e-15


def test_fixed_point_residual_non_increasing(O):
    # ADMM is a Douglas-Rachford iteration on (v, w, b): the distance between
    # consecutive iterates is non-increasing (firm non-expansiveness).
    img, lab, wl = synth.make_workload_image("ellipses64")
    st = O.admm_run(img, wl.codebook(), wl.J, wl.Lambda(), wl.gamma, 120)
    r = st["fp_res"]
    assert np.all(np.diff(r) <= 1e-12 * r[:-1] + 1e-14)
    assert r[-1] < 1e-3 * r[0]


def test_kkt_at_convergence(O):
    # At a fixed point, A u = (v, w) and s + gamma^-1 A^T b = 0, i.e.
    # gamma s + S^T b_v + b_w = 0; also |b_v| <= gamma Lambda and w in C.
    rng = np.random.default_rng(1)
    H = W = 32
    K, J = 3, 2
    lab = np.zeros((H, W), int)
    lab[8:20, 5:25] = 1
    lab[22:30, 10:30] = 2
    cb = np.array([0.2, 0.5, 0.8])
    f = cb[lab] + 0.05 * rng.standard_normal((H, W))
    Lam = synth.scale_weights(0.1, J)
    gamma = 1.0
    st = O.admm_run(f, cb, J, Lam, gamma, 1500)
    kkt = gamma * st["s"] + O.synthesize(st["bv"], J) + st["bw"]
    assert np.abs(kkt).max() < 1e-3
    assert np.abs(st["u"] - st["w"]).max() < 1e-3
    assert np.abs(O.analyze(st["u"], J) - st["v"]).max() < 1e-3
    thr = O.thresholds(J, Lam, gamma)[None, :, None, None]
    assert np.all(np.abs(st["bv"]) <= thr + 1e-12)
    assert np.all(st["w"] >= 0) and np.abs(st["w"].sum(0) - 1).max() < 1e-12
    assert (st["labels"] != lab).mean() < 0.01


def test_zero_regulariser_gives_nearest_codebook(O):
    # Lambda = 0: the problem is min <u, s> over C, whose minimiser puts each
    # pixel on the vertex of its smallest data cost (nearest codebook entry).
    img, lab, wl = synth.make_workload_image("ellipses64")
    st = O.admm_run(img, wl.codebook(), wl.J, np.zeros(wl.J + 1), 1.0, 60)
    s = st["s"]
    srt = np.sort(s, axis=0)
    clear = (srt[1] - srt[0]) > 1e-3
    assert np.array_equal(st["labels"][clear], s.argmin(0)[clear])


def test_constant_image_single_label(O):
    # f = c_{k0} everywhere and an unpenalised low-pass: u = e_{k0} has zero data
    # cost and zero regulariser (only the low-pass sees a constant), so it is the
    # minimiser; the iterates go there.
    cb = np.array([0.1, 0.45, 0.9, 0.6])
    H, W, J = 24, 32, 2
    f = np.full((H, W), cb[2])
    Lam = np.array([0.0, 0.3, 0.6])
    st = O.admm_run(f, cb, J, Lam, 1.0, 80)
    assert np.all(st["labels"] == 2)
    assert np.abs(st["w"][2] - 1.0).max() < 1e-6


def test_projection_variants_give_same_trajectory(O):
    img, lab, wl = synth.make_workload_image("ellipses64")
    img = img[:, :32, :48]
    a = O.admm_run(img, wl.codebook(), wl.J, wl.Lambda(), wl.gamma, 20, proj="sort")
    b = O.admm_run(img, wl.codebook(), wl.J, wl.Lambda(), wl.gamma, 20, proj="repeated")
    for key in ("u", "w", "bw", "bv"):
        assert np.abs(a[key] - b[key]).max() < 1e-12


def test_noisy_grid_segmentation(O):
    # First example of Sec. 4: a noisy 0/1 grid (sigma = 0.2, codebook {0, 1})
    # is segmented without error by the shearlet-regularised model, although
    # the nearest-codebook labelling has errors.  Stand-in grid of our own
    # geometry; weights Lambda = 0.1 (0, 0.1, 0.2, 0.4), gamma = 1, 50 iterations.
    rng = np.random.default_rng(synth.seed_for(0, 7))
    img, lab = synth.grid_image(128, 128, rng)
    cb = np.array([0.0, 1.0])
    J = 3
    st = O.admm_run(img, cb, J, synth.scale_weights(0.1, J), 1.0, 50)
    nearest = O.data_term(img, cb).argmin(0)
    assert (nearest != lab).mean() > 0.003
    assert (st["labels"] != lab).mean() == 0.0


def test_energy_decreases_from_first_iterate(O):
    img, lab, wl = synth.make_workload_image("ellipses64")
    s = O.data_term(img, wl.codebook())
    st = O.zero_state(wl.K, wl.J, wl.H, wl.W)
    O.admm_iterate(st, s, wl.J, wl.Lambda(), wl.gamma, 1)
    e1 = O.energy(st["w"], s, wl.J, wl.Lambda())
    O.admm_iterate(st, s, wl.J, wl.Lambda(), wl.gamma, 99)
    e100 = O.energy(st["w"], s, wl.J, wl.Lambda())
    assert e100 < e1


def test_energy_and_labels_hand_values(O):
    # Energy of a one-hot labelling of a constant image: data cost only, since
    # the shearlets of a constant vanish and the low-pass is unpenalised.
    H, W, J = 16, 16, 1
    x = np.zeros((2, H, W))
    x[1] = 1.0
    s = np.stack([np.full((H, W), 0.5), np.full((H, W), 0.25)])
    assert abs(O.energy(x, s, J, [0.0, 3.0]) - 0.25 * H * W) < 1e-10
    # with a penalised low-pass: + Lambda_0 * ||1||_1
    assert abs(O.energy(x, s, J, [2.0, 3.0]) - (0.25 + 2.0) * H * W) < 1e-9
    lab, gap = O.labels(np.array([[[0.2, 0.5]], [[0.7, 0.5]], [[0.1, 0.0]]]))
    assert lab.tolist() == [[1, 0]] and np.allclose(gap, [[0.5, 0.0]])


def test_data_term_hand_values(O):
    # eq. computationOfs (p = 2) and its RGB form.
    f = np.array([[0.0, 1.0]])
    s = O.data_term(f, [0.25, 1.0])
    assert np.allclose(s[:, 0], [[0.0625, 0.5625], [1.0, 0.0]])
    rgb = np.zeros((3, 1, 1))
    rgb[:, 0, 0] = [0.1, 0.2, 0.3]
    s = O.data_term(rgb, [[0.1, 0.2, 0.3], [0.0, 0.0, 0.0]])
    assert np.allclose(s[:, 0, 0], [0.0, 0.14])
