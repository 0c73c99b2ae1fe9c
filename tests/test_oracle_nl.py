"""Pins for the oracle's NL-means regulariser, the second comparison model of
Sec. 4: patch distances d_a, the greedy symmetric neighbour graph (p = 5,
varpi = 15, a = 2, mt = 5), the difference matrix D, the u-step solve with
I + D^T D, and the ADMM of Sec. 3 with S replaced by D.

Hand values and closed forms pin the pieces (distances of single bright
pixels, D^T D = 2 L of the neighbour graph, the energy of an isolated pixel);
a plain Python transcription of the paper's neighbour selection checks the
graph on small images; the iteration is pinned like the TV model's."""

import math

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth

S1 = 1 + 2 * math.exp(-1 / 8) + 2 * math.exp(-1 / 2)  # sum of exp(-t^2/8), t = -2..2 (a = 2)


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def test_patch_distance_hand_values(O):
    # a single bright pixel q: d(i, j) = G(q - i) for j far away (its patch is 0),
    # with the normalised Gaussian G(t) = exp(-|t|^2 / 8) / S1^2 on the 5 x 5 patch
    f = np.zeros((20, 20))
    f[10, 10] = 1.0
    far = (3, 17)
    assert O.nl_distance(f, (10, 10), far) == pytest.approx(1 / S1 ** 2, rel=1e-14)
    assert O.nl_distance(f, (11, 10), far) == pytest.approx(math.exp(-1 / 8) / S1 ** 2, rel=1e-14)
    assert O.nl_distance(f, (12, 9), far) == pytest.approx(math.exp(-5 / 8) / S1 ** 2, rel=1e-14)
    assert O.nl_distance(f, (13, 10), far) == 0.0  # q outside the patch
    # symmetry and d(i, i) = 0
    rng = np.random.default_rng(2)
    g = rng.uniform(0, 1, (12, 14))
    assert O.nl_distance(g, (4, 5), (7, 9)) == O.nl_distance(g, (7, 9), (4, 5))
    assert O.nl_distance(g, (6, 6), (6, 6)) == 0.0
    # mirrored border: the bright pixel at row 1 is seen at rows -1 and 1 by row 0
    h = np.zeros((20, 20))
    h[1, 10] = 1.0
    assert O.nl_distance(h, (0, 10), far) == pytest.approx(2 * math.exp(-1 / 8) / S1 ** 2, rel=1e-14)
    # channels add
    rgb = np.zeros((3, 20, 20))
    rgb[:, 10, 10] = [1.0, 0.5, 0.0]
    assert O.nl_distance(rgb, (10, 10), far) == pytest.approx(1.25 / S1 ** 2, rel=1e-14)


def _greedy_graph(O, f, p, win, a, mt):
    """The paper's neighbour selection written out in plain Python (raster
    order; k = min(mt, 2 mt - l) new neighbours with the smallest distances;
    candidates already linked or at 2 mt neighbours are passed over)."""
    H, W = f.shape[-2:]
    r = win // 2
    nb = [set() for _ in range(H * W)]
    for ri in range(H):
        for ci in range(W):
            i = ri * W + ci
            cand = []
            for rj in range(max(0, ri - r), min(H, ri + r + 1)):
                for cj in range(max(0, ci - r), min(W, ci + r + 1)):
                    j = rj * W + cj
                    if j != i:
                        cand.append((O.nl_distance(f, (ri, ci), (rj, cj), p, a), j))
            cand.sort()
            k = min(mt, 2 * mt - len(nb[i]))
            for _, j in cand:
                if k <= 0:
                    break
                if j in nb[i] or len(nb[j]) >= 2 * mt:
                    continue
                nb[i].add(j)
                nb[j].add(i)
                k -= 1
    return nb


@pytest.mark.parametrize("H,W,C,p,win,mt", [(10, 12, 1, 3, 5, 2), (9, 11, 3, 5, 7, 3), (12, 12, 1, 5, 15, 5)])
def test_graph_matches_the_papers_selection(O, H, W, C, p, win, mt):
    rng = np.random.default_rng(H * W + C)
    f = rng.uniform(0, 1, (C, H, W))
    nbr, deg = O.nl_graph(f, p=p, win=win, a=2.0, mt=mt)
    ref = _greedy_graph(O, f, p, win, 2.0, mt)
    for i in range(H * W):
        got = [j for j in nbr[i] if j >= 0]
        assert got == sorted(ref[i]), i
        assert deg[i] == len(ref[i]) <= 2 * mt
        assert all(nbr[i, b] == -1 for b in range(deg[i], 2 * mt))


def test_graph_invariants_on_the_workload_image(O):
    img, _, _ = synth.make_workload_image("ellipses64")
    nbr, deg = O.nl_graph(img)
    H = W = 64
    for i in range(H * W):
        nb = nbr[i, : deg[i]]
        assert len(set(nb)) == len(nb) and i not in nb
        assert np.all(np.diff(nb) > 0)
        for j in nb:
            assert i in nbr[j, : deg[j]]  # symmetric weights
            assert abs(j // W - i // W) <= 7 and abs(j % W - i % W) <= 7  # inside the search window
    assert deg.max() <= 10 and deg.min() >= 5  # every pixel picks up to 5 itself


def test_D_structure(O):
    rng = np.random.default_rng(4)
    f = rng.uniform(0, 1, (16, 18))
    nbr, deg = O.nl_graph(f)
    u = rng.standard_normal((2, 16, 18))
    q = rng.standard_normal((2, 10, 16, 18))
    Du = O.nl_D(nbr, u)
    assert abs((Du * q).sum() - (u * O.nl_Dt(nbr, q)).sum()) < 1e-10  # adjoint
    assert np.abs(O.nl_D(nbr, np.ones((1, 16, 18)))).max() == 0.0  # constants lie in the kernel
    # zero rows where a pixel has fewer neighbours than the block index
    for i in range(16 * 18):
        assert np.all(Du[:, deg[i]:, i // 18, i % 18] == 0.0)
    # D^T D = 2 L: (D^T D u)(j) = 2 sum_{n in N(j)} (u(j) - u(n)) for symmetric neighbour sets
    lap = np.zeros_like(u)
    uf = u.reshape(2, -1)
    for j in range(16 * 18):
        nb = nbr[j, : deg[j]]
        lap.reshape(2, -1)[:, j] = 2 * (deg[j] * uf[:, j] - uf[:, nb].sum(axis=1))
    assert np.abs(O.nl_Dt(nbr, Du) - lap).max() < 1e-12


def test_solve(O):
    rng = np.random.default_rng(6)
    f = rng.uniform(0, 1, (6, 7))
    nbr, deg = O.nl_graph(f, win=5, mt=3)
    n = 42
    M = np.zeros((n, n))
    for i in range(n):
        e = np.zeros((1, 6, 7))
        e.flat[i] = 1.0
        M[:, i] = (e + O.nl_Dt(nbr, O.nl_D(nbr, e))).ravel()
    rhs = rng.standard_normal((1, 6, 7))
    assert np.abs(O.nl_solve(nbr, rhs).ravel() - np.linalg.solve(M, rhs.ravel())).max() < 1e-12
    # eigenvalues of I + D^T D in [1, 1 + 4 * max degree] (Gershgorin on 2 L)
    ev = np.linalg.eigvalsh(M)
    assert ev.min() > 1 - 1e-12 and ev.max() <= 1 + 4 * deg.max() + 1e-12


def test_energy_of_an_isolated_pixel(O):
    # one pixel x0 of label 1 in label 0: at x0 all deg(x0) differences are 1 in
    # both labels, sqrt(2 deg(x0)); at each neighbour one difference, sqrt(2)
    rng = np.random.default_rng(8)
    f = rng.uniform(0, 1, (14, 14))
    nbr, deg = O.nl_graph(f)
    x = np.zeros((2, 14, 14))
    x[0] = 1.0
    x0 = 7 * 14 + 6
    x[0].flat[x0], x[1].flat[x0] = 0.0, 1.0
    s = np.stack([np.full((14, 14), 0.3), np.full((14, 14), 0.1)])
    d0 = deg[x0]
    want = 0.3 * (196 - 1) + 0.1 + 0.25 * (math.sqrt(2 * d0) + d0 * math.sqrt(2))
    assert O.nl_energy(x, s, nbr, 0.25) == pytest.approx(want, rel=1e-14)


def test_one_iteration_matches_subproblem_optimality(O):
    rng = np.random.default_rng(10)
    K, H, W, lam, gamma = 3, 12, 14, 0.1, 0.5
    f = rng.uniform(0, 1, (H, W))
    nbr, _ = O.nl_graph(f)
    s = rng.uniform(0, 1, (K, H, W))
    st = O.nl_zero_state(K, 10, H, W)
    for key in ("v", "bv", "w", "bw"):
        st[key][...] = rng.standard_normal(st[key].shape) * 0.3
    old = {k: v.copy() for k, v in st.items()}
    O.nl_admm_iterate(st, s, nbr, lam, gamma, 1)
    u = st["u"]
    r = gamma * s + O.nl_Dt(nbr, O.nl_D(nbr, u) + old["bv"] - old["v"]) + (u + old["bw"] - old["w"])
    assert np.abs(r).max() < 1e-10
    g = old["bv"] + O.nl_D(nbr, u)
    n = np.sqrt((g ** 2).sum(axis=(0, 1)))
    fac = np.where(n > gamma * lam, 1 - gamma * lam / np.maximum(n, 1e-300), 0.0)
    assert np.abs(st["v"] - g * fac).max() < 1e-14
    assert np.abs(st["bv"] - (g - st["v"])).max() < 1e-14


def test_fixed_point_residual_and_kkt(O):
    rng = np.random.default_rng(1)
    H = W = 24
    lab = np.zeros((H, W), int)
    lab[5:15, 4:18] = 1
    lab[16:22, 8:22] = 2
    cb = np.array([0.2, 0.5, 0.8])
    f = cb[lab] + 0.05 * rng.standard_normal((H, W))
    lam, gamma = 1 / 32, 1 / 5
    st = O.nl_admm_run(f, cb, lam, gamma, 1500)
    r = st["fp_res"]
    assert np.all(np.diff(r) <= 1e-12 * r[:-1] + 1e-14)
    nbr = st["nbr"]
    assert np.abs(gamma * st["s"] + O.nl_Dt(nbr, st["bv"]) + st["bw"]).max() < 1e-3
    assert np.abs(st["u"] - st["w"]).max() < 1e-3
    nb = np.sqrt((st["bv"] ** 2).sum(axis=(0, 1)))
    assert nb.max() <= gamma * lam * (1 + 1e-12)
    assert (st["labels"] != lab).mean() < 0.01


def test_constant_image_single_label(O):
    cb = np.array([0.1, 0.45, 0.9])
    f = np.full((14, 16), cb[2])
    st = O.nl_admm_run(f, cb, 0.1, 0.5, 100)
    assert np.all(st["labels"] == 2)
    assert np.abs(st["w"][2] - 1.0).max() < 1e-6


def test_energy_decreases_and_denoises(O):
    rng = np.random.default_rng(synth.seed_for(0, 13))
    cb = np.array([0.2, 0.5, 0.8])
    img, lab = synth.ellipse_image(48, 48, cb[:, None], rng, sigma=0.12)
    nbr, deg = O.nl_graph(img)
    s = O.data_term(img, cb)
    st = O.nl_zero_state(3, 10, 48, 48)
    O.nl_admm_iterate(st, s, nbr, 1 / 32, 0.2, 1)
    e1 = O.nl_energy(st["w"], s, nbr, 1 / 32)
    O.nl_admm_iterate(st, s, nbr, 1 / 32, 0.2, 99)
    assert O.nl_energy(st["w"], s, nbr, 1 / 32) < e1
    labels, _ = O.labels(st["w"])
    assert (labels != lab).mean() < (s.argmin(0) != lab).mean()
