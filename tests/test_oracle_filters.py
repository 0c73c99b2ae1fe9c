"""Pins for the oracle's filter bank (Sec. 2, "Finite Discrete Shearlets",
Theorem on the Parseval frame, Remark 1)."""

import numpy as np
import pytest

SIZES = [(8, 8, 1), (64, 64, 2), (64, 64, 3), (96, 160, 3), (30, 50, 2), (15, 25, 1), (384, 640, 4),
         (512, 512, 4)]


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _freq(N):
    n = np.arange(N)
    return np.where(n < (N + 1) // 2, n, n - N)


def test_filter_count_remark1(O):
    # Remark 1: four scales give 61 coefficient images; eta = 1 + sum_j 2^(j+2).
    assert O.num_filters(4) == 61
    for J in range(1, 7):
        specs = O.filter_specs(J)
        assert len(specs) == O.num_filters(J) == 1 + sum(2 ** (j + 2) for j in range(J))
        for j in range(J):
            sj = specs[(specs[:, 0] > 0) & (specs[:, 1] == j)]
            assert len(sj) == 2 ** (j + 2)
            # h and v cones carry |k| <= 2^j - 1, glued ones k = -2^j, +2^j
            for kind in (1, 2):
                assert sorted(sj[sj[:, 0] == kind][:, 2]) == list(range(-(2 ** j) + 1, 2 ** j))
            assert sorted(sj[sj[:, 0] == 3][:, 2]) == [-(2 ** j), 2 ** j]


@pytest.mark.parametrize("H,W,J", SIZES)
def test_partition_of_unity(O, H, W, J):
    # Theorem (Parseval frame): sum_f |W_f(w)|^2 = 1 at every grid frequency.
    F = O.filters(H, W, J)
    assert F.shape == (O.num_filters(J), H, W)
    assert np.abs((F ** 2).sum(0) - 1.0).max() < 1e-13


@pytest.mark.parametrize("H,W,J", [(64, 64, 2), (96, 160, 3), (30, 50, 2), (15, 25, 1)])
def test_partition_without_symmetrisation(O, H, W, J):
    # The unsymmetrised bank is the paper's literal construction; it already
    # partitions unity pointwise, the symmetrisation keeps that property.
    F = O.filters_unsymmetrised(H, W, J)
    assert np.abs((F ** 2).sum(0) - 1.0).max() < 1e-13


@pytest.mark.parametrize("H,W,J", [(64, 64, 2), (96, 160, 3), (30, 50, 2), (15, 25, 1)])
def test_filters_even_under_dft_partner(O, H, W, J):
    # Real, even filters: W_f at n equals W_f at (-n mod N); this is what makes
    # every coefficient of a real image real.
    F = O.filters(H, W, J)
    Fp = F[:, (-np.arange(H)) % H][:, :, (-np.arange(W)) % W]
    assert np.array_equal(F, Fp)


def test_unsymmetrised_bank_is_not_even_on_nyquist(O):
    # Why the symmetrisation is needed: on the Nyquist line of an even axis the
    # DFT partner is not the continuous mirror, so sheared filters differ there.
    H = W = 64
    F = O.filters_unsymmetrised(H, W, 2)
    Fp = F[:, (-np.arange(H)) % H][:, :, (-np.arange(W)) % W]
    d = np.abs(F - Fp)
    assert d.max() > 1e-3
    off = np.ones((H, W), bool)
    off[H // 2, :] = False
    off[:, W // 2] = False
    assert d[:, off].max() == 0.0  # elsewhere the construction is already even
    # and so its coefficients of a real image are not real
    rng = np.random.default_rng(0)
    u = rng.standard_normal((H, W))
    G = np.fft.ifft2(F * np.fft.fft2(u)[None])
    assert np.abs(G.imag).max() > 1e-6


def test_lowpass_and_origin(O):
    F = O.filters(64, 64, 3)
    assert F[0, 0, 0] == 1.0
    assert np.all(F[1:, 0, 0] == 0.0)


@pytest.mark.parametrize("H,W,J", [(64, 64, 2), (96, 160, 3), (384, 640, 4)])
def test_cones(O, H, W, J):
    # Horizontal-cone shearlets vanish where |xi_2| >= |xi_1|, vertical-cone ones
    # where |xi_1| >= |xi_2| (characteristic functions of C^h, C^v).
    F = O.filters_unsymmetrised(H, W, J)
    specs = O.filter_specs(J)
    a1 = np.abs(_freq(H))[:, None] * W  # |xi_1| up to the common factor 4^J/(H W)
    a2 = np.abs(_freq(W))[None, :] * H
    for f, (kind, j, k) in enumerate(specs):
        if kind == 1:
            assert np.all(F[f][a2 >= a1] == 0.0)
        if kind == 2:
            assert np.all(F[f][a1 >= a2] == 0.0)


@pytest.mark.parametrize("H,W,J", [(64, 64, 2), (64, 64, 3), (96, 160, 3), (512, 512, 4)])
def test_scale_energy_equals_psi1(O, H, W, J):
    # Lemma (shear partition): the shears of one scale sum in square to
    # |psi1_hat(4^-j xi_main)|^2, xi_main the larger of |xi_1|, |xi_2|, with
    # xi_a = omega_a 4^J / N_a.  Checked off the Nyquist lines.
    F = O.filters_unsymmetrised(H, W, J)
    specs = O.filter_specs(J)
    x1 = np.abs(_freq(H))[:, None] * 4.0 ** J / H
    x2 = np.abs(_freq(W))[None, :] * 4.0 ** J / W
    xm = np.maximum(x1, x2)
    for j in range(J):
        sel = (specs[:, 0] > 0) & (specs[:, 1] == j)
        tot = (F[sel] ** 2).sum(0)
        expect = O.window("psi1", (xm * 4.0 ** (-j)).ravel()).reshape(H, W) ** 2
        assert np.abs(tot - expect).max() < 1e-13, j
    # and the low-pass is varphi(max(|xi_1|, |xi_2|))
    assert np.abs(F[0] - O.window("varphi", xm.ravel()).reshape(H, W)).max() == 0.0


def test_transpose_closure_square(O):
    # For square images the filter set is closed under transposition (h <-> v
    # with the same j, k): the reason the row/column orientation is immaterial.
    H = W = 64
    J = 3
    F = O.filters(H, W, J)
    specs = [tuple(s) for s in O.filter_specs(J)]
    for f, (kind, j, k) in enumerate(specs):
        partner = {0: 0, 1: 2, 2: 1, 3: 3}[kind]
        g = specs.index((partner, j, k))
        assert np.array_equal(F[f].T, F[g]), (kind, j, k)


def test_literal_grid_when_2J_equals_log2N(O):
    # For N = 4^J the normalisation xi = omega 4^J / N is the identity, i.e. the
    # integer frequencies of the paper: scale j = J-1 reaches the Nyquist
    # frequency N/2 = 4^J / 2 inside the flat part of the scale sum.
    N, J = 64, 3
    F = O.filters(N, N, J)
    specs = O.filter_specs(J)
    top = (specs[:, 0] > 0) & (specs[:, 1] == J - 1)
    e = (F[top] ** 2).sum(0)
    f = _freq(N)
    ring = np.maximum(np.abs(f)[:, None], np.abs(f)[None, :])
    assert np.all(np.abs(e[ring >= 2 * 4 ** (J - 1)] - 1.0) < 1e-13)
