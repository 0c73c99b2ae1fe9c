"""Pins for the oracle's shearlet transform S and its adjoint (eq. wichtig,
the Theorem, the synthesis paragraph after it, eq. important)."""

import numpy as np
import pytest

SIZES = [(64, 64, 2), (96, 160, 3), (30, 50, 2), (15, 25, 1), (8, 8, 1)]


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


@pytest.mark.parametrize("H,W,J", SIZES)
def test_parseval_reconstruction(O, H, W, J):
    # eq. important: S^T S = I, and ||S u|| = ||u|| (Parseval frame).
    rng = np.random.default_rng(H * W + J)
    u = rng.standard_normal((2, H, W))
    c, mi = O.analyze(u, J, return_imag=True)
    assert c.shape == (2, O.num_filters(J), H, W)
    assert mi < 1e-12  # real filters that are even under the DFT partner map
    r = O.synthesize(c, J)
    assert np.abs(r - u).max() < 1e-12
    assert abs(np.linalg.norm(c) / np.linalg.norm(u) - 1.0) < 1e-13


@pytest.mark.parametrize("H,W,J", SIZES)
def test_adjointness(O, H, W, J):
    # <S u, c> = <u, S^T c> for arbitrary (not only analysis) coefficients.
    rng = np.random.default_rng(7 + H)
    u = rng.standard_normal((H, W))
    c = rng.standard_normal((O.num_filters(J), H, W))
    lhs = (O.analyze(u, J) * c).sum()
    rhs = (u * O.synthesize(c, J)).sum()
    assert abs(lhs - rhs) < 1e-11 * np.abs(c).sum() ** 0.5


def test_frame_is_redundant(O):
    # Parseval frame but not a basis: S S^T != I (U U^T = I only for bases).
    rng = np.random.default_rng(3)
    c = rng.standard_normal((O.num_filters(1), 16, 16))
    cc = O.analyze(O.synthesize(c, 1), 1)
    assert np.abs(cc - c).max() > 0.1


@pytest.mark.parametrize("H,W,J", [(8, 8, 1), (12, 10, 1), (8, 12, 2)])
def test_coefficients_are_inner_products_with_translated_atoms(O, H, W, J):
    # eq. wichtig: SH(f)(kappa, j, k, m) = <f, psi_{j,k,m}> with
    # psi_hat_{j,k,m}(omega) = W(omega) exp(-2 pi i <omega, m>/N).  The atoms are
    # synthesised by the defining sum and the inner products taken directly.
    rng = np.random.default_rng(11)
    f = rng.standard_normal((H, W))
    F = O.filters(H, W, J)
    coef = O.analyze(f, J)
    a = np.arange(H)[:, None]
    b = np.arange(W)[None, :]
    for fi in range(F.shape[0]):
        for m1, m2 in [(0, 0), (1, 2), (H - 1, W // 2), (3, W - 1)]:
            # psi_{f,m}(x) = N^-2 sum_omega W(omega) exp(2 pi i <omega, x - m>/N)
            atom = np.zeros((H, W), complex)
            for n1 in range(H):
                for n2 in range(W):
                    if F[fi, n1, n2] == 0.0:
                        continue
                    atom += F[fi, n1, n2] * np.exp(2j * np.pi * (n1 * (a - m1) / H + n2 * (b - m2) / W))
            atom /= H * W
            assert np.abs(atom.imag).max() < 1e-12
            ip = (f * np.conj(atom)).sum()
            assert abs(ip - coef[fi, m1, m2]) < 1e-12


def test_translation_invariance(O):
    # The undecimated transform commutes with cyclic shifts of the image.
    rng = np.random.default_rng(2)
    u = rng.standard_normal((32, 48))
    c = O.analyze(u, 2)
    cs = O.analyze(np.roll(u, (5, -7), axis=(0, 1)), 2)
    assert np.abs(np.roll(c, (5, -7), axis=(1, 2)) - cs).max() < 1e-12


def test_lowpass_of_constant(O):
    # A constant image lives at omega = 0 where only the low-pass is non-zero.
    u = np.full((16, 16), 0.7)
    c = O.analyze(u, 2)
    assert np.abs(c[0] - 0.7).max() < 1e-14
    assert np.abs(c[1:]).max() < 1e-14
