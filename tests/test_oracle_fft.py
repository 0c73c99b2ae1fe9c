"""Pins for the oracle's own FFT (fft2 / ifft2 conventions of Sec. 2)."""

import numpy as np
import pytest


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


@pytest.mark.parametrize("H,W", [(8, 8), (3, 5), (6, 10), (12, 20), (7, 11), (16, 9), (1, 8), (25, 4)])
def test_fft_matches_brute_force_dft(O, H, W):
    rng = np.random.default_rng(H * 100 + W)
    x = rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
    for inv in (False, True):
        a, b = O.fft2(x, inv), O.dft2_brute(x, inv)
        assert np.abs(a - b).max() < 1e-12 * max(1.0, np.abs(b).max())


def test_brute_force_on_delta_and_constant(O):
    # fft2 of a delta at m is exp(-2 pi i <omega, m>/N); of a constant is N^2 at 0.
    H, W = 8, 8
    x = np.zeros((H, W), complex)
    x[2, 3] = 1.0
    y = O.dft2_brute(x)
    a, b = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    assert np.abs(y - np.exp(-2j * np.pi * (2 * a / H + 3 * b / W))).max() < 1e-14
    c = O.dft2_brute(np.ones((H, W), complex))
    assert abs(c[0, 0] - H * W) < 1e-12 and np.abs(c.ravel()[1:]).max() < 1e-12


@pytest.mark.parametrize("H,W", [(64, 64), (384, 640), (96, 160), (128, 30)])
def test_fft_matches_numpy(O, H, W):
    rng = np.random.default_rng(H + W)
    x = rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
    assert np.abs(O.fft2(x) - np.fft.fft2(x)).max() < 1e-10
    assert np.abs(O.fft2(x, True) - np.fft.ifft2(x)).max() < 1e-14
    assert np.abs(O.fft2(O.fft2(x), True) - x).max() < 1e-13


def test_plancherel(O):
    # <f, g> = N^-2 <f_hat, g_hat>  (Sec. 2)
    rng = np.random.default_rng(5)
    f, g = rng.standard_normal((2, 24, 40))
    lhs = (f * g).sum()
    rhs = (O.fft2(f) * np.conj(O.fft2(g))).sum().real / f.size
    assert abs(lhs - rhs) < 1e-12
