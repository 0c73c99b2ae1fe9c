"""Pins for the oracle's 1-D windows (Sec. 2, "Continuous Shearlets").

Each test checks an identity the paper states (or that follows from its
definitions) against the oracle's implementation; none re-types the formula
being tested."""

import numpy as np
import pytest


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def test_v_boundary_values_and_symmetry(O):
    x = np.linspace(0.0, 1.0, 10001)
    v = O.window("v", x)
    # v(x) + v(1 - x) = 1: the property behind both partitions of the Lemma.
    assert np.abs(v + O.window("v", 1.0 - x) - 1.0).max() < 1e-13  # monomial form: cancellation ~3e-14
    assert O.window("v", np.array([0.0]))[0] == 0.0
    assert abs(O.window("v", np.array([1.0]))[0] - 1.0) < 1e-15
    assert np.all(O.window("v", np.array([-3.0, -1e-9])) == 0.0)
    assert np.all(O.window("v", np.array([1.0 + 1e-9, 7.0])) == 1.0)
    assert np.all(np.diff(v) >= -1e-13)  # monotone on [0, 1] up to rounding


def test_v_is_c3_at_the_ends(O):
    # The degree-7 polynomial is the smooth step: derivatives 1..3 vanish at 0 and 1.
    h = 1e-3
    for x0 in (0.0, 1.0):
        xs = x0 + h * np.arange(-2, 3)
        d1 = (O.window("v", xs[3:4]) - O.window("v", xs[1:2])) / (2 * h)
        assert abs(d1[0]) < 1e-6  # O(h^3) for a C^3 step, O(h) otherwise


def test_supports_of_fig1(O):
    # Fig. 1 caption: supp psi1_hat = [-4,-1/2] u [1/2,4], supp psi2_hat = [-1,1].
    x = np.linspace(-6, 6, 120001)
    p1 = O.window("psi1", x)
    inside1 = (np.abs(x) > 0.5) & (np.abs(x) < 4.0)
    assert np.abs(p1[~inside1]).max() <= 1e-16  # cos(pi/2) rounds to 6e-17 at |x| = 4
    assert np.all(p1[inside1] > 0.0)
    p2 = O.window("psi2", x)
    inside2 = np.abs(x) < 1.0
    assert np.all(p2[~inside2] == 0.0)
    assert np.all(p2[inside2] > 0.0)
    assert O.window("psi2", np.array([0.0]))[0] == 1.0


def test_windows_are_even(O):
    x = np.linspace(0, 5, 5001)
    for name in ("b", "psi1", "psi2", "varphi"):
        assert np.array_equal(O.window(name, x), O.window(name, -x)), name


def test_meyer_dyadic_partition(O):
    # b^2(x) + b^2(x/2) = 1 on [2,4] (the sin/cos pieces share their argument),
    # hence sum_m b^2(2^m x) = 1 for every x != 0.
    x = np.exp(np.linspace(np.log(1e-3), np.log(1e3), 4001))
    tot = sum(O.window("b", x * 2.0 ** m) ** 2 for m in range(-20, 21))
    assert np.abs(tot - 1.0).max() < 1e-14


def test_lemma_psi1_partition(O):
    # Lemma: sum_{j>=0} |psi1_hat(2^{-2j} w)|^2 = 1 for |w| > 1.
    w = np.concatenate([np.linspace(1.0 + 1e-12, 4096.0, 20001), -np.linspace(1.0 + 1e-12, 300.0, 2001)])
    tot = sum(O.window("psi1", w * 4.0 ** (-j)) ** 2 for j in range(0, 40))
    assert np.abs(tot - 1.0).max() < 1e-14


def test_lemma_psi2_partition(O):
    # Lemma: sum_{k=-2^j}^{2^j} |psi2_hat(k + 2^j w)|^2 = 1 for |w| <= 1, j >= 0.
    w = np.linspace(-1.0, 1.0, 4001)
    for j in range(0, 6):
        tot = sum(O.window("psi2", k + 2.0 ** j * w) ** 2 for k in range(-(2 ** j), 2 ** j + 1))
        assert np.abs(tot - 1.0).max() < 1e-13, j


def test_scale_sum_piecewise_form(O):
    # The displayed piecewise form of sum_{j>=0} |psi1_hat(2^{-2j} w)|^2 next to
    # eq. OverlapPsi1_2: 0 on |w| <= 1/2, sin^2(pi/2 v(2|w|-1)) on (1/2, 1), 1 above.
    w = np.linspace(0.0, 3.0, 30001)
    tot = sum(O.window("psi1", w * 4.0 ** (-j)) ** 2 for j in range(0, 40))
    low, mid, high = w <= 0.5, (w > 0.5) & (w < 1.0), w >= 1.0
    assert np.all(tot[low] == 0.0)
    expect_mid = np.sin(0.5 * np.pi * O.window("v", 2 * w[mid] - 1)) ** 2
    assert np.abs(tot[mid] - expect_mid).max() < 1e-14
    assert np.abs(tot[high] - 1.0).max() < 1e-14


def test_overlap_identity(O):
    # eq. OverlapPsi1_2: |psi1_hat(w)|^2 + |varphi(w)|^2 = 1 for |w| in [1/2, 1].
    w = np.linspace(0.5, 1.0, 5001)
    for sgn in (1.0, -1.0):
        lhs = O.window("psi1", sgn * w) ** 2 + O.window("varphi", sgn * w) ** 2
        assert np.abs(lhs - 1.0).max() < 1e-14


def test_varphi_plateau_and_support(O):
    w = np.linspace(-3, 3, 60001)
    phi = O.window("varphi", w)
    assert np.all(phi[np.abs(w) <= 0.5] == 1.0)
    assert np.all(phi[np.abs(w) >= 1.0] == 0.0)
    mid = (np.abs(w) > 0.5) & (np.abs(w) < 1.0)
    assert np.all((phi[mid] > 0.0) & (phi[mid] <= 1.0))
    assert np.all(np.diff(phi[(w > 0.5) & (w < 1.0)]) <= 0.0)
