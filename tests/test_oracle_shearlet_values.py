"""Pins for individual shearlets of the oracle's bank (Sec. 2, "Finite
Discrete Shearlets": the cone shearlets psi1_hat(4^-j xi1) psi2_hat(2^j xi2/xi1
+ k), their vertical-cone mirror images and the glued seam shearlets).

The partition-of-unity, cone and evenness pins do not tell k from -k, nor the
two cones apart, so here single filters are read at chosen grid points where
the closed forms of Sec. 2 give a value by hand:

* psi1_hat(x) = sqrt(b(2x)^2 + b(x)^2) = 1 for 1 <= |x| <= 2, because there
  b(x) = sin(pi/2 v(|x|-1)) and b(2x) = cos(pi/2 v(|x|-1));
* psi2_hat(0) = sqrt(v(1)) = 1, psi2_hat(+-1/2) = sqrt(v(1/2)) = sqrt(1/2)
  (v(1/2) = 35/16 - 84/32 + 70/64 - 20/128 = 1/2), psi2_hat(w) = 0 for |w| >= 1;
* varphi(w) = 1 for |w| <= 1/2.

So at a point with 4^-j |xi1| in [1, 2] a horizontal-cone shearlet (j, k)
equals psi2_hat(2^j xi2/xi1 + k): 1 where 2^j xi2/xi1 = -k, sqrt(1/2) half a
shear step away, 0 a whole step or more away.  Frequencies are normalised per
axis, xi_a = omega_a 4^J / N_a (the reading that makes the J scales reach
Nyquist), and omega_1 belongs to the row axis."""

import math

import numpy as np
import pytest

S = math.sqrt(0.5)


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _index(O, J):
    specs = O.filter_specs(J)
    return {(int(kind), int(j), int(k)): f for f, (kind, j, k) in enumerate(specs)}


def _at(F, H, W, J, xi1, xi2):
    """Value of every filter at the grid point with normalised frequency (xi1, xi2)."""
    w1 = xi1 * H / 4 ** J
    w2 = xi2 * W / 4 ** J
    assert w1 == int(w1) and w2 == int(w2), "choose grid points"
    return F[:, int(w1) % H, int(w2) % W]


# (H, W, J): square and non-square grids (the latter pins the per-axis
# normalisation: xi2 = omega2 16 / 128 there)
GRIDS = [(64, 64, 2), (64, 128, 2), (128, 96, 2)]


@pytest.mark.parametrize("H,W,J", GRIDS)
def test_horizontal_cone_shears_sign_and_order(O, H, W, J):
    F = O.filters(H, W, J)
    idx = _index(O, J)
    # scale j = 1 (shears k = -1, 0, 1), xi1 = 5: 4^-1 xi1 = 1.25 in [1, 2]
    for xi2, want in [(-2.5, {1: 1.0, 0: 0.0, -1: 0.0}),      # 2 xi2/xi1 = -1 -> k = +1 centred
                      (2.5, {-1: 1.0, 0: 0.0, 1: 0.0}),       # +1 -> k = -1 centred
                      (0.0, {0: 1.0, 1: 0.0, -1: 0.0}),       # 0 -> k = 0 centred
                      (-1.25, {0: S, 1: S, -1: 0.0})]:         # -1/2: halfway between k = 0 and k = +1
        if (xi2 * W / 4 ** J) != int(xi2 * W / 4 ** J):
            continue
        vals = _at(F, H, W, J, 5.0, xi2)
        for k, v in want.items():
            assert vals[idx[(1, 1, k)]] == pytest.approx(v, abs=1e-14), (xi2, k)
    # scale j = 0 (k = 0 only), xi1 = -1.5 (|x| in [1, 2]): psi2_hat(xi2/xi1)
    vals = _at(F, H, W, J, -1.5, 0.0)
    assert vals[idx[(1, 0, 0)]] == pytest.approx(1.0, abs=1e-14)
    # the same point belongs to no other scale-0 shearlet and to no scale-1 one
    # (4^-1 * 1.5 < 1/2, where psi1_hat vanishes)
    for key, f in idx.items():
        if key != (1, 0, 0) and key[0] != 0:
            assert vals[f] == pytest.approx(0.0, abs=1e-14), key


@pytest.mark.parametrize("H,W,J", GRIDS)
def test_vertical_cone_mirrors_the_horizontal_one(O, H, W, J):
    F = O.filters(H, W, J)
    idx = _index(O, J)
    # roles of xi1 and xi2 exchanged: xi2 = 5, 2 xi1/xi2 = -1 -> vertical k = +1
    if (-2.5 * H / 4 ** J) != int(-2.5 * H / 4 ** J):
        pytest.skip("point not on this grid")
    vals = _at(F, H, W, J, -2.5, 5.0)
    assert vals[idx[(2, 1, 1)]] == pytest.approx(1.0, abs=1e-14)
    assert vals[idx[(2, 1, -1)]] == pytest.approx(0.0, abs=1e-14)
    assert vals[idx[(1, 1, 1)]] == pytest.approx(0.0, abs=1e-14)  # the point is in the vertical cone
    assert vals[idx[(1, 1, -1)]] == pytest.approx(0.0, abs=1e-14)


@pytest.mark.parametrize("H,W,J", GRIDS)
def test_glued_seam_shearlets(O, H, W, J):
    F = O.filters(H, W, J)
    idx = _index(O, J)
    # on the seam |xi1| = |xi2| the glued shearlet k = -2^j sign(xi2/xi1) takes
    # psi1_hat(4^-j xi1) psi2_hat(0) and its partner 0; j = 1, xi1 = 5
    for s2, kon, koff in [(1.0, -2, 2), (-1.0, 2, -2)]:
        vals = _at(F, H, W, J, 5.0, 5.0 * s2)
        assert vals[idx[(3, 1, kon)]] == pytest.approx(1.0, abs=1e-14)
        assert vals[idx[(3, 1, koff)]] == pytest.approx(0.0, abs=1e-14)
        # no cone shearlet of the scale reaches the seam (|2 xi2/xi1 + k| >= 1)
        for k in (-1, 0, 1):
            assert vals[idx[(1, 1, k)]] == pytest.approx(0.0, abs=1e-14)
            assert vals[idx[(2, 1, k)]] == pytest.approx(0.0, abs=1e-14)
    # inside the horizontal cone the glued k = -2 follows the horizontal
    # formula: xi2/xi1 = 0.75 -> psi2_hat(1.5 - 2) = sqrt(1/2); k = +2 gives
    # psi2_hat(3.5) = 0
    if (3.75 * W / 4 ** J) == int(3.75 * W / 4 ** J):
        vals = _at(F, H, W, J, 5.0, 3.75)
        assert vals[idx[(3, 1, -2)]] == pytest.approx(S, abs=1e-14)
        assert vals[idx[(3, 1, 2)]] == pytest.approx(0.0, abs=1e-14)
        assert vals[idx[(1, 1, 1)]] == pytest.approx(0.0, abs=1e-14)
        assert vals[idx[(1, 1, -1)]] == pytest.approx(S, abs=1e-14)  # psi2_hat(1.5 - 1) = sqrt(1/2)


@pytest.mark.parametrize("H,W,J", GRIDS)
def test_low_pass_near_the_origin(O, H, W, J):
    F = O.filters(H, W, J)
    idx = _index(O, J)
    vals = _at(F, H, W, J, 0.25, -0.5)  # max(|xi1|, |xi2|) = 1/2: varphi = 1, every shearlet 0
    assert vals[idx[(0, 0, 0)]] == pytest.approx(1.0, abs=1e-14)
    assert np.abs(np.delete(vals, idx[(0, 0, 0)])).max() == pytest.approx(0.0, abs=1e-14)
