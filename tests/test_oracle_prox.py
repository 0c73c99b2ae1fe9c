"""Pins for the proximal maps of Sec. 3: soft shrinkage (v-step) and the
pixelwise projection onto the unit simplex (w-step)."""

import itertools

import numpy as np
import pytest


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def test_soft_shrink_is_prox_of_abs(O):
    # S_t(x) = argmin_v t|v| + 1/2 (v - x)^2, checked by brute-force minimisation.
    grid = np.linspace(-4, 4, 800001)
    for t in (0.0, 0.3, 1.7):
        for x in (-3.1, -1.7, -0.2, 0.0, 0.29, 0.31, 2.5):
            obj = t * np.abs(grid) + 0.5 * (grid - x) ** 2
            vmin = grid[np.argmin(obj)]
            assert abs(O.soft_shrink(np.array([x]), t)[0] - vmin) < 2e-5, (t, x)


def test_soft_shrink_plus_clip_is_identity(O):
    # x = S_t(x) + clip(x, -t, t): the split b_v = g_v - v used by the dual update.
    rng = np.random.default_rng(0)
    x = rng.standard_normal(10000) * 3
    t = 0.8
    assert np.abs(O.soft_shrink(x, t) + np.clip(x, -t, t) - x).max() < 1e-15


def _brute_simplex(g):
    # Minimise ||x - g|| over the simplex by enumerating supports: on a support
    # A the minimiser of the equality-constrained problem is g_A + (1 - sum g_A)/|A|;
    # keep the feasible candidate closest to g.
    K = len(g)
    best, bestd = None, np.inf
    for r in range(1, K + 1):
        for A in itertools.combinations(range(K), r):
            x = np.zeros(K)
            idx = list(A)
            x[idx] = g[idx] + (1 - g[idx].sum()) / r
            if np.all(x >= -1e-15):
                d = np.linalg.norm(x - g)
                if d < bestd:
                    best, bestd = x, d
    return best


@pytest.mark.parametrize("K", [1, 2, 3, 4, 6, 8])
def test_simplex_projection_brute_force(O, K):
    rng = np.random.default_rng(K)
    g = rng.standard_normal((300, K)) * rng.uniform(0.1, 3, size=(300, 1))
    for method in ("sort", "repeated"):
        x = O.project_simplex(g, method)
        for i in range(0, 300, 7):
            assert np.abs(x[i] - _brute_simplex(g[i])).max() < 1e-12, (method, i)


@pytest.mark.parametrize("K", [2, 3, 5, 8, 16])
def test_simplex_projection_kkt(O, K):
    # KKT: x >= 0, sum x = 1, and a threshold tau with g_k - x_k = tau where
    # x_k > 0 and g_k <= tau where x_k = 0.
    rng = np.random.default_rng(100 + K)
    g = rng.standard_normal((2000, K)) * 2
    x = O.project_simplex(g)
    assert np.all(x >= 0)
    assert np.abs(x.sum(1) - 1).max() < 1e-13
    for i in range(2000):
        pos = x[i] > 0
        tau = (g[i][pos] - x[i][pos]).mean()
        assert np.abs(g[i][pos] - x[i][pos] - tau).max() < 1e-13
        assert np.all(g[i][~pos] <= tau + 1e-13)
    # the paper's repeated hyperplane projection reaches the same point
    assert np.abs(O.project_simplex(g, "repeated") - x).max() < 1e-14


def test_simplex_projection_hyperplane_case(O):
    # When the hyperplane projection g + (1 - sum g)/q is already non-negative
    # it is the answer (first step of the paper's construction).
    g = np.array([[0.3, 0.2, 0.1, 0.0], [1.0, 1.0, 1.0, 1.0]])
    x = O.project_simplex(g)
    assert np.abs(x[0] - (g[0] + (1 - 0.6) / 4)).max() < 1e-15
    assert np.abs(x[1] - 0.25).max() < 1e-15
    # a vertex
    assert np.array_equal(O.project_simplex(np.array([[5.0, 0.0, -1.0]])), np.array([[1.0, 0.0, 0.0]]))
