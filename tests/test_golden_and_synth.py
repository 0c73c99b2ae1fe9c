"""Fixtures printed in the paper, and the seeded input generators."""

import os

import numpy as np
import pytest

from paper_1112_1805_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split("=", 1)
            out[k.strip()] = v.split()
    return out


def test_remark1_count(oracle_mod):
    assert oracle_mod.num_filters(4) == int(_golden()["images_at_four_scales"][0])


def test_fish_codebook_rgb_data_term(oracle_mod):
    # Sec. 4, RGB data term: s = ||(f_R,f_G,f_B) - (c_R,c_G,c_B)||_2^2 with the
    # printed fish codebook; a pixel equal to a codebook colour has zero cost
    # for that label only.
    g = _golden()
    cb = np.array([[float(x) for x in g[f"fish_codebook_{c}"]] for c in "RGB"]).T  # [K=4][C=3]
    f = np.zeros((3, 1, 4))
    for k in range(4):
        f[:, 0, k] = cb[k]
    s = oracle_mod.data_term(f, cb)
    assert s.shape == (4, 1, 4)
    assert np.all(np.diag(s[:, 0, :]) == 0.0)
    off = s[:, 0, :][~np.eye(4, dtype=bool)]
    assert off.min() > 0.05
    assert abs(s[1, 0, 0] - ((cb[0] - cb[1]) ** 2).sum()) < 1e-15


def test_scale_weights_follow_printed_pattern():
    g = _golden()
    pat = [float(x) for x in g["fish_shearlet"][5:10]]
    assert np.allclose(synth.scale_weights(1.0, 4), pat)


def test_generators_are_seeded_and_shaped():
    a, la, wl = synth.make_workload_image("ellipses64")
    b, lb, _ = synth.make_workload_image("ellipses64")
    assert np.array_equal(a, b) and np.array_equal(la, lb)
    assert a.shape == (1, 64, 64) and la.max() < wl.K
    c, lc, wl2 = synth.make_workload_image("bezier512")
    assert c.shape == (1, 512, 512) and set(np.unique(lc)) == set(range(wl2.K))
    shapes = synth.batch_shapes()
    assert len(shapes) == 64 and shapes[0][:2] == (384, 640)
    for H, W, K, J in shapes:
        assert 2 <= K <= 6 and J == int(np.floor(0.5 * np.log2(min(H, W))))


@pytest.mark.parametrize("lam", [0.1, 1.0])
def test_scale_weights_shape(lam):
    L = synth.scale_weights(lam, 5)
    assert L[0] == 0 and np.allclose(L[2:] / L[1:-1], 2.0)
