"""GPU parity: filter bank and shearlet transform through the C ABI vs the oracle.

Tolerances: the bank is FP64-evaluated and rounded once to FP32, so it must
match the oracle to 2 FP32 ulps of 1 (2.4e-7).  The transforms run FP32 FFTs
whose rounding error grows like eps * log2(H W); the bound used is 2e-5 of the
largest coefficient (eps = 6e-8, log2(512^2) = 18, a safety factor of ~20)."""

import numpy as np
import pytest

from tests.gpu_util import half_plane, need_cuda, rel_max_err

pytestmark = pytest.mark.gpu

SIZES = [(8, 8, 1), (64, 64, 2), (96, 160, 3), (30, 50, 2), (15, 16, 1), (384, 640, 4), (512, 512, 4),
         (128, 96, 6)]


@pytest.fixture(scope="module")
def torch_mod():
    return need_cuda()


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


@pytest.mark.parametrize("H,W,J", SIZES)
def test_bank_matches_oracle(torch_mod, O, H, W, J):
    from paper_1112_1805_gb300.api import FilterBank

    fb = FilterBank(H, W, J)
    assert fb.eta == O.num_filters(J)
    got = fb.spectra().cpu().numpy().astype(np.float64)
    ref = half_plane(O.filters(H, W, J))
    assert np.abs(got - ref).max() <= 2.4e-7
    # partition of unity over the full plane, from the stored half plane
    assert np.abs((got ** 2).sum(0) - 1).max() < 1e-6


@pytest.mark.parametrize("H,W,J", SIZES)
def test_analyze_matches_oracle(torch_mod, O, H, W, J):
    torch = torch_mod
    from paper_1112_1805_gb300.api import FilterBank

    rng = np.random.default_rng(H * 7 + W)
    u = rng.standard_normal((2, H, W))
    fb = FilterBank(H, W, J)
    coef = fb.analyze(torch.tensor(u, dtype=torch.float32, device="cuda")).cpu().numpy()
    ref = O.analyze(u.astype(np.float32).astype(np.float64), J)
    assert coef.shape == ref.shape
    assert rel_max_err(coef, ref) < 2e-5


@pytest.mark.parametrize("H,W,J", SIZES)
def test_synthesize_matches_oracle(torch_mod, O, H, W, J):
    torch = torch_mod
    from paper_1112_1805_gb300.api import FilterBank

    rng = np.random.default_rng(H * 11 + W)
    c = rng.standard_normal((2, O.num_filters(J), H, W)).astype(np.float32)
    fb = FilterBank(H, W, J)
    got = fb.synthesize(torch.tensor(c, device="cuda")).cpu().numpy()
    ref = O.synthesize(c.astype(np.float64), J)
    assert rel_max_err(got, ref) < 2e-5


@pytest.mark.parametrize("H,W,J", [(64, 64, 2), (384, 640, 4), (512, 512, 4), (2048, 2048, 5)])
def test_parseval_on_device(torch_mod, H, W, J):
    # eq. important: S^T S = I, and ||S u|| = ||u||, at sizes up to the RGB workload.
    torch = torch_mod
    from paper_1112_1805_gb300.api import FilterBank

    g = torch.Generator(device="cuda").manual_seed(3)
    u = torch.randn((1, H, W), device="cuda", generator=g)
    fb = FilterBank(H, W, J)
    c = fb.analyze(u)
    r = fb.synthesize(c)
    assert float((r - u).abs().max()) < 2e-5 * float(u.abs().max())
    assert abs(float(c.double().norm() / u.double().norm()) - 1) < 1e-5


def test_bad_sizes_rejected(torch_mod):
    from paper_1112_1805_gb300 import binding as B

    for H, W, J in [(7, 8, 1), (8, 9, 1), (14, 16, 1), (64, 44, 2), (4096, 64, 2), (64, 64, 0), (64, 64, 7)]:
        with pytest.raises(B.ShearsegError) as ei:
            B.shfilters_build(H, W, J)
        assert ei.value.code in (B.SHF_ERR_SIZE, B.SHF_ERR_ARG)
