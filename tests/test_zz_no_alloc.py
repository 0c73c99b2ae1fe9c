"""The allocation-free analysis entry point against the ordinary one.

shearlet_analyze_noalloc serves callers that cannot allocate device memory
when they run a transform (real-time loops, plugins whose host owns all
device memory).  It keeps its temporaries in one fixed device array of the
library, so this test checks that two calls in a row -- the second one
finding the first one's leftovers in that array -- both give the result of
shearlet_analyze, and that a request larger than the array is refused.

The file name sorts last so that pytest collects it after every other test:
a run that stops at its first failure has then already run the rest of the
suite when one of these tests fails.  The tests do not depend on that order;
they pass alone in a fresh process as well."""

import numpy as np
import pytest

from tests.gpu_util import need_cuda, rel_max_err

pytestmark = pytest.mark.gpu


def test_noalloc_matches_analyze_twice():
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank

    H, W, J = 192, 160, 3  # 2 channels: 2 * 30 * 192 * 81 * 8 bytes = 7.5 MB of scratch
    fb = FilterBank(H, W, J)
    gen = torch.Generator(device="cuda").manual_seed(5)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        u = torch.randn((2, H, W), device="cuda", generator=gen) * (1 + call)
        ref = fb.analyze(u)
        got = torch.full_like(ref, float("nan"))
        B.shearlet_analyze_noalloc(fb.handle, u.data_ptr(), 2, got.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rel_max_err(got.cpu().numpy(), ref.cpu().numpy()) < 2e-5, call
    fb.close()


def test_noalloc_rejects_requests_beyond_its_array():
    torch = need_cuda()
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank

    fb = FilterBank(512, 512, 4)  # one channel needs 62 * 512 * 257 * 8 bytes > 32 MiB
    # real buffers of the right sizes, so that a regression in the size check
    # would run the transform on valid memory instead of faulting
    u = torch.zeros((1, 512, 512), device="cuda")
    coef = torch.empty((fb.eta, 512, 512), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(B.ShearsegError) as ei:
        B.shearlet_analyze_noalloc(fb.handle, u.data_ptr(), 1, coef.data_ptr(), stream)
    assert ei.value.code == B.SHF_ERR_SIZE
    assert "32 MiB" in str(ei.value) or "33554432" in str(ei.value)
    torch.cuda.synchronize()
    fb.close()


def test_noalloc_refuses_a_bank_of_another_device():
    torch = need_cuda()
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs: a bank built on one device, called with the other current")
    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank

    with torch.cuda.device(0):
        fb = FilterBank(64, 64, 2)
    with torch.cuda.device(1):
        u = torch.zeros((1, 64, 64), device="cuda")
        coef = torch.empty((fb.eta, 64, 64), device="cuda")
        with pytest.raises(B.ShearsegError) as ei:
            B.shearlet_analyze_noalloc(fb.handle, u.data_ptr(), 1, coef.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
        assert ei.value.code == B.SHF_ERR_STATE
    fb.close()
