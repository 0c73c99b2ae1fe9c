"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the oracle)."""

import numpy as np
import pytest


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def half_plane(F):
    """Full-plane oracle spectra [.., H, W] -> the stored half plane [.., H, W//2+1]."""
    return F[..., : F.shape[-1] // 2 + 1]


def rel_max_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def labels_agree(lab_gpu, lab_oracle, gap_oracle, tie=1e-4):
    """Label maps agree except where the oracle's top-two gap is below `tie`."""
    lab_gpu = np.asarray(lab_gpu)
    clear = np.asarray(gap_oracle) >= tie
    return bool(np.array_equal(lab_gpu[clear], np.asarray(lab_oracle)[clear]))
