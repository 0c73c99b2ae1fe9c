"""Host-side check of the V-value FFTs of the v-step, fan and gather (shf_fftv.cuh).

Compiles tests/fftv_host.cu for the host with nvcc and runs it: the radix-12,
radix-20 or radix-32 first pass, the radix-4/2 (or second radix-32) passes, the
group buffer's Stockham exchanges (swizzled or padded) and the partner-lane
packing of real rows are emulated lane by lane and compared with FP64 DFTs for
the half widths 3 2^a (24..384), 5 2^a (40..640) and 1024; the column batch transforms (8 or 4 columns per
CTA, two exchange buffers) likewise for heights 24..2560.  Every exchange
layout is also checked to stay inside its buffer and to give each element its
own slot.  No GPU is needed.
"""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1112_1805_gb300", "csrc")


def test_fftv_host(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "fftv_host")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-o", exe, os.path.join(HERE, "fftv_host.cu")],
                   check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count(" ok") == 21
