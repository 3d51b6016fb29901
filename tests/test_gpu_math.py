"""The library's FP32 reciprocal cube root (Newton step from hardware
base-2 log/exp, used by the charge kernel) against an FP64 reference and
against CUDA's rcbrtf, over 1e-2 .. 1e4: within 2e-7 relative (about 1.7
ulp), and never more than twice rcbrtf's own worst error."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1802_07871_gb300", "csrc")


def test_rcbrt_accuracy(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "rcbrt_probe")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC,
                    "-I", os.path.join(os.path.dirname(HERE), "include"),
                    os.path.join(HERE, "cuda", "rcbrt_probe.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    n, ea, eb = int(out[0]), float(out[1]), float(out[2])
    assert n == 1 << 20
    assert ea < 2e-7, (ea, eb)
    assert ea <= 2.0 * max(eb, 6e-8), (ea, eb)
