"""The split-TF32 tcgen05 form of the FP32 factor's bulk update (tests/csrc/tc_update_check.cu):
its 128 x 128 x 64 tile products match an FP64 CPU product to 1e-5 relative (measured ~1.1e-6:
TF32 rounding of the hi parts and the dropped lo*lo term), with and without the triangular mask,
on ragged sizes.  The program checks itself; this test builds it for sm_103a and runs it."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tcgen05_split_tf32_update(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "tc_update_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "csrc", "tc_update_check.cu")], check=True, capture_output=True, timeout=600)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(out.stdout)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout + out.stderr
