"""Host logic of the multigrid preconditioner, on the CPU: the inverse of the
coarsest level's operator that the exact coarsest solve applies
(mgd::coarse_inverse in csrc/mg.cu), compiled from the library's own source
into a host program (no GPU call)."""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_coarse_inverse(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "coarse_inverse_check")
    src = os.path.join(HERE, "host", "coarse_inverse_check.cu")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-w", "-o", exe, src], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    spd = re.search(r"spd ok=(\d) err=(\S+) dead_zero=(\d)", out)
    assert spd, out
    assert spd.group(1) == "1"
    assert float(spd.group(2)) < 1e-5  # A inv = I to FP32 rounding of the inverse
    assert spd.group(3) == "1"        # the zero-diagonal node stays a zero of the correction
    assert re.search(r"singular ok=0", out), out  # a singular operator keeps the Jacobi sweeps
