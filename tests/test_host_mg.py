"""Host logic of the library, on the CPU, compiled from its own source into
host programs (no GPU call): the inverse of the multigrid's coarsest-level
operator that the exact coarsest solve applies (mgd::coarse_inverse in
csrc/mg.cu), and the width of the FP32 sweep's population offsets
(fp32::pop_idx_kind in csrc/fp32_device.cuh)."""
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


def test_population_offset_widths(tmp_path):
    """Signed 32-bit offsets while 19 N < 2^31, unsigned 32-bit while
    19 N < 2^32, 64-bit beyond; the largest offset of every case is exact in
    the width chosen."""
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "pop_idx_check")
    src = os.path.join(HERE, "host", "pop_idx_check.cu")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-w", "-o", exe, src], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {int(n): (int(k), int(e)) for n, k, e in re.findall(r"N=(\d+) kind=(\d) exact=(\d)", out)}
    assert len(got) == 9, out
    for n, (kind, exact) in got.items():
        want = 0 if 19 * n < 2 ** 31 else (1 if 19 * n < 2 ** 32 else 2)
        assert kind == want, (n, kind, want)
        assert exact == 1, (n, kind)
    assert got[113025455][0] == 0 and got[113025456][0] == 1  # 19 N crosses 2^31
    assert got[226050910][0] == 1 and got[226050911][0] == 2  # 19 N crosses 2^32
