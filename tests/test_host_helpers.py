"""Host-side checks of integer helpers shared by the kernels, compiled with nvcc
for the host (no GPU): the 128 x 256 tile order of the wide split product
(every tile that reaches the diagonal, each exactly once) and the exact
fixed-point trace accumulation of the batched kernel (rounding to the 2^-40
grid within half a unit; sums of grid values without rounding)."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2401_13772_gb300", "csrc")


def test_wide_tiles_and_fixed_point_traces(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "host_helpers_check")
    cmd = [nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-x", "cu",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           os.path.join(HERE, "host_helpers_check.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "wide_tile failures 0, fixed40 failures 0" in r.stdout
