"""The register FFT passes' arithmetic (small DFTs with compile-time
constants and the two-phase split of every supported length), compiled for
the host by nvcc and run on the CPU against the DFT definition."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_register_fft_arithmetic_on_host(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "fftreg_check"
    cmd = [nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2506_04710_gb300", "csrc"),
           os.path.join(ROOT, "tests", "host", "fftreg_check.cu"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "checked" in r.stdout
