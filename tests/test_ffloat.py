"""Float-float (double-word) primitives of the FP64-storage transform passes,
checked on the host against long-double arithmetic: FP64 <-> float-float
conversions by bit manipulation (round trip within 2^-47), the
double-word sum and product within the published bounds (3u^2 and a few
u^2, u = 2^-24), normalisation, and special values.  The same header is
compiled into the device passes."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_ffloat_host_check(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "ffloat_check"
    build = subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off", "-x", "cu",
                            os.path.join(HERE, "ffloat_check.cu"), "-o", str(exe)],
                           capture_output=True, text=True, timeout=600)
    assert build.returncode == 0, build.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "OK" in run.stdout
