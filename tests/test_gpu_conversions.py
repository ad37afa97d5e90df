"""The integer-pipe FP32 <-> FP64 conversions of the step kernels equal the hardware conversions.

tests/gpu_conversions.cu includes the library's internal header and compares f32_to_f64 on all
2^32 float bit patterns and f64_to_f32 on 2^28 doubles (every exponent around the float range,
exact ties, random bit patterns) with the hardware conversions, bit for bit.
"""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2003_14061_gb300", "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")


def test_integer_pipe_conversions_are_exact(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "gpu_conversions")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC, "-I", INCLUDE,
                    os.path.join(HERE, "gpu_conversions.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "f32_to_f64 mismatches 0" in out.stdout and "f64_to_f32 mismatches 0" in out.stdout, out.stdout
