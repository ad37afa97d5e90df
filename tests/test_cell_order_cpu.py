"""The library's cell numbering (rows of cells in blocks of kz z planes), checked on the host.

tests/cell_order_check.cu includes the library's internal header and runs its row_pos,
cell_index and cell_coords on the CPU: the row numbering is a bijection in the order
(z / kz, y, z % kz), x runs fastest within a row, cell_coords inverts cell_index, and a few
positions match values worked out by hand.  No GPU is needed (nvcc builds host code).
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2003_14061_gb300", "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")


def test_cell_numbering_on_the_host(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc) and shutil.which(nvcc) is None:
        pytest.skip("no nvcc")
    exe = str(tmp_path / "cell_order_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-I", CSRC, "-I", INCLUDE,
                    os.path.join(HERE, "cell_order_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("bad 0"), out.stdout
