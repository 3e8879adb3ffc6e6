"""The hand-written reverse of the per-node collision (csrc/fcd_adjoint.cuh)
against forward-mode (dual-number) derivatives of the same node function,
compiled for the host by nvcc (no GPU needed): tests/native/adjoint_node_check.cu."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_node_reverse_is_the_transpose_of_the_forward_derivative(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "adjoint_node_check")
    subprocess.check_call([nvcc, "-std=c++17", "-O1",
                           "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2410_11129_gb300", "csrc"),
                           os.path.join(HERE, "native", "adjoint_node_check.cu"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "worst relative mismatch" in out.stdout
