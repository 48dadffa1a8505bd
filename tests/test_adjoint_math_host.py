"""CPU check of the hand-written reverse-mode arithmetic (adjoint_math.cuh) against finite
differences of the forward arithmetic (flux_math.cuh): both compiled for the host by nvcc from the
same headers the kernels include, so the derivatives of the code the GPU runs are checked here."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def test_vjps_match_finite_differences(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "check_adjoint_math"
    src = os.path.join(ROOT, "tests", "native", "check_adjoint_math.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-diag-suppress", "177", src, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    worst = {line.split()[0]: float(line.split()[1]) for line in out.strip().splitlines()}
    assert len(worst) >= 18
    for name, err in worst.items():
        # second-order differences (fourth-order for WENO) with h ~ 1e-6: truncation ~1e-7
        assert err < 2e-6, (name, err)
