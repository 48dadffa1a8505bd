"""CPU check of the TENO6-A face arithmetic the FP64 kernels run (teno_math.cuh with the generated
teno_coeffs.cuh: scale sensors, the cut-off as thresholds on the smallest sensor, the paired
six-cell smoothness measures of a window and its mirror image, the table of normalised weights),
compiled for the host by nvcc and compared with the oracle's TENO6-A (Sec. 3.1) on seeded windows:
smooth, stepped, noisy, oscillating and near-zero data.  Both face states and the cut-off of every
window must agree to rounding (relative 1e-13 of the window's scale)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from oracle import teno


def windows(n=6000, seed=11):
    rng = np.random.default_rng(seed)
    x = np.arange(6) - 2.0
    out = []
    for k in range(n):
        kind = k % 5
        base = rng.uniform(0.5, 2.0)
        if kind == 0:      # smooth: low-order polynomial with a small slope
            c = rng.normal(size=4) * 10.0 ** rng.uniform(-6, -1)
            q = base + c[0] * x + c[1] * x ** 2 + c[2] * x ** 3
        elif kind == 1:    # a step somewhere in the window
            j = rng.integers(1, 6)
            q = np.where(np.arange(6) < j, base, base * rng.uniform(0.1, 3.0))
        elif kind == 2:    # noise on a constant
            q = base + 10.0 ** rng.uniform(-8, -1) * rng.normal(size=6)
        elif kind == 3:    # grid-scale oscillation
            q = base + 10.0 ** rng.uniform(-4, -1) * (-1.0) ** np.arange(6)
        else:              # near zero with a bump (the limiter's regime)
            q = 1e-3 * rng.uniform(0.5, 1.5) + rng.uniform(0, 1) * np.exp(-((x - rng.uniform(-2, 3)) / 0.8) ** 2)
        out.append(q)
    return np.array(out)


def test_face_states_match_the_oracle(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "check_teno_math"
    src = os.path.join(ROOT, "tests", "native", "check_teno_math.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-diag-suppress", "177", src, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    Q = windows()
    inp = "\n".join(" ".join("%.17g" % v for v in q) for q in Q) + "\n"
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
    got = np.array([[float(t) for t in line.split()] for line in out.strip().splitlines()])
    assert got.shape == (len(Q), 3)
    cols = [Q[:, j] for j in range(6)]
    wl = teno.teno6a(cols)
    wr = teno.teno6a(cols[::-1])
    ct = teno.cutoff(cols)
    scale = np.max(np.abs(Q), axis=1)
    assert np.array_equal(got[:, 2], ct)
    assert np.max(np.abs(got[:, 0] - wl) / scale) <= 1e-13
    assert np.max(np.abs(got[:, 1] - wr) / scale) <= 1e-13
