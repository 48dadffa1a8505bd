"""The kernels' own reciprocal, reciprocal square root and square root (third-order steps from
the hardware estimates) against CUDA's IEEE division and square root on the GPU."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_newton_reciprocal_within_two_ulp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build, native
    build.build()
    lib = native.lib()
    rng = np.random.default_rng(0)
    y = np.concatenate([10.0 ** rng.uniform(-250, 250, 200000), rng.uniform(0.5, 2.0, 200000),
                        np.array([1.0, 2.0, 3.0, 1e-300, 1e300, 0.1])])
    yd = torch.from_numpy(y).cuda()
    fast, ieee = torch.empty_like(yd), torch.empty_like(yd)
    st = lib.fluid_check_rcp(ctypes.c_void_p(yd.data_ptr()), ctypes.c_void_p(fast.data_ptr()),
                             ctypes.c_void_p(ieee.data_ptr()), len(y),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    f, e = fast.cpu().numpy(), ieee.cpu().numpy()
    assert np.array_equal(e, 1.0 / y)
    ulp = np.abs(f - e) / np.spacing(np.abs(e))
    assert np.max(ulp) <= 2.0, np.max(ulp)


def test_rsqrt_and_sqrt_within_a_few_ulp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build, native
    build.build()
    lib = native.lib()
    rng = np.random.default_rng(1)
    y = np.concatenate([10.0 ** rng.uniform(-300, 300, 200000), rng.uniform(0.25, 4.0, 200000),
                        np.array([1.0, 2.0, 4.0, 0.5, 1e-300, 1e300, 71.42857142857143])])
    special = np.array([0.0, -0.0, -1.0, np.inf, 5e-324])
    yd = torch.from_numpy(np.concatenate([y, special])).cuda()
    rs, sq, ieee = torch.empty_like(yd), torch.empty_like(yd), torch.empty_like(yd)
    st = lib.fluid_check_sqrt(*(ctypes.c_void_p(t.data_ptr()) for t in (yd, rs, sq, ieee)), len(yd),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    r, q, e = rs.cpu().numpy(), sq.cpu().numpy(), ieee.cpu().numpy()
    n = len(y)
    assert np.array_equal(e[:n], np.sqrt(y))
    # square root: within 2 ulp of the correctly rounded value
    assert np.max(np.abs(q[:n] - e[:n]) / np.spacing(e[:n])) <= 2.0
    # reciprocal square root: within 3 ulp of 1/sqrt(y) (itself up to 1 ulp from the exact value)
    ref = 1.0 / np.sqrt(y)
    assert np.max(np.abs(r[:n] - ref) / np.spacing(ref)) <= 3.0
    # zero, negative, infinite and denormal inputs take the library square root
    with np.errstate(invalid="ignore"):
        assert np.array_equal(q[n:], np.sqrt(special), equal_nan=True)
