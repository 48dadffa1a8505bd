"""The kernels' Newton-Raphson reciprocal against CUDA's IEEE division on the GPU."""
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
