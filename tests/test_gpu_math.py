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


def _small_ratio(e):
    """(p, q) with 0 < p, q <= 16 and p / q equal to e within a few ulp, else None (the rule the
    library applies to the power-law exponent)."""
    for q in range(1, 17):
        p = int(e * q + 0.5)
        if 1 <= p <= 16 and abs(p / q - e) <= 4 * 2.220446049250313e-16 * abs(e):
            return p, q
    return None


@pytest.mark.parametrize("e", [0.7, 2.0 / 3.0, 0.5, 0.75, 1.5, 0.76, 5.0])
def test_power_law_within_a_few_ulp(e):
    """The power-law viscosity ratio x^e as the kernels form it: for e = p / q with small p, q (all
    but 0.76 = 19 / 25 here) one Halley step from an FP32 estimate, within 4 ulp of x^(p/q) (taken
    in extended precision; the FP64 exponent 0.7 itself differs from 7/10 by 4e-17, which moves
    x^0.7 by that times ln x, up to 13 ulp at x = 1e14 and a fraction of an ulp near 1, where
    temperature ratios sit); elsewhere exactly the library's exp(e log x)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build, native
    build.build()
    lib = native.lib()
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(0.05, 20.0, 100000), rng.uniform(0.9, 1.1, 100000),
                        10.0 ** rng.uniform(-14.5, 14.5, 30000), 10.0 ** rng.uniform(-40, 40, 2000),
                        np.array([1.0, 2.0, 0.5, 1e-15, 1e15, 2.0 ** -49, 2.0 ** 49,
                                  np.nextafter(2.0 ** 49, 0.0), np.nextafter(2.0 ** -49, 0.0)])])
    xd = torch.from_numpy(x).cuda()
    fast, libv = torch.empty_like(xd), torch.empty_like(xd)
    st = lib.fluid_check_pow(*(ctypes.c_void_p(t.data_ptr()) for t in (xd, fast, libv)), len(xd), e,
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    f, l = fast.cpu().numpy(), libv.cpu().numpy()
    pq = _small_ratio(e)
    # the fast range [2^-B, 2^B): B = 49, or less where the FP32 estimate or x^p would leave the
    # normal range
    if pq:
        B = 49
        while B > 1 and (B * e >= 125.0 or B * pq[0] >= 1021):
            B -= 1
    inside = (x >= 2.0 ** -B) & (x < 2.0 ** B) if pq else np.zeros(x.shape, bool)
    if pq:
        ex = np.longdouble(pq[0]) / np.longdouble(pq[1])
        ref = (x[inside].astype(np.longdouble) ** ex).astype(np.float64)
        assert np.max(np.abs(f[inside] - ref) / np.spacing(ref)) <= 4.0
        # near 1 the Halley value and the library's exp(e log x) agree to an ulp or two
        near = (x > 0.9) & (x < 1.1)
        assert np.max(np.abs(f[near] - l[near]) / np.spacing(l[near])) <= 3.0
    # elsewhere the library expression itself
    assert np.array_equal(f[~inside], l[~inside])


def test_integer_widening_equals_the_conversion_instruction():
    """The mixed face kernels widen their FP32 flux changes to FP64 from the bit fields; the result
    must be the exact widening (numpy's) and the conversion instruction's, bit for bit, over
    random bit patterns, the subnormal range, signed zeros and infinities (NaN stays NaN)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build, native
    build.build()
    lib = native.lib()
    rng = np.random.default_rng(2)
    pats = rng.integers(0, 2 ** 32, 400000, dtype=np.uint64).astype(np.uint32)
    sub = rng.integers(1, 2 ** 23, 20000, dtype=np.uint64).astype(np.uint32)
    x = np.concatenate([pats.view(np.float32), sub.view(np.float32), -sub.view(np.float32),
                        np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, 1.1754942e-38, 1.1754944e-38,
                                  3.4028235e38, 1.0, -2.5], np.float32)])
    xd = torch.from_numpy(x).cuda()
    bits = torch.empty(len(x), dtype=torch.float64, device="cuda")
    cvt = torch.empty_like(bits)
    st = lib.fluid_check_widen(*(ctypes.c_void_p(t.data_ptr()) for t in (xd, bits, cvt)), len(x),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    b, c = bits.cpu().numpy(), cvt.cpu().numpy()
    with np.errstate(invalid="ignore"):
        ref = x.astype(np.float64)
    nan = np.isnan(ref)
    assert np.all(np.isnan(b[nan])) and np.all(np.isnan(c[nan]))
    assert np.array_equal(b[~nan].view(np.uint64), ref[~nan].view(np.uint64))
    assert np.array_equal(c[~nan].view(np.uint64), ref[~nan].view(np.uint64))


def test_bulk_staging_copies_and_its_bounded_wait():
    """The bulk-copy staging helpers of the mixed tiles: with the exact expected byte count the
    rows arrive in shared memory and come back unchanged, no flag; with the expected count raised
    above what the copies deliver the phase cannot complete, the bounded wait runs out, the block
    reports FLAG_STAGING and returns, and the context stays usable (a following staging call and a
    solver step still work)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build, native
    build.build()
    lib = native.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    src = torch.arange(8 * 36, dtype=torch.float32, device="cuda") * 0.5 - 7.0
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")

    def run(nrows, extra):
        dst = torch.full((8 * 36,), -1.0, dtype=torch.float32, device="cuda")
        flags.zero_()
        r = lib.fluid_check_bulk_staging(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                         nrows, extra, ctypes.c_void_p(flags.data_ptr()), st)
        assert r == 0
        torch.cuda.synchronize()
        return dst, int(flags.item())

    dst, fl = run(8, 0)
    assert fl == 0 and torch.equal(dst, src)
    dst, fl = run(3, 0)
    assert fl == 0 and torch.equal(dst[:3 * 36], src[:3 * 36]) and bool((dst[3 * 36:] == -1.0).all())
    dst, fl = run(5, 16)
    assert fl == 4 and bool((dst == -1.0).all())
    dst, fl = run(8, 0)
    assert fl == 0 and torch.equal(dst, src)
    # argument checks on the host: row count, alignment
    bad = lib.fluid_check_bulk_staging(ctypes.c_void_p(src.data_ptr() + 4), ctypes.c_void_p(src.data_ptr()),
                                       2, 0, ctypes.c_void_p(flags.data_ptr()), st)
    assert bad == native.FLUID_EINVAL
    assert lib.fluid_check_bulk_staging(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(src.data_ptr()),
                                        9, 0, ctypes.c_void_p(flags.data_ptr()), st) == native.FLUID_EINVAL
    from paper_2406_19494_gb300 import workloads as wl
    from paper_2406_19494_gb300.solver import Solver
    s = Solver(wl.tgv_case(16), precision="mixed")
    cen = [s.grid(a)[0][3:-3] for a in range(3)]
    W = np.pad(wl.tgv_prims(wl.tgv_case(16), *cen), [(0, 0)] + [(3, 3)] * 3, mode="edge")
    U = s.prim_to_cons(torch.from_numpy(W).cuda())
    s.tune_faces(0, 1)
    s.step(U, 2)
    s.check()
