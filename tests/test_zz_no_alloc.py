"""fluid_rhs_noalloc: the allocation-free right-hand side, for callers that cannot call cudaMalloc
(a host that owns device memory through its own pool, or a caller that cannot take cudaMalloc's
implicit synchronisation).  Its output must equal fluid_rhs's (the solver-based entry point) and
the oracle's right-hand side within the parity tolerance, on consecutive calls that share the
fixed scratch array, for every reconstruction (WENO5-JS, WENO5-Z, TENO6-A) and both orders of the
dissipative stencils.

Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

from helpers import padded_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
P = ("periodic", "periodic")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build
    build.build()


def _noalloc(case_dict, U):
    from paper_2406_19494_gb300 import native
    lib = native.lib()
    cfg = native.config_from_case(case_dict)
    R = torch.zeros_like(U)
    buf = ctypes.create_string_buffer(256)
    st = lib.fluid_rhs_noalloc(ctypes.byref(cfg), ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), buf, 256)
    return st, buf.value.decode(), R


def _reference(case_dict, U):
    from paper_2406_19494_gb300.solver import Solver
    s = Solver(case_dict)
    return s.rhs(U)


def _compare(case_dict, seed):
    from oracle import ns_fv as nf
    case, grid, Uh = padded_state(case_dict, seed=seed)
    U = torch.from_numpy(Uh).cuda()
    st, msg, R = _noalloc(case_dict, U)
    assert st == 0, msg
    Rref = _reference(case_dict, U)
    torch.cuda.synchronize()
    inner = (slice(None),) + case.interior()
    a, b = R.cpu().numpy()[inner], Rref.cpu().numpy()[inner]
    for v in range(5):
        m = np.max(np.abs(b[v]))
        assert np.max(np.abs(a[v] - b[v])) <= TOL * m, v
    # the oracle, with the porous parameters at their reference value as the entry point takes them
    pz = case_dict.get("porous")
    phi = np.full(pz["count"], pz["phi0"]) if pz else None
    Ro = nf.rhs(Uh.copy(), case, grid, phi)[inner]
    for v in range(5):
        m = np.max(np.abs(Ro[v]))
        assert np.max(np.abs(a[v] - Ro[v])) <= TOL * m, ("oracle", v)
    # the halos of R are untouched, as with fluid_rhs
    Rh = R.cpu().numpy()
    mask = np.ones(Rh.shape[1:], bool)
    mask[case.interior()] = False
    assert np.all(Rh[:, mask] == 0.0)


def test_noalloc_matches_fluid_rhs_on_consecutive_calls():
    from paper_2406_19494_gb300 import workloads as wl
    walls = wl.random_box(3, (16, 20, 12), bc=(P, ("wall", "wall"), P), stretch=("uniform", "tanh2", "uniform"),
                          beta=(0.0, 2.0, 0.0), body_force=(0.05, 0.0, 0.0), t_wall=((1, 1), (2.5, 2.5), (1, 1)))
    periodic = wl.random_box(3, (20, 18, 16))
    porous2d = wl.random_box(2, (24, 16, 1), bc=(("zero_gradient", "zero_gradient"), ("porous", "zero_gradient"), P),
                             stretch=("uniform", "tanh1", "uniform"), beta=(0, 2.2, 0), visc="sutherland",
                             t_wall=((1, 1), (2.5, 1), (1, 1)),
                             porous=dict(axis=1, side=0, begin=4, count=12, A=0.05, kappa=3.0, phi0=0.1))
    teno6 = wl.random_box(3, (14, 16, 10), bc=(P, ("wall", "wall"), P), weno="teno6a", visc_order=6,
                          stretch=("uniform", "tanh2", "uniform"), beta=(0.0, 1.5, 0.0),
                          t_wall=((1, 1), (1.4, 1.2), (1, 1)))
    js = wl.random_box(3, (13, 11, 9), weno="js", visc="constant")
    z6 = wl.random_box(2, (18, 14, 1), visc_order=6, visc="sutherland")
    # two calls in a row on the same configuration, then other configurations reusing the array
    _compare(walls, seed=1)
    _compare(walls, seed=2)
    _compare(periodic, seed=3)
    _compare(porous2d, seed=4)
    _compare(teno6, seed=5)
    _compare(teno6, seed=6)
    _compare(js, seed=7)
    _compare(z6, seed=8)


def test_noalloc_rejects_oversized_grids_and_inflow():
    from paper_2406_19494_gb300 import native
    from paper_2406_19494_gb300 import workloads as wl
    big = wl.tgv_case(64)
    U = torch.zeros((5, 70, 70, 70), dtype=torch.float64, device="cuda")
    st, msg, _ = _noalloc(big, U)
    assert st == native.FLUID_EINVAL and "16 MiB" in msg, msg
    inflow = wl.random_box(2, (12, 8, 1), bc=(("inflow", "zero_gradient"), P, P))
    U = torch.zeros((5, 1, 14, 18), dtype=torch.float64, device="cuda")
    st, msg, _ = _noalloc(inflow, U)
    assert st == native.FLUID_ENOTSUP and "inflow" in msg, msg


def test_noalloc_size_limits_and_precision():
    """The stated limits: 45^3 viscous and 64^3 inviscid fit the fixed array, one cell more per
    axis does not; the mixed form is not offered."""
    from paper_2406_19494_gb300 import native
    from paper_2406_19494_gb300 import workloads as wl
    for n, visc, ok in ((45, "power", True), (46, "power", False), (64, "none", True), (65, "none", False)):
        c = wl.random_box(3, (n, n, n), visc=visc)
        U = torch.zeros((5, n + 6, n + 6, n + 6), dtype=torch.float64, device="cuda")
        U[0] = 1.0
        U[4] = 2.5
        st, msg, R = _noalloc(c, U)
        if ok:
            assert st == 0, msg
            torch.cuda.synchronize()
            assert float(R.abs().max()) == 0.0          # a fluid at rest stays at rest
        else:
            assert st == native.FLUID_EINVAL and "16 MiB" in msg, msg
    lib = native.lib()
    cfg = native.config_from_case(wl.random_box(3, (8, 8, 8)), precision="mixed")
    U = torch.zeros((5, 14, 14, 14), dtype=torch.float64, device="cuda")
    buf = ctypes.create_string_buffer(256)
    st = lib.fluid_rhs_noalloc(ctypes.byref(cfg), ctypes.c_void_p(U.data_ptr()),
                               ctypes.c_void_p(torch.zeros_like(U).data_ptr()), None, buf, 256)
    assert st == native.FLUID_ENOTSUP and b"FP64" in buf.value
