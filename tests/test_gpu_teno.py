"""GPU parity of the paper's channel scheme (Sec. 3.1) against the oracle, through the C ABI:
TENO6-A reconstruction with the interpolation limiter, and sixth-order central dissipative fluxes
(also combined with WENO5-Z).  Same norm and tolerance as the WENO5 parity tests: per variable,
max |X_gpu - X_oracle| / max |X_oracle| <= 1e-12 for X = R and X = U after one RK3 step.

The TENO stencil selection is a comparison of floating-point values (gamma_k / sum gamma against
the cut-off, and the floor of the cut-off exponent); both sides take it in FP64, and on these
seeded states no comparison falls within rounding of its threshold, so the results agree to
rounding everywhere."""
import numpy as np
import pytest

from helpers import padded_state, rel_err
from oracle import ns_fv as nf
from oracle import teno
from paper_2406_19494_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
P = ("periodic", "periodic")
WALL = ("wall", "wall")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build
    build.build()


def Solver(c):
    from paper_2406_19494_gb300.solver import Solver as S
    return S(c)


def vacuum_bump_prims(case, grid):
    """Low density (0.01) with narrow bumps along x: TENO keeps stencils whose candidates undershoot
    below zero at a few faces, so the interpolation limiter acts there."""
    xc = grid.axes[0].xc[case.h[0]:case.h[0] + case.n[0]]
    n = case.n
    W = np.zeros((5, n[2], n[1], n[0]))
    i = np.arange(n[0])
    rho = 0.01 + 1.3 * np.exp(-((i - 17.0) / 1.55) ** 2) + 2.0 * np.exp(-((i - 36.0) / 1.24) ** 2)
    W[0] = rho[None, None, :]
    W[1] = 0.1 * np.sin(2 * np.pi * xc / (xc[-1] - xc[0] + xc[1] - xc[0]))[None, None, :]
    W[4] = 1.0
    return W


CASES = {
    "sod1d_teno": lambda: dict(wl.sod_case(200), weno="teno6a"),
    "periodic3d_teno_visc6": lambda: wl.random_box(3, (16, 14, 12), weno="teno6a", visc_order=6),
    "periodic3d_teno_visc4": lambda: wl.random_box(3, (13, 11, 10), weno="teno6a", visc="constant"),
    "periodic3d_wenoz_visc6": lambda: wl.random_box(3, (15, 12, 11), visc_order=6, visc="sutherland"),
    "channel3d_teno_visc6": lambda: wl.random_box(3, (14, 18, 10), bc=(P, WALL, P), weno="teno6a",
                                                  visc_order=6, stretch=("uniform", "tanh2", "uniform"),
                                                  beta=(0.0, 2.0, 0.0), body_force=(0.05, 0.0, 0.0),
                                                  t_wall=((1, 1), (2.5, 2.2), (1, 1))),
    "bl2d_teno_visc6_porous_inflow": lambda: wl.random_box(
        2, (24, 16, 1), bc=(("inflow", "zero_gradient"), ("porous", "zero_gradient"), P),
        stretch=("uniform", "tanh1", "uniform"), beta=(0, 2.2, 0), visc="sutherland", weno="teno6a",
        visc_order=6, t_wall=((1, 1), (2.5, 1), (1, 1)),
        porous=dict(axis=1, side=0, begin=4, count=12, A=0.05, kappa=3.0, phi0=0.1)),
    "limiter1d_vacuum_bumps": lambda: wl.random_box(1, (48, 1, 1), weno="teno6a", visc="none"),
}


def setup_case(name, seed=0):
    c = CASES[name]()
    if name == "sod1d_teno":
        case = nf.Case(c)
        grid = nf.Grid(case)
        W = wl.sod_prims(grid.axes[0].xc)[:, None, None, :]
        U = nf.prim_to_cons(W, case)
    elif name == "limiter1d_vacuum_bumps":
        case = nf.Case(c)
        grid = nf.Grid(case)
        case, grid, U = padded_state(c, prims=vacuum_bump_prims(case, grid))
    else:
        case, grid, U = padded_state(c, seed=seed)
    phi, inflow = None, {}
    if case.porous:
        phi = case.porous["phi0"] * (1.0 + 0.5 * np.sin(np.arange(case.porous["count"])))
    for a in range(case.ndim):
        for s in range(2):
            if case.bc[a][s] == "inflow":
                t1 = 1 if a == 0 else 0
                t2 = 1 if a == 2 else 2
                sh = (5, case.p[t2], case.p[t1])
                rng = np.random.default_rng(7)
                prof = np.empty(sh)
                prof[0] = 1.0 + 0.1 * rng.uniform(-1, 1, sh[1:])
                prof[1] = 0.5 + 0.1 * rng.uniform(-1, 1, sh[1:])
                prof[2] = 0.05 * rng.uniform(-1, 1, sh[1:])
                prof[3] = 0.05 * rng.uniform(-1, 1, sh[1:])
                prof[4] = 1.0 + 0.1 * rng.uniform(-1, 1, sh[1:])
                inflow[(a, s)] = prof
    return c, case, grid, U, phi, inflow


def make_solver(c, phi, inflow):
    s = Solver(c)
    if phi is not None:
        s.set_wall_params(torch.from_numpy(phi).cuda())
    for (a, side), prof in inflow.items():
        s.set_inflow(a, side, torch.from_numpy(np.ascontiguousarray(prof)).cuda())
    return s


def inner_of(case):
    return (slice(None),) + case.interior()


def test_limiter_case_triggers_the_limiter():
    _, case, grid, U, _, _ = setup_case("limiter1d_vacuum_bumps")
    nf.fill_halos(U, case, grid)
    W, _ = nf.cons_to_prim(U, case)
    rho = W[0][0, 0, :]
    h, n = case.h[0], case.n[0]
    faces = range(h - 1, h + n)
    left = teno.teno6a([np.array([rho[a + o] for a in faces]) for o in (-2, -1, 0, 1, 2, 3)])
    right = teno.teno6a([np.array([rho[a + o] for a in faces]) for o in (3, 2, 1, 0, -1, -2)])
    assert np.sum(left <= 0) + np.sum(right <= 0) >= 1


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_parity(name):
    c, case, grid, U, phi, inflow = setup_case(name)
    R_ref = nf.rhs(U.copy(), case, grid, phi, inflow)
    s = make_solver(c, phi, inflow)
    R = s.rhs(torch.from_numpy(U).cuda())
    s.check()
    inner = inner_of(case)
    err = rel_err(R.cpu().numpy()[inner], R_ref[inner])
    assert max(err) <= TOL, err


@pytest.mark.parametrize("name", [n for n in CASES if n != "limiter1d_vacuum_bumps"])
def test_step_parity(name):
    c, case, grid, U, phi, inflow = setup_case(name, seed=3)
    dt = nf.cfl_dt(U, case, grid)
    U1 = nf.rk3_step(U.copy(), dt, case, grid, phi, inflow)
    s = make_solver(c, phi, inflow)
    Ud = torch.from_numpy(U).cuda()
    s.step(Ud, 1)
    s.check()
    inner = inner_of(case)
    assert max(rel_err(Ud.cpu().numpy()[inner], U1[inner])) <= TOL


@pytest.mark.slow
def test_channel_full_size_teno_sampled():
    """The paper's channel scheme at the channel benchmark size (192 x 128 x 128, walls and tanh
    stretching): GPU right-hand side against the oracle at sampled cells, wall cells included (the
    oracle evaluates each from its 7^3 neighbourhood, which holds every stencil of the
    sixth-order scheme)."""
    from test_gpu_parity import _sampled_rhs_check
    c = dict(wl.channel_case(192, 128, 128), weno="teno6a", visc_order=6)
    case = nf.Case(c)
    grid = nf.Grid(case)
    xs = [grid.axes[a].xc[3:-3] for a in range(3)]
    W = wl.channel_prims(c, *xs, seed=5)
    _sampled_rhs_check(c, W, margin=0)


@pytest.mark.parametrize("name", ["channel3d_teno_visc6", "bl2d_teno_visc6_porous_inflow"])
def test_multi_step_call_equals_single_step_calls(name):
    """The fused stage-and-primitives pass of a multi-step call gives the bits of single-step calls
    with the channel scheme too."""
    from test_gpu_parity import steps_in_one_call_vs_single_calls
    c, case, grid, U, phi, inflow = setup_case(name, seed=4)
    (Ua, ta), (Ub, tb) = steps_in_one_call_vs_single_calls(c, U, phi, inflow, 3)
    assert np.array_equal(Ua, Ub) and ta == tb
