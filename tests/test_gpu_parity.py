"""GPU (sm_103a) parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerance (per variable v, interior cells): max |X_gpu - X_oracle| / max |X_oracle| <= 1e-12,
X = R for right-hand sides and X = U after one RK3 step.  Both sides compute in FP64; the residual
differences come from operation order and fused multiply-adds (about 1e-16 relative per
operation, amplified by the flux-difference cancellation of Eq. ODE to about 1e-14 here).

Time steps are compared at 1e-12 relative too: on tanh-stretched axes the cell width is a
difference of mapped face coordinates, each side evaluating tanh with its own math library, so a
one-ulp difference in a face coordinate x becomes ulp(x) / dx (about 1e-14) in the width.
"""
import math

import numpy as np
import pytest

from helpers import padded_state, rel_err
from oracle import ns_fv as nf
from paper_2406_19494_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
P = ("periodic", "periodic")
WALL = ("wall", "wall")
ZG = ("zero_gradient", "zero_gradient")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build
    build.build()


def Solver(c):
    from paper_2406_19494_gb300.solver import Solver as S
    return S(c)


def inner_of(case):
    return (slice(None),) + case.interior()


def inflows(c, case, grid):
    out = {}
    for a in range(case.ndim):
        for s in range(2):
            if case.bc[a][s] == "inflow":
                t1 = 1 if a == 0 else 0
                t2 = 1 if a == 2 else 2
                sh = (5, case.p[t2], case.p[t1])
                # a smooth profile over the face plane built from the interior edge state
                rng = np.random.default_rng(a * 2 + s)
                prof = np.empty(sh)
                prof[0] = 1.0 + 0.1 * rng.uniform(-1, 1, sh[1:])
                prof[1] = 0.5 + 0.1 * rng.uniform(-1, 1, sh[1:])
                prof[2] = 0.05 * rng.uniform(-1, 1, sh[1:])
                prof[3] = 0.05 * rng.uniform(-1, 1, sh[1:])
                prof[4] = 1.0 + 0.1 * rng.uniform(-1, 1, sh[1:])
                out[(a, s)] = prof
    return out


CASES = {
    "sod1d": lambda: wl.sod_case(200),
    "periodic3d_z_power": lambda: wl.random_box(3, (20, 18, 16)),
    "periodic3d_js_const": lambda: wl.random_box(3, (17, 13, 11), weno="js", visc="constant"),
    "channel3d_walls_force": lambda: wl.random_box(3, (16, 20, 12), bc=(P, WALL, P),
                                                     stretch=("uniform", "tanh2", "uniform"),
                                                     beta=(0.0, 2.0, 0.0), body_force=(0.05, 0.01, -0.02),
                                                     t_wall=((1, 1), (2.5, 2.2), (1, 1))),
    "mixed3d_adiabatic_zg_stretchx": lambda: wl.random_box(3, (14, 12, 10),
                                                             bc=(ZG, ("adiabatic", "adiabatic"), P),
                                                             stretch=("tanh1", "uniform", "uniform"),
                                                             beta=(1.5, 0.0, 0.0), visc="sutherland"),
    "bl2d_porous_inflow": lambda: wl.random_box(2, (24, 16, 1), bc=(("inflow", "zero_gradient"),
                                                                    ("porous", "zero_gradient"), P),
                                                  stretch=("uniform", "tanh1", "uniform"), beta=(0, 2.2, 0),
                                                  visc="sutherland", t_wall=((1, 1), (2.5, 1), (1, 1)),
                                                  porous=dict(axis=1, side=0, begin=4, count=12, A=0.05,
                                                              kappa=3.0, phi0=0.1)),
    "euler3d_minimal_n3": lambda: wl.random_box(3, (3, 3, 3), visc="none"),
    "visc3d_minimal_n3_walls": lambda: wl.random_box(3, (3, 3, 3), bc=(P, ("wall", "wall"), P),
                                                     t_wall=((1, 1), (1.4, 1.1), (1, 1))),
    "ragged2d_xwall": lambda: wl.random_box(2, (37, 5, 1), bc=(WALL, P, P), t_wall=((2.5, 2.6), (1, 1), (1, 1))),
}


def setup_case(name, seed=0):
    c = CASES[name]()
    if name == "sod1d":
        case = nf.Case(c)
        grid = nf.Grid(case)
        W = wl.sod_prims(grid.axes[0].xc)[:, None, None, :]
        U = nf.prim_to_cons(W, case)
    else:
        case, grid, U = padded_state(c, seed=seed)
    phi = None
    if case.porous:
        phi = case.porous["phi0"] * (1.0 + 0.5 * np.sin(np.arange(case.porous["count"])))
    return c, case, grid, U, phi, inflows(c, case, grid)


def make_solver(c, phi, inflow):
    s = Solver(c)
    if phi is not None:
        s.set_wall_params(torch.from_numpy(phi).cuda())
    for (a, side), prof in inflow.items():
        s.set_inflow(a, side, torch.from_numpy(np.ascontiguousarray(prof)).cuda())
    return s


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_parity(name):
    c, case, grid, U, phi, inflow = setup_case(name)
    R_ref = nf.rhs(U.copy(), case, grid, phi, inflow)
    s = make_solver(c, phi, inflow)
    R = s.rhs(torch.from_numpy(U).cuda())
    s.check()
    R = R.cpu().numpy()
    inner = inner_of(case)
    err = rel_err(R[inner], R_ref[inner])
    assert max(err) <= TOL, err


@pytest.mark.parametrize("name", list(CASES))
def test_dt_parity(name):
    c, case, grid, U, phi, inflow = setup_case(name)
    dt_ref = nf.cfl_dt(U, case, grid)
    s = make_solver(c, phi, inflow)
    dt = s.compute_dt(torch.from_numpy(U).cuda()).item()
    assert abs(dt - dt_ref) <= TOL * dt_ref, (dt, dt_ref)


@pytest.mark.parametrize("name", list(CASES))
def test_step_parity(name):
    c, case, grid, U, phi, inflow = setup_case(name, seed=3)
    dt = nf.cfl_dt(U, case, grid)
    U1 = nf.rk3_step(U.copy(), dt, case, grid, phi, inflow)
    U2 = nf.rk3_step(U1.copy(), nf.cfl_dt(U1, case, grid), case, grid, phi, inflow)
    s = make_solver(c, phi, inflow)
    Ud = torch.from_numpy(U).cuda()
    s.step(Ud, 1)
    s.check()
    inner = inner_of(case)
    got1 = Ud.cpu().numpy()
    assert max(rel_err(got1[inner], U1[inner])) <= TOL
    t, last = s.time()
    assert abs(last - dt) <= TOL * dt and abs(t - dt) <= TOL * dt
    # per-step parity from the oracle's own state
    Ud = torch.from_numpy(U1).cuda()
    s.step(Ud, 1)
    s.check()
    assert max(rel_err(Ud.cpu().numpy()[inner], U2[inner])) <= TOL


def _solver_with_bcs(c, phi, inflow, precision):
    from paper_2406_19494_gb300.solver import Solver as S
    s = S(c, precision=precision)
    if phi is not None:
        s.set_wall_params(torch.from_numpy(phi).cuda())
    for (a, side), prof in inflow.items():
        s.set_inflow(a, side, torch.from_numpy(np.ascontiguousarray(prof)).cuda())
    return s


def steps_in_one_call_vs_single_calls(c, U, phi, inflow, nsteps, precision="fp64", t_end=0.0):
    """(state, time) after one fluid_step call of nsteps and after nsteps calls of one step."""
    out = []
    for calls, per_call in ((1, nsteps), (nsteps, 1)):
        s = _solver_with_bcs(c, phi, inflow, precision)
        Ud = torch.from_numpy(U).cuda()
        for _ in range(calls):
            s.step(Ud, per_call, t_end=t_end)
        s.check()
        out.append((Ud.cpu().numpy(), s.time()))
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", [n for n in CASES if n != "sod1d"])
def test_multi_step_call_equals_single_step_calls(name, precision):
    """Within one fluid_step call each RK3 stage writes the primitives of its result together with
    the result, and the next right-hand side starts from them; a single-step call converts U with
    the primitive kernel instead.  Both must give the same bits, halo cells and all boundary kinds
    included."""
    c, case, grid, U, phi, inflow = setup_case(name, seed=5)
    (Ua, ta), (Ub, tb) = steps_in_one_call_vs_single_calls(c, U, phi, inflow, 3, precision)
    assert np.array_equal(Ua, Ub) and ta == tb


def test_multi_step_call_past_t_end_equals_single_step_calls():
    """Sod past t = 0.2 in one call and in single-step calls: the steps after the clipped one have
    dt = 0 and leave the state as it is, in both."""
    c, case, grid, U, _, _ = setup_case("sod1d")
    (Ua, ta), (Ub, tb) = steps_in_one_call_vs_single_calls(c, U, None, {}, 180, t_end=0.2)
    assert np.array_equal(Ua, Ub) and ta == tb and ta[0] == 0.2


def test_sod_run_to_t02():
    """Whole Sod run to t = 0.2 (175 steps, last step clipped): same number of steps, same final
    time, and per-step parity at several points of the trajectory."""
    c, case, grid, U0, _, _ = setup_case("sod1d")
    s = Solver(c)
    Ud = torch.from_numpy(U0).cuda()
    s.step(Ud, 1000, t_end=0.2)
    s.check()
    t, _ = s.time()
    assert t == 0.2
    U, tt, k = nf.advance(U0.copy(), case, grid, 1000, 0.0, 0.2)
    assert k == 175
    inner = inner_of(case)
    err = rel_err(Ud.cpu().numpy()[inner], U[inner])
    assert max(err) <= 1e-11, err           # accumulated over 175 steps
    # per-step parity at steps 50, 120, 174 of the oracle trajectory
    Uk = U0.copy()
    tk = 0.0
    checkpoints = {50, 120, 174}
    for step in range(175):
        dt = min(nf.cfl_dt(Uk, case, grid), 0.2 - tk)
        Unext = nf.rk3_step(Uk.copy(), dt, case, grid)
        if step in checkpoints:
            s2 = Solver(dict(c, dt_fixed=dt))
            Ug = torch.from_numpy(Uk).cuda()
            s2.step(Ug, 1)
            assert max(rel_err(Ug.cpu().numpy()[inner], Unext[inner])) <= TOL
        Uk, tk = Unext, tk + dt


def test_nonfinite_state_is_reported():
    c, case, grid, U, phi, inflow = setup_case("periodic3d_z_power")
    U[4, 5, 5, 5] = np.nan
    s = Solver(c)
    Ud = torch.from_numpy(U).cuda()
    s.step(Ud, 1)
    from paper_2406_19494_gb300 import native
    with pytest.raises(native.FluidError) as ei:
        s.check()
    assert ei.value.status == native.FLUID_ENONFINITE
    s.check()                                     # the flag is cleared by the check


def test_negative_ghost_temperature_is_reported():
    c = CASES["channel3d_walls_force"]()
    c["t_wall"] = ((1, 1), (0.05, 0.05), (1, 1))   # 2 T_w - T < 0 next to the walls
    case, grid, U = padded_state(c, seed=1)
    s = Solver(c)
    s.rhs(torch.from_numpy(U).cuda())
    from paper_2406_19494_gb300 import native
    with pytest.raises(native.FluidError) as ei:
        s.check()
    assert ei.value.status == native.FLUID_ENONFINITE and "ghost" in str(ei.value)


def test_null_and_aliased_pointers_rejected():
    from paper_2406_19494_gb300 import native
    import ctypes
    s = Solver(CASES["periodic3d_z_power"]())
    L = s.lib
    st = L.fluid_rhs(s.handle, None, None, None)
    assert st == native.FLUID_EINVAL
    U = s.new_state()
    p = ctypes.c_void_p(U.data_ptr())
    assert L.fluid_rhs(s.handle, p, p, None) == native.FLUID_EINVAL
    assert L.fluid_step(s.handle, p, -1, 0.0, None) == native.FLUID_EINVAL


# ---------------------------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark uses: sampled cells
# ---------------------------------------------------------------------------------------------
class _SubAxis:
    def __init__(self, ax, lo, hi):
        for k in ("xc", "dx", "mc", "mf"):
            setattr(self, k, getattr(ax, k)[lo:hi])


class _SubGrid(nf.Grid):
    def __init__(self, axes):
        self.axes = axes


def _patch_rhs(Ufilled, case, grid, cell):
    """Oracle R at one interior cell from the 7^3 neighbourhood of an already halo-filled state."""
    sub = dict(ndim=case.ndim, n=(1, 1, 1), lo=case.lo, hi=case.hi, bc=case.bc, gamma=case.gamma,
               R=case.R, Pr=case.Pr, visc=case.visc, mu_ref=case.mu_ref, T_ref=case.T_ref,
               visc_exp=case.visc_exp, suth_S=case.suth_S, weno=case.weno, weno_eps=case.weno_eps,
               body_force=case.body_force, t_wall=case.t_wall, visc_order=case.visc_order)
    sc = nf.Case(sub)
    axes = [_SubAxis(grid.axes[a], cell[a] - 3, cell[a] + 4) for a in range(3)]
    sl = (slice(None),) + tuple(slice(cell[a] - 3, cell[a] + 4) for a in (2, 1, 0))
    R = nf.rhs_filled(Ufilled[sl].copy(), sc, _SubGrid(axes))
    return R[:, 3, 3, 3]


def _sampled_rhs_check(c, W, nsamp=48, seed=0, margin=3):
    case = nf.Case(c)
    grid = nf.Grid(case)
    Wp = np.pad(W, [(0, 0)] + [(3, 3)] * 3, mode="edge")
    U = nf.prim_to_cons(Wp, case)
    s = Solver(c)
    Rg = s.rhs(torch.from_numpy(U).cuda())
    s.check()
    Rg = Rg.cpu().numpy()
    Uf = nf.fill_halos(U.copy(), case, grid)
    rng = np.random.default_rng(seed)
    cells = [tuple(int(rng.integers(3 + margin, 3 + case.n[a] - margin)) for a in range(3))
             for _ in range(nsamp)]
    cells += [(3, 3, 3), (3 + case.n[0] - 1, 3 + case.n[1] - 1, 3 + case.n[2] - 1)]
    ref = np.array([_patch_rhs(Uf, case, grid, cl) for cl in cells])
    got = np.array([Rg[:, cl[2], cl[1], cl[0]] for cl in cells])
    scale = np.max(np.abs(ref), axis=0)
    err = np.max(np.abs(got - ref), axis=0) / scale
    assert np.all(err <= TOL), err
    return Rg, case, grid


def _perturbed(W, seed, amp=0.05):
    """W with seeded relative noise on rho and p and absolute noise on the velocity."""
    r = wl.uniform01(seed, W.size).reshape(W.shape) * 2.0 - 1.0
    out = W.copy()
    out[0] *= 1.0 + amp * r[0]
    out[1:4] += amp * r[1:4]
    out[4] *= 1.0 + amp * r[4]
    return out


def _tgv_full(n=128):
    c = wl.tgv_case(n)
    case = nf.Case(c)
    grid = nf.Grid(case)
    xs = [grid.axes[a].xc[3:-3] for a in range(3)]
    return c, case, grid, wl.tgv_prims(c, *xs)


@pytest.mark.slow
def test_tgv_128_full_size_sampled_rhs():
    """R of the TGV 128^3 state with a seeded 5 % perturbation (at t = 0 the closed-form field is
    divergence free, so R_rho and R_E are cancellations of fluxes 10^3 larger than themselves and
    the max-normalised norm would measure only rounding order)."""
    c, case, grid, W = _tgv_full()
    Rg, case, grid = _sampled_rhs_check(c, _perturbed(W, seed=7))
    vol = grid.inner_volume(case)
    inner = case.interior()
    for v in range(5):
        tot = np.sum(Rg[v][inner] * vol)
        assert abs(tot) <= 1e-13 * np.sum(np.abs(Rg[v][inner]) * vol), v


def _patch_step(Uint, case, grid, cell, dt, r=9):
    """Oracle U^{n+1} at one cell of a fully periodic state from its radius-9 neighbourhood: the
    three RK3 stages run on shrinking blocks (each right-hand side consumes three cells per side).
    Block index k on axis a is the interior cell (cell[a] - r + off + k) mod n[a]."""
    n = case.n
    idx = [np.arange(cell[a] - r, cell[a] + r + 1) % n[a] for a in range(3)]
    Up = Uint[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]

    def sub_rhs(V, off):
        size = V.shape[1:][::-1]                 # (x, y, z) sizes of the block
        sub = dict(ndim=3, n=tuple(s - 6 for s in size), lo=case.lo, hi=case.hi, bc=case.bc,
                   gamma=case.gamma, R=case.R, Pr=case.Pr, visc=case.visc, mu_ref=case.mu_ref,
                   T_ref=case.T_ref, visc_exp=case.visc_exp, suth_S=case.suth_S, weno=case.weno,
                   weno_eps=case.weno_eps, body_force=case.body_force, t_wall=case.t_wall)
        axes = []
        for a in range(3):
            cells = (np.arange(size[a]) + cell[a] - r + off) % n[a] + case.h[a]
            ax = _SubAxis(grid.axes[a], 0, 1)
            for k in ("xc", "dx", "mc", "mf"):
                setattr(ax, k, getattr(grid.axes[a], k)[cells])
            axes.append(ax)
        return nf.rhs_filled(V, nf.Case(sub), _SubGrid(axes))

    c3 = (slice(None),) + (slice(3, -3),) * 3
    R1 = sub_rhs(Up, 0)
    U1 = Up[c3] + dt * R1[c3]                                    # offset 3, 13^3
    R2 = sub_rhs(U1, 3)
    U2 = 0.75 * Up[c3][c3] + 0.25 * (U1[c3] + dt * R2[c3])       # offset 6, 7^3
    R3 = sub_rhs(U2, 6)
    U3 = (1.0 / 3.0) * Up[c3][c3][c3] + (2.0 / 3.0) * (U2[c3] + dt * R3[c3])
    return U3[:, 0, 0, 0]


@pytest.mark.slow
@pytest.mark.parametrize("perturb", [False, True])
def test_tgv_128_full_size_step(perturb):
    """One RK3 step of the full-size TGV in the benchmark's launch configuration, at sampled cells
    (the oracle evaluates each from its periodic radius-9 neighbourhood)."""
    c, case, grid, W = _tgv_full()
    if perturb:
        W = _perturbed(W, seed=8)
    Wp = np.pad(W, [(0, 0)] + [(3, 3)] * 3, mode="edge")
    U = nf.prim_to_cons(Wp, case)
    dt = nf.cfl_dt(U, case, grid)
    s = Solver(dict(c, dt_fixed=dt))
    Ud = torch.from_numpy(U).cuda()
    s.step(Ud, 1)
    s.check()
    got = Ud.cpu().numpy()
    Uint = U[(slice(None),) + case.interior()]
    rng = np.random.default_rng(9)
    cells = [tuple(int(rng.integers(0, 128)) for _ in range(3)) for _ in range(24)] + [(0, 0, 0), (127, 127, 127)]
    ref = np.array([_patch_step(Uint, case, grid, cl, dt) for cl in cells])
    gv = np.array([got[:, cl[2] + 3, cl[1] + 3, cl[0] + 3] for cl in cells])
    scale = np.max(np.abs(Uint.reshape(5, -1)), axis=1)
    scale = np.where(scale > 0, scale, 1.0)          # rho w is identically zero in the TGV
    err = np.max(np.abs(gv - ref), axis=0) / scale
    assert np.all(err <= TOL), err


@pytest.mark.slow
def test_channel_full_size_sampled():
    c = wl.channel_case(192, 128, 128)
    case = nf.Case(c)
    grid = nf.Grid(case)
    xs = [grid.axes[a].xc[3:-3] for a in range(3)]
    W = wl.channel_prims(c, *xs, seed=0)
    _sampled_rhs_check(c, W, margin=0)


@pytest.mark.slow
def test_longest_axis_one_dimensional():
    """The longest axis the configuration admits (2^20 cells, 1-D Sod-type data repeated along x):
    sampled cells of one right-hand side and of one step against the oracle on 7-cell patches."""
    n = 1 << 20
    c = dict(wl.sod_case(200), n=(n, 1, 1), hi=(float(n) / 200.0, 1.0, 1.0))
    case = nf.Case(c)
    grid = nf.Grid(case)
    xc = grid.axes[0].xc
    # a Sod state every 200 cells (discontinuities all along the axis)
    W = wl.sod_prims((xc % 1.0))[:, None, None, :]
    U = nf.prim_to_cons(W, case)
    s = Solver(c)
    Rg = s.rhs(torch.from_numpy(U).cuda())
    s.check()
    Rg = Rg.cpu().numpy()
    Uf = nf.fill_halos(U.copy(), case, grid)
    rng = np.random.default_rng(1)
    cells = [int(v) for v in rng.integers(3, 3 + n, 40)] + [3, 3 + n - 1, 3 + n // 2]
    sub = dict(c, n=(1, 1, 1))
    sc = nf.Case(sub)
    ref, got = [], []
    for x in cells:
        axes = [_SubAxis(grid.axes[0], x - 3, x + 4), _SubAxis(grid.axes[1], 0, 1), _SubAxis(grid.axes[2], 0, 1)]
        R = nf.rhs_filled(Uf[:, :, :, x - 3:x + 4].copy(), sc, _SubGrid(axes))
        ref.append(R[:, 0, 0, 3])
        got.append(Rg[:, 0, 0, x])
    ref, got = np.array(ref), np.array(got)
    scale = np.max(np.abs(ref), axis=0)
    scale = np.where(scale > 0, scale, 1.0)
    assert np.all(np.max(np.abs(got - ref), axis=0) / scale <= TOL)


@pytest.mark.parametrize("name", ["channel3d_walls_force", "bl2d_porous_inflow"])
def test_wall_fluxes_parity(name):
    """fluid_wall_fluxes (wall heat flux and wall shear per wall cell) against the oracle's
    wall_fluxes at 1e-12 of their largest magnitude, on the isothermal / porous faces."""
    c = CASES[name]()
    case, grid, U = padded_state(c, seed=9)
    s = Solver(c)
    phi = None
    inflow = inflows(c, case, grid)
    for (a, sd), prof in inflow.items():
        s.set_inflow(a, sd, torch.from_numpy(np.ascontiguousarray(prof)).cuda())
    if c.get("porous"):
        phi = wl.porous_phi(c, seed=3)
        s.set_wall_params(torch.from_numpy(phi).cuda())
    Ud = torch.from_numpy(U).cuda()
    faces = [(a, sd) for a in range(case.ndim) for sd in range(2) if case.bc[a][sd] in ("wall", "porous")]
    assert faces
    for a, sd in faces:
        qw, tw = s.wall_fluxes(Ud, a, sd)
        q_ref, t_ref = nf.wall_fluxes(U.copy(), case, grid, a, sd, phi, inflow)
        q_ref = np.squeeze(q_ref)
        t_ref = np.squeeze(t_ref)
        got_q, got_t = np.squeeze(qw.cpu().numpy()), np.squeeze(tw.cpu().numpy())
        assert got_q.shape == q_ref.shape
        assert np.max(np.abs(got_q - q_ref)) <= TOL * np.max(np.abs(q_ref)), (a, sd)
        assert np.max(np.abs(got_t - t_ref)) <= TOL * np.max(np.abs(t_ref)), (a, sd)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zero_steps_change_nothing(precision):
    """fluid_step with nsteps = 0 launches nothing: the state and the solver's clock stay as they
    are, bit for bit."""
    c = CASES["ragged2d_xwall"]()
    case, grid, U = padded_state(c, seed=4)
    from paper_2406_19494_gb300.solver import Solver as S
    s = S(c, precision=precision)
    s.set_time(0.25)
    Ud = torch.from_numpy(U).cuda()
    s.step(Ud, 0)
    s.check()
    assert np.array_equal(Ud.cpu().numpy(), U)
    assert s.time()[0] == 0.25
