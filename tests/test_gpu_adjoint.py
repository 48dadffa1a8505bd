"""Hand-written discrete adjoint (FP64) against complex-step derivatives of the CPU oracle.

For random cotangents mu and directions (dU, dphi), the complex-step derivative of the oracle,
Im f(U + i h dU, phi + i h dphi) / h with h = 1e-30, is exact to rounding; the adjoint must satisfy
<mu, df> = <(df/dU)^T mu, dU> + <(df/dphi)^T mu, dphi>.  Bounds: 1e-10 relative for one right-hand
side, one RK3 step and the wall loss; 1e-6 relative for the end-to-end gradient through many steps
(the bound the gradients are required to meet).
"""
import numpy as np
import pytest

from helpers import padded_state
from oracle import ns_fv as nf
from paper_2406_19494_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 1e-30
P = ("periodic", "periodic")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_19494_gb300 import build
    build.build()


def Solver(c, **kw):
    from paper_2406_19494_gb300.solver import Solver as S
    return S(c, adjoint=True, **kw)


POROUS = dict(axis=1, side=0, begin=3, count=10, A=0.05, kappa=3.0, phi0=0.1)
CASES = {
    "periodic3d_z_power": lambda: wl.random_box(3, (10, 9, 8)),
    "channel3d_walls_force_js": lambda: wl.random_box(3, (8, 10, 6), bc=(P, ("wall", "wall"), P),
                                                        stretch=("uniform", "tanh2", "uniform"),
                                                        beta=(0.0, 2.0, 0.0), weno="js",
                                                        body_force=(0.05, 0.02, 0.0),
                                                        t_wall=((1, 1), (2.5, 2.2), (1, 1))),
    "bl2d_porous_inflow": lambda: wl.random_box(2, (16, 12, 1), bc=(("inflow", "zero_gradient"),
                                                                    ("porous", "zero_gradient"), P),
                                                  stretch=("uniform", "tanh1", "uniform"), beta=(0, 2.2, 0),
                                                  visc="sutherland", t_wall=((1, 1), (2.5, 1), (1, 1)),
                                                  porous=POROUS),
    "adiabatic_zg_3d_const": lambda: wl.random_box(3, (8, 7, 6), bc=(("zero_gradient", "zero_gradient"),
                                                                     ("adiabatic", "adiabatic"), P),
                                                     visc="constant"),
    "sod1d_js_inviscid": lambda: wl.sod_case(40),
}


def _setup(name, seed=0):
    c = CASES[name]()
    if name.startswith("sod"):
        case = nf.Case(c)
        grid = nf.Grid(case)
        W = wl.sod_prims(grid.axes[0].xc)[:, None, None, :]
        U = nf.prim_to_cons(W, case)
    else:
        case, grid, U = padded_state(c, seed=seed)
    rng = np.random.default_rng(seed + 100)
    phi = None
    inflow = {}
    if case.porous:
        phi = case.porous["phi0"] * (1.0 + 0.3 * rng.uniform(-1, 1, case.porous["count"]))
    for a in range(case.ndim):
        for s in range(2):
            if case.bc[a][s] == "inflow":
                t1 = 1 if a == 0 else 0
                t2 = 1 if a == 2 else 2
                sh = (5, case.p[t2], case.p[t1])
                prof = np.empty(sh)
                prof[0] = 1.0 + 0.1 * rng.uniform(-1, 1, sh[1:])
                prof[1] = 0.5 + 0.1 * rng.uniform(-1, 1, sh[1:])
                prof[2] = 0.05 * rng.uniform(-1, 1, sh[1:])
                prof[3] = 0.0
                prof[4] = 1.0 + 0.1 * rng.uniform(-1, 1, sh[1:])
                inflow[(a, s)] = prof
    return c, case, grid, U, phi, inflow


def _solver(c, phi, inflow, **kw):
    s = Solver(c, **kw)
    if phi is not None:
        s.set_wall_params(torch.from_numpy(phi).cuda())
    for (a, side), prof in inflow.items():
        s.set_inflow(a, side, torch.from_numpy(np.ascontiguousarray(prof)).cuda())
    return s


def _interior_random(case, rng, shape):
    X = np.zeros(shape)
    inner = (slice(None),) + case.interior()
    X[inner] = rng.uniform(-1, 1, X[inner].shape)
    return X


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_adjoint_matches_complex_step(name):
    c, case, grid, U, phi, inflow = _setup(name)
    rng = np.random.default_rng(7)
    mu = _interior_random(case, rng, U.shape)
    dU = _interior_random(case, rng, U.shape) * np.abs(U).max(axis=(1, 2, 3))[:, None, None, None] * 0.1
    dphi = rng.uniform(-1, 1, phi.shape) if phi is not None else None
    Uc = U + 1j * H * dU
    phic = phi + 1j * H * dphi if phi is not None else None
    Rc = nf.rhs(Uc.copy(), case, grid, phic, inflow)
    lhs = float(np.sum(mu * Rc.imag / H))
    s = _solver(c, phi, inflow)
    gphi = torch.zeros(len(phi), dtype=torch.float64, device="cuda") if phi is not None else None
    gU = s.adjoint_rhs(torch.from_numpy(U).cuda(), torch.from_numpy(mu).cuda(), gphi=gphi).cpu().numpy()
    inner = (slice(None),) + case.interior()
    rhs = float(np.sum(gU[inner] * dU[inner]))
    if phi is not None:
        rhs += float(np.sum(gphi.cpu().numpy() * dphi))
    scale = float(np.sum(np.abs(mu * Rc.imag / H))) + 1e-300
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs)


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_adjoint_matches_differences_of_the_gpu_forward(name):
    """The dot-product identity <mu, (dR/dU) dU> = <(dR/dU)^T mu, dU> with the left side from
    central differences of the GPU right-hand side itself (fluid_rhs), so the adjoint kernels are
    checked against the kernels they differentiate, not only against the oracle."""
    c, case, grid, U, phi, inflow = _setup(name, seed=4)
    rng = np.random.default_rng(13)
    mu = _interior_random(case, rng, U.shape)
    dU = _interior_random(case, rng, U.shape) * np.abs(U).max(axis=(1, 2, 3))[:, None, None, None] * 0.1
    s = _solver(c, phi, inflow)
    h = 1e-6
    Rp = s.rhs(torch.from_numpy(U + h * dU).cuda()).cpu().numpy()
    Rm = s.rhs(torch.from_numpy(U - h * dU).cuda()).cpu().numpy()
    inner = (slice(None),) + case.interior()
    jvp = (Rp - Rm)[inner] / (2 * h)
    lhs = float(np.sum(mu[inner] * jvp))
    gU = s.adjoint_rhs(torch.from_numpy(U).cuda(), torch.from_numpy(mu).cuda()).cpu().numpy()
    rhs = float(np.sum(gU[inner] * dU[inner]))
    scale = float(np.sum(np.abs(mu[inner] * jvp))) + 1e-300
    assert abs(lhs - rhs) <= 1e-6 * scale, (lhs, rhs)


@pytest.mark.parametrize("stored_stages", [False, True])
@pytest.mark.parametrize("name", ["bl2d_porous_inflow", "channel3d_walls_force_js"])
def test_step_adjoint_matches_complex_step(name, stored_stages):
    c, case, grid, U, phi, inflow = _setup(name, seed=2)
    dt = 0.5 * nf.cfl_dt(U, case, grid)
    c = dict(c, dt_fixed=dt)
    case = nf.Case(c)
    rng = np.random.default_rng(11)
    lam = _interior_random(case, rng, U.shape)
    dU = _interior_random(case, rng, U.shape) * np.abs(U).max(axis=(1, 2, 3))[:, None, None, None] * 0.1
    dphi = rng.uniform(-1, 1, phi.shape) if phi is not None else None
    U3c = nf.rk3_step(U + 1j * H * dU, dt, case, grid, phi + 1j * H * dphi if phi is not None else None, inflow)
    inner = (slice(None),) + case.interior()
    lhs = float(np.sum(lam[inner] * U3c[inner].imag / H))
    s = _solver(c, phi, inflow)
    gphi = torch.zeros(len(phi), dtype=torch.float64, device="cuda") if phi is not None else None
    Ud = torch.from_numpy(U).cuda()
    lam_d = torch.from_numpy(lam).cuda()
    if stored_stages:
        U1, U2 = torch.zeros_like(Ud), torch.zeros_like(Ud)
        s.step_stages(Ud.clone(), U1, U2)
        s.adjoint_step(Ud, lam_d, gphi, U1, U2)
    else:
        s.adjoint_step(Ud, lam_d, gphi)
    got = lam_d.cpu().numpy()
    rhs = float(np.sum(got[inner] * dU[inner]))
    if phi is not None:
        rhs += float(np.sum(gphi.cpu().numpy() * dphi))
    scale = float(np.sum(np.abs(lam[inner] * U3c[inner].imag / H)))
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs)


def test_wall_heat_loss_value_and_gradient():
    c = wl.porous_bl_case(48, 24)
    case = nf.Case(c)
    grid = nf.Grid(case)
    xc, yc = grid.axes[0].xc[3:-3], grid.axes[1].xc[3:-3]
    W = wl.porous_bl_prims(c, xc, yc)
    U = nf.prim_to_cons(np.pad(W, [(0, 0), (0, 0), (3, 3), (3, 3)], mode="edge"), case)
    phi = wl.porous_phi(c, seed=0)
    prof = wl.porous_bl_inflow(c, grid.axes[1].xc)
    J_ref = nf.wall_heat_loss(U, case, grid, 1, 0, phi, {(0, 0): prof})
    s = _solver(c, phi, {(0, 0): prof})
    J, dJ = s.wall_heat_loss(torch.from_numpy(U).cuda(), 1, 0, grad=True)
    assert abs(J.item() - J_ref) <= 1e-12 * abs(J_ref)
    rng = np.random.default_rng(3)
    dU = _interior_random(case, rng, U.shape) * np.abs(U).max(axis=(1, 2, 3))[:, None, None, None] * 0.1
    Jc = nf.wall_heat_loss(U + 1j * H * dU, case, grid, 1, 0, phi, {(0, 0): prof})
    lhs = Jc.imag / H
    inner = (slice(None),) + case.interior()
    rhs = float(np.sum(dJ.cpu().numpy()[inner] * dU[inner]))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs), (lhs, rhs)


def _bl_small(nx=32, ny=16, count=16):
    c = wl.porous_bl_case(nx, ny, porous_count=count)
    case = nf.Case(c)
    grid = nf.Grid(case)
    xc, yc = grid.axes[0].xc[3:-3], grid.axes[1].xc[3:-3]
    W = wl.porous_bl_prims(c, xc, yc)
    U = nf.prim_to_cons(np.pad(W, [(0, 0), (0, 0), (3, 3), (3, 3)], mode="edge"), case)
    dt = 0.5 * nf.cfl_dt(U, case, grid)
    c = dict(c, dt_fixed=dt)
    return c, nf.Case(c), grid, U, wl.porous_bl_inflow(c, grid.axes[1].xc)


def test_end_to_end_gradient_against_complex_step_and_differences():
    """J = wall heat flux after 12 steps of a 32 x 16 porous boundary layer, checkpoints every 5
    steps (segments of 5, 5, 2): dJ/dphi from the autograd function against the complex-step
    derivative of the oracle's trajectory (3 components and one random direction, <= 1e-6) and
    against central differences of the GPU forward (all components)."""
    from paper_2406_19494_gb300.adjoint import wall_heat_loss
    c, case, grid, U0, prof = _bl_small()
    nsteps, K = 12, 5
    phi0 = wl.porous_phi(c, seed=1)
    s = _solver(c, None, {(0, 0): prof})
    phi = torch.from_numpy(phi0).cuda().requires_grad_(True)
    J = wall_heat_loss(phi, s, torch.from_numpy(U0).cuda(), nsteps, K, 1, 0)
    J.backward()
    g = phi.grad.cpu().numpy()

    def oracle_J(ph):
        U = U0.astype(np.result_type(ph, np.float64)).copy()
        for _ in range(nsteps):
            U = nf.rk3_step(U, c["dt_fixed"], case, grid, ph, {(0, 0): prof})
        return nf.wall_heat_loss(U, case, grid, 1, 0, ph, {(0, 0): prof})

    J_ref = oracle_J(phi0)
    assert abs(J.item() - J_ref) <= 1e-11 * abs(J_ref)
    gnorm = np.max(np.abs(g))
    rng = np.random.default_rng(5)
    dirs = [np.eye(len(phi0))[i] for i in (0, len(phi0) // 2, len(phi0) - 1)] + [rng.uniform(-1, 1, len(phi0))]
    for d in dirs:
        cs = oracle_J(phi0 + 1j * H * d).imag / H
        assert abs(cs - float(np.dot(g, d))) <= 1e-6 * gnorm * np.sum(np.abs(d)), (cs, np.dot(g, d))
    # central differences of the GPU forward, every component
    h = 1e-5 * np.max(np.abs(phi0))
    fd = np.zeros_like(phi0)
    for i in range(len(phi0)):
        vals = []
        for sgn in (1.0, -1.0):
            ph = phi0.copy()
            ph[i] += sgn * h
            vals.append(wall_heat_loss(torch.from_numpy(ph).cuda(), s, torch.from_numpy(U0).cuda(), nsteps, K, 1, 0).item())
        fd[i] = (vals[0] - vals[1]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-5 * gnorm, np.max(np.abs(fd - g)) / gnorm


def test_long_trajectory_gradient_stays_bounded():
    """150 steps of a 64 x 32 porous boundary layer (a nearly uniform Ma 6 free stream above the
    layer): the adjoint directional derivative matches central differences of the GPU forward.
    Guards the translation-invariant form of the WENO5 cotangents, without which rounding in the
    free stream is amplified by the weight derivatives until the adjoint overflows."""
    from paper_2406_19494_gb300.adjoint import wall_heat_loss
    c, case, grid, U0, prof = _bl_small(64, 32, 32)
    s = _solver(c, None, {(0, 0): prof})
    phi0 = torch.from_numpy(wl.porous_phi(c, seed=2)).cuda()
    d = torch.from_numpy(np.random.default_rng(4).uniform(-1, 1, phi0.numel())).cuda()
    p = phi0.clone().requires_grad_(True)
    J = wall_heat_loss(p, s, torch.from_numpy(U0).cuda(), 150, 20, 1, 0)
    J.backward()
    adj = float((p.grad * d).sum())
    h = 1e-6 * 0.1
    Jp = wall_heat_loss(phi0 + h * d, s, torch.from_numpy(U0).cuda(), 150, 20, 1, 0).item()
    Jm = wall_heat_loss(phi0 - h * d, s, torch.from_numpy(U0).cuda(), 150, 20, 1, 0).item()
    fd = (Jp - Jm) / (2 * h)
    assert abs(adj - fd) <= 1e-5 * abs(fd), (adj, fd)


@pytest.mark.slow
def test_w4_gradient_against_complex_step_relative():
    """The porous boundary-layer workload's gradient as the benchmark computes it: 512 x 128 cells,
    256 porous wall cells, 400 steps with checkpoints every 20 (the oracle's complex-step run takes
    about four minutes on one host core): the directional derivative of the autograd gradient along
    a seeded random direction equals the complex-step derivative of the oracle's trajectory within
    1e-6 of itself (relative, not scaled by the direction's size), and J equals the oracle's within
    1e-10."""
    from paper_2406_19494_gb300.adjoint import wall_heat_loss
    c, case, grid, U0, prof = _bl_small(512, 128, 256)
    nsteps, K = 400, 20
    phi0 = wl.porous_phi(c, seed=0)
    s = _solver(c, None, {(0, 0): prof})
    phi = torch.from_numpy(phi0).cuda().requires_grad_(True)
    J = wall_heat_loss(phi, s, torch.from_numpy(U0).cuda(), nsteps, K, 1, 0)
    J.backward()
    g = phi.grad.cpu().numpy()
    d = np.random.default_rng(7).uniform(-1.0, 1.0, len(phi0))
    ph = phi0 + 1j * H * d
    U = U0.astype(np.complex128)
    for _ in range(nsteps):
        U = nf.rk3_step(U, c["dt_fixed"], case, grid, ph, {(0, 0): prof})
    Jc = nf.wall_heat_loss(U, case, grid, 1, 0, ph, {(0, 0): prof})
    cs = Jc.imag / H
    adj = float(np.dot(g, d))
    assert abs(J.item() - Jc.real) <= 1e-10 * abs(Jc.real), (J.item(), Jc.real)
    assert abs(adj - cs) <= 1e-6 * abs(cs), (adj, cs, abs(adj - cs) / abs(cs))
