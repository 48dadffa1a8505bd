"""Pins of the CPU oracle against what the mathematics and the literature fix (no GPU).

Each test pins a part of the oracle to something other than itself: printed textbook values, closed
forms, invariants, conservation, convergence orders and special cases.  The inputs are seeded.
"""
import math

import numpy as np
import pytest

from conftest import read_golden
from helpers import padded_state, rel_err
from oracle import exact_riemann as er
from oracle import ns_fv as nf
from paper_2406_19494_gb300 import workloads as wl

SOD_L, SOD_R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)


# ---------------------------------------------------------------------------------------------
# exact Riemann solver (pins the Sod reference itself)
# ---------------------------------------------------------------------------------------------
def test_exact_riemann_matches_toro_table():
    vals = {k: float(v) for k, v in read_golden("toro_sod_star.txt")}
    p, u = er.star_state(SOD_L, SOD_R)
    assert abs(p - vals["p_star"]) < 5e-6
    assert abs(u - vals["u_star"]) < 5e-6


def test_exact_riemann_jump_conditions():
    """Rankine-Hugoniot across the right shock, isentrope and Riemann invariant across the left
    rarefaction, continuity of p and u across the contact."""
    g = 1.4
    p, u = er.star_state(SOD_L, SOD_R)
    S = er.shock_speed(SOD_L, SOD_R)
    # behind the shock (just left of it) and ahead of it
    rb, ub, pb = er.sample(SOD_L, SOD_R, S - 1e-9)
    ra, ua, pa = er.sample(SOD_L, SOD_R, S + 1e-9)
    assert (ra, ua, pa) == SOD_R
    mass = lambda r, v: r * (v - S)
    mom = lambda r, v, q: r * v * (v - S) + q
    ener = lambda r, v, q: (q / (g - 1) + 0.5 * r * v * v) * (v - S) + q * v
    assert abs(mass(rb, ub) - mass(ra, ua)) < 1e-12
    assert abs(mom(rb, ub, pb) - mom(ra, ua, pa)) < 1e-12
    assert abs(ener(rb, ub, pb) - ener(ra, ua, pa)) < 1e-12
    # left rarefaction: p / rho^gamma and u + 2c/(gamma-1) constant
    for s in np.linspace(-1.1, -0.1, 7):
        r, v, q = er.sample(SOD_L, SOD_R, s)
        assert abs(q / r ** g - 1.0) < 1e-12
        assert abs(v + 2 * math.sqrt(g * q / r) / (g - 1) - 2 * math.sqrt(g) / (g - 1)) < 1e-12
    # contact: p and u continuous, rho jumps
    rl, vl, ql = er.sample(SOD_L, SOD_R, u - 1e-9)
    rr, vr, qr = er.sample(SOD_L, SOD_R, u + 1e-9)
    assert abs(ql - qr) < 1e-14 and abs(vl - vr) < 1e-14 and abs(rl - rr) > 0.1


# ---------------------------------------------------------------------------------------------
# Sod shock tube: WENO5-JS + HLLC + TVD-RK3, CFL 0.5, to t = 0.2
# ---------------------------------------------------------------------------------------------
def _sod_l1(n):
    c = wl.sod_case(n)
    case = nf.Case(c)
    grid = nf.Grid(case)
    xc = grid.axes[0].xc
    W = wl.sod_prims(xc)[:, None, None, :]
    U = nf.prim_to_cons(W, case)
    U, t, k = nf.advance(U, case, grid, 100000, 0.0, 0.2)
    assert t == 0.2
    rho = U[0, 0, 0, 3:-3]
    xf = np.linspace(0.0, 1.0, n + 1)
    ex = er.cell_averages(SOD_L, SOD_R, 0.5, 0.2, xf, nsub=16)
    return float(np.mean(np.abs(rho - ex[0]))), k


def test_sod_against_exact_solution():
    e200, k200 = _sod_l1(200)
    e400, _ = _sod_l1(400)
    assert e200 < 5e-3
    assert e400 < 0.75 * e200
    # first dt is CFL dx / max(|u| + c) = 0.5 * 0.005 / sqrt(1.4) on the initial state
    case = nf.Case(wl.sod_case(200))
    grid = nf.Grid(case)
    U = nf.prim_to_cons(wl.sod_prims(grid.axes[0].xc)[:, None, None, :], case)
    assert abs(nf.cfl_dt(U, case, grid) - 0.5 * 0.005 / math.sqrt(1.4)) < 1e-17


# ---------------------------------------------------------------------------------------------
# WENO5
# ---------------------------------------------------------------------------------------------
def _quadratic_through_averages(q, cells):
    """Quadratic P (numpy poly1d) whose averages over unit cells [c-1/2, c+1/2] are q."""
    # average of x^m over [c-1/2, c+1/2] = ((c+1/2)^{m+1} - (c-1/2)^{m+1}) / (m+1)
    A = np.array([[((c + 0.5) ** (m + 1) - (c - 0.5) ** (m + 1)) / (m + 1) for m in range(3)]
                  for c in cells])
    coef = np.linalg.solve(A, np.asarray(q, dtype=np.float64))
    return np.poly1d(coef[::-1])


def test_weno_candidates_and_smoothness_match_their_definitions():
    """p_k is the value at x = 1/2 of the quadratic matching the three cell averages of stencil k,
    and beta_k = sum_{l=1,2} int_{-1/2}^{1/2} (P_k^(l))^2 dx (Jiang & Shu's definition, dx = 1)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.normal(size=5)
        stencils = [(-2, -1, 0), (-1, 0, 1), (0, 1, 2)]
        ps, bs = [], []
        for k, st in enumerate(stencils):
            P = _quadratic_through_averages(q[[c + 2 for c in st]], st)
            ps.append(P(0.5))
            b = 0.0
            for l in (1, 2):
                D = P.deriv(l)
                I = np.polyint(D * D)
                b += I(0.5) - I(-0.5)
            bs.append(b)
        # linear weights: must reproduce sum d_k p_k; with beta_k known, JS / Z follow the formulas
        lin = nf.weno5(*q, scheme="linear", eps=0.0)
        assert abs(lin - (0.1 * ps[0] + 0.6 * ps[1] + 0.3 * ps[2])) < 1e-13
        aJ = [d / (1e-6 + b) ** 2 for d, b in zip(nf.WENO_D, bs)]
        js = nf.weno5(*q, scheme="js", eps=1e-6)
        assert abs(js - sum(a * p for a, p in zip(aJ, ps)) / sum(aJ)) < 1e-12
        tau = abs(bs[0] - bs[2])
        aZ = [d * (1 + (tau / (b + 1e-40)) ** 2) for d, b in zip(nf.WENO_D, bs)]
        z = nf.weno5(*q, scheme="z", eps=1e-40)
        assert abs(z - sum(a * p for a, p in zip(aZ, ps)) / sum(aZ)) < 1e-12


def test_weno_linear_weights_exact_for_quartics():
    """With the optimal weights the five-cell reconstruction is exact for cell averages of any
    polynomial of degree <= 4."""
    rng = np.random.default_rng(4)
    for deg in range(5):
        c = rng.normal(size=deg + 1)
        P = np.poly1d(c)
        I = np.polyint(P)
        h = 0.37
        avg = [(I((j + 0.5) * h) - I((j - 0.5) * h)) / h for j in range(-2, 3)]
        assert abs(nf.weno5(*avg, scheme="linear", eps=0.0) - P(0.5 * h)) < 1e-12


def test_weno_worked_examples():
    for name, scheme, *rest in read_golden("weno_worked_examples.txt"):
        q = [float(v) for v in rest[:5]]
        expected, tol = float(rest[5]), float(rest[6])
        got = nf.weno5(*[np.float64(v) for v in q], scheme=scheme, eps=1e-6 if scheme == "js" else 1e-40)
        assert abs(got - expected) <= tol * abs(expected), (name, got, expected)


def test_weno_is_essentially_non_oscillatory_across_a_jump():
    # JS's eps = 1e-6 is not scale-free, so its bound is looser than Z's
    for scheme, eps, bound in (("js", 1e-6, 1e-6), ("z", 1e-40, 1e-12)):
        for h in (0.1, 1.0, 10.0):
            v = nf.weno5(0.0, 0.0, 0.0, h, h, scheme=scheme, eps=eps)
            assert abs(v) < bound * h


# ---------------------------------------------------------------------------------------------
# HLLC
# ---------------------------------------------------------------------------------------------
def _W(r, u, v, w, p):
    return [np.array([x], dtype=np.float64) for x in (r, u, v, w, p)]


def test_hllc_consistency_all_axes():
    rng = np.random.default_rng(5)
    for _ in range(20):
        r, p = rng.uniform(0.2, 3.0, size=2)
        vel = rng.uniform(-3, 3, size=3)
        W = _W(r, *vel, p)
        for d in range(3):
            F = nf.hllc_flux(W, W, d, 1.4)
            Fe, _ = nf.euler_flux(W, d, 1.4)
            for c in range(5):
                assert abs(F[c][0] - Fe[c][0]) <= 1e-13 * (1 + abs(Fe[c][0]))


def test_hllc_resolves_contact_exactly():
    # stationary contact: mass and energy fluxes vanish, momentum flux is the pressure
    F = nf.hllc_flux(_W(1.0, 0, 0.3, -0.2, 0.7), _W(0.2, 0, -0.1, 0.5, 0.7), 0, 1.4)
    assert abs(F[0][0]) < 1e-15 and abs(F[4][0]) < 1e-15 and abs(F[1][0] - 0.7) < 1e-15
    # moving contact (u > 0): the upwind (left) Euler flux
    WL, WR = _W(1.0, 0.4, 0.3, 0.0, 0.7), _W(0.2, 0.4, -0.1, 0.5, 0.7)
    F = nf.hllc_flux(WL, WR, 0, 1.4)
    Fe, _ = nf.euler_flux(WL, 0, 1.4)
    for c in range(5):
        assert abs(F[c][0] - Fe[c][0]) < 1e-14


def test_hllc_supersonic_upwinding_and_mirror():
    WL, WR = _W(1.0, 3.0, 0.1, 0.2, 0.5), _W(0.5, 2.5, 0.0, 0.1, 0.4)
    F = nf.hllc_flux(WL, WR, 0, 1.4)
    Fe, _ = nf.euler_flux(WL, 0, 1.4)
    assert all(F[c][0] == Fe[c][0] for c in range(5))
    rng = np.random.default_rng(6)
    for _ in range(20):
        a = rng.uniform([0.2, -2, -1, -1, 0.2], [3, 2, 1, 1, 3])
        b = rng.uniform([0.2, -2, -1, -1, 0.2], [3, 2, 1, 1, 3])
        F = nf.hllc_flux(_W(*a), _W(*b), 0, 1.4)
        ma, mb = a.copy(), b.copy()
        ma[1] = -ma[1]
        mb[1] = -mb[1]
        G = nf.hllc_flux(_W(*mb), _W(*ma), 0, 1.4)
        sgn = (-1, 1, -1, -1, -1)
        for c in range(5):
            assert abs(G[c][0] - sgn[c] * F[c][0]) < 1e-13 * (1 + abs(F[c][0]))


def test_roe_average_has_the_roe_property():
    """The Roe-averaged Jacobian maps the jump of U onto the jump of F exactly (Roe 1981):
    A(u~, H~) (U_R - U_L) = F_R - F_L for the 1-D Euler system; and c~^2 = (g-1)(H~ - u~^2/2)."""
    g = 1.4
    rng = np.random.default_rng(7)
    for _ in range(20):
        a = rng.uniform([0.2, -2, 0, 0, 0.2], [3, 2, 0, 0, 3])
        b = rng.uniform([0.2, -2, 0, 0, 0.2], [3, 2, 0, 0, 3])
        WL, WR = _W(*a), _W(*b)
        vt, Ht, ct = nf.roe_average(WL, WR, 0, g)
        u, H = vt[0][0], Ht[0]
        A = np.array([[0.0, 1.0, 0.0],
                      [0.5 * (g - 3) * u * u, (3 - g) * u, g - 1],
                      [u * (0.5 * (g - 1) * u * u - H), H - (g - 1) * u * u, g * u]])
        U = lambda W: np.array([W[0][0], W[0][0] * W[1][0], W[4][0] / (g - 1) + 0.5 * W[0][0] * W[1][0] ** 2])
        FL, _ = nf.euler_flux(WL, 0, g)
        FR, _ = nf.euler_flux(WR, 0, g)
        dF = np.array([FR[0][0] - FL[0][0], FR[1][0] - FL[1][0], FR[4][0] - FL[4][0]])
        assert np.max(np.abs(A @ (U(WR) - U(WL)) - dF)) < 1e-12 * (1 + np.max(np.abs(dF)))
        assert abs(ct[0] ** 2 - (g - 1) * (H - 0.5 * u * u)) < 1e-13


def test_hllc_star_states_are_consistent():
    """Integral form of the Riemann fan (Toro Ch. 10): with speeds S_L < S* < S_R,
    (S* - S_L) U*_L + (S_R - S*) U*_R = S_R U_R - S_L U_L - (F_R - F_L), and the wave speeds
    bound the signal speeds of both states: S_L <= u_L - c_L, S_R >= u_R + c_R."""
    g = 1.4
    rng = np.random.default_rng(8)
    for d in range(3):
        for _ in range(20):
            a = rng.uniform([0.2, -2, -1, -1, 0.2], [3, 2, 1, 1, 3])
            b = rng.uniform([0.2, -2, -1, -1, 0.2], [3, 2, 1, 1, 3])
            h = nf.hllc_parts(_W(*a), _W(*b), d, g)
            SL, SR, Ss = h["SL"][0], h["SR"][0], h["Ss"][0]
            assert SL < Ss < SR
            assert SL <= a[1 + d] - math.sqrt(g * a[4] / a[0]) + 1e-15
            assert SR >= b[1 + d] + math.sqrt(g * b[4] / b[0]) - 1e-15
            for c in range(5):
                lhs = (Ss - SL) * h["UsL"][c][0] + (SR - Ss) * h["UsR"][c][0]
                rhs = SR * h["UR"][c][0] - SL * h["UL"][c][0] - (h["FR"][c][0] - h["FL"][c][0])
                assert abs(lhs - rhs) < 1e-12 * (1 + abs(rhs))


# ---------------------------------------------------------------------------------------------
# dissipative fluxes
# ---------------------------------------------------------------------------------------------
def _visc_case(n=(12, 12, 12), visc="constant"):
    P = ("periodic", "periodic")
    return wl.random_box(3, n, bc=(P, P, P), visc=visc, mu_ref=0.3, lo=(0.0, 0.0, 0.0),
                         hi=(1.0, 1.0, 1.0))


def _field_state(case_dict, fn):
    case = nf.Case(case_dict)
    grid = nf.Grid(case)
    z, y, x = np.meshgrid(grid.axes[2].xc, grid.axes[1].xc, grid.axes[0].xc, indexing="ij")
    W = np.stack(fn(x, y, z))
    return case, grid, W


def _tangential_interior(case, d):
    """Index of the faces along d restricted to interior cells along the other axes."""
    s = list(case.interior())
    s[2 - d] = slice(None)
    return tuple(s)


def test_viscous_flux_linear_fields():
    """Linear velocity and temperature fields: the fourth-order stencils are exact.  Rigid rotation
    has no stress; a shear u = s y gives tau_xy = mu s on y faces; T = 1 + t x gives
    q_x = -lambda t on x faces; the stress is trace-free (Stokes hypothesis)."""
    c = _visc_case()
    one = lambda x: np.ones_like(x)
    vf = lambda W, T, case, grid, d: [f[_tangential_interior(case, d)]
                                      for f in nf.viscous_face_flux(W, T, case, grid, d)]
    case, grid, W = _field_state(c, lambda x, y, z: (one(x), -0.7 * y, 0.7 * x, 0 * x, one(x)))
    T = W[4] / (W[0] * case.R)
    for d in range(3):
        F = vf(W, T, case, grid, d)
        for comp in F[1:4]:
            assert np.max(np.abs(comp)) < 1e-13
    s, t, mu = 0.9, 0.3, 0.3
    case, grid, W = _field_state(c, lambda x, y, z: (one(x), s * y, 0 * x, 0 * x, 1 + t * x))
    T = W[4] / (W[0] * case.R)
    Fy = vf(W, T, case, grid, 1)
    assert np.max(np.abs(Fy[1] - mu * s)) < 1e-13
    Fx = vf(W, T, case, grid, 0)
    lam = mu * case.cp / case.Pr
    # energy flux on x faces: u tau_xx + v tau_xy + w tau_xz + lambda dT/dx with v = w = 0 and
    # tau_xx = 0 (u depends on y only), so energy = lambda t
    assert np.max(np.abs(Fx[4] - lam * t)) < 1e-12
    # compressive field u = a x: tau_xx = mu (2a - 2a/3), tau_yy = tau_zz = -mu 2a/3
    a = 0.4
    case, grid, W = _field_state(c, lambda x, y, z: (one(x), a * x, 0 * x, 0 * x, one(x)))
    T = W[4] / (W[0] * case.R)
    txx = vf(W, T, case, grid, 0)[1]
    tyy = vf(W, T, case, grid, 1)[2]
    tzz = vf(W, T, case, grid, 2)[3]
    assert np.max(np.abs(txx - mu * 4 * a / 3)) < 1e-12
    assert np.max(np.abs(tyy + mu * 2 * a / 3)) < 1e-12
    assert np.max(np.abs(tzz + mu * 2 * a / 3)) < 1e-12


def _visc_error(n):
    """Max error of the x-face dissipative flux on a smooth periodic field (point values)."""
    c = wl.random_box(3, (n, n, n), visc="power", mu_ref=0.1, lo=(0.0, 0.0, 0.0),
                      hi=(2 * math.pi,) * 3)
    k = 1.0
    f = lambda x, y, z: (1 + 0.2 * np.sin(x + y), np.sin(k * x) * np.cos(y), np.cos(x) * np.sin(z),
                         0.5 * np.sin(y + z), 1.0 + 0.1 * np.cos(x - z))
    case, grid, W = _field_state(c, f)
    T = W[4] / (W[0] * case.R)
    F = nf.viscous_face_flux(W, T, case, grid, 0)
    h = case.h
    xf = grid.axes[0].xc[h[0] - 1:h[0] + n] + 0.5 * grid.axes[0].dx[0]
    z, y, x = np.meshgrid(grid.axes[2].xc, grid.axes[1].xc, xf, indexing="ij")
    rho = 1 + 0.2 * np.sin(x + y)
    p = 1.0 + 0.1 * np.cos(x - z)
    Te = p / rho
    u, v, w = np.sin(x) * np.cos(y), np.cos(x) * np.sin(z), 0.5 * np.sin(y + z)
    ux, uy, uz = np.cos(x) * np.cos(y), -np.sin(x) * np.sin(y), 0 * x
    vx, vy = -np.sin(x) * np.sin(z), 0 * x
    wx, wz = 0 * x, 0.5 * np.cos(y + z)
    rx = 0.2 * np.cos(x + y)
    px = -0.1 * np.sin(x - z)
    Tx = (px * rho - p * rx) / rho ** 2
    mu = 0.1 * Te ** 0.7
    div = ux + vy + wz
    txx = mu * (2 * ux - 2.0 / 3.0 * div)
    txy = mu * (uy + vx)
    txz = mu * (uz + wx)
    en = u * txx + v * txy + w * txz + mu * case.cp / case.Pr * Tx
    inner = (slice(h[2], h[2] + n), slice(h[1], h[1] + n), slice(None))
    err = 0.0
    for got, ex in zip(F[1:], (txx, txy, txz, en)):
        err = max(err, np.max(np.abs(got[inner] - ex[inner])))
    return err


def test_viscous_flux_fourth_order():
    e = [_visc_error(n) for n in (16, 32)]
    order = math.log2(e[0] / e[1])
    assert order > 3.7, (e, order)


# ---------------------------------------------------------------------------------------------
# convergence of the convective operator (smooth density wave, periodic)
# ---------------------------------------------------------------------------------------------
def _wave_error(n, ndim, weno):
    """L1 error of R_rho for rho = 1 + 0.2 sin(2 pi (x + y + z)), u = v = w = 1, p = 1, against the
    exact cell average of -div(rho u)."""
    P = ("periodic", "periodic")
    n3 = tuple(n if a < ndim else 1 for a in range(3))
    c = wl.random_box(ndim, n3, bc=(P, P, P), visc="none", weno=weno, lo=(0.0, 0.0, 0.0),
                      hi=(1.0, 1.0, 1.0))
    case = nf.Case(c)
    grid = nf.Grid(case)
    h = 1.0 / n
    k = 2 * math.pi
    sinc = math.sin(k * h / 2) / (k * h / 2)
    ax = [grid.axes[a].xc if a < ndim else np.zeros(1) for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    s = x + y + z
    rho = 1 + 0.2 * np.sin(k * s) * sinc ** ndim
    one = np.ones_like(rho)
    W = np.stack([rho, one if ndim >= 1 else 0 * one, one if ndim >= 2 else 0 * one,
                  one if ndim >= 3 else 0 * one, one])
    U = nf.prim_to_cons(W, case)
    R = nf.rhs(U, case, grid)
    inner = case.interior()
    exact = np.zeros_like(rho)
    for d in range(ndim):
        # face averages of rho over the tangential directions at x_d +- h/2
        fp = 0.2 * np.sin(k * (s + h / 2)) * sinc ** (ndim - 1)
        fm = 0.2 * np.sin(k * (s - h / 2)) * sinc ** (ndim - 1)
        exact -= (fp - fm) / h
    return float(np.mean(np.abs(R[0][inner] - exact[inner])))


@pytest.mark.parametrize("ndim,ns", [(1, (32, 64, 128)), (3, (12, 24))])
def test_weno_z_fifth_order_convergence(ndim, ns):
    e = [_wave_error(n, ndim, "z") for n in ns]
    orders = [math.log2(e[i] / e[i + 1]) * (1.0 if ns[i + 1] == 2 * ns[i] else 1.0) for i in range(len(e) - 1)]
    assert orders[-1] > 4.6, (e, orders)


def test_weno_js_converges():
    e = [_wave_error(n, 1, "js") for n in (32, 64, 128)]
    assert math.log2(e[1] / e[2]) > 4.5, e


# ---------------------------------------------------------------------------------------------
# conservation, free-stream preservation, symmetry
# ---------------------------------------------------------------------------------------------
def test_periodic_conservation():
    P = ("periodic", "periodic")
    c = wl.random_box(3, (12, 10, 8), bc=(P, P, P), stretch=("uniform", "tanh2", "uniform"))
    case, grid, U = padded_state(c, seed=1)
    R = nf.rhs(U.copy(), case, grid)
    inner = case.interior()
    vol = grid.inner_volume(case)
    for v in range(5):
        tot = np.sum(R[v][inner] * vol)
        scale = np.sum(np.abs(R[v][inner]) * vol)
        assert abs(tot) < 1e-14 * scale, (v, tot, scale)


def test_freestream_preserved_on_stretched_grids():
    P = ("periodic", "periodic")
    c = wl.random_box(3, (10, 12, 8), bc=(P, P, P), stretch=("tanh1", "tanh2", "uniform"),
                      beta=(1.3, 2.0, 0.0))
    case, grid, U = padded_state(c, uniform=(1.2, 0.3, -0.2, 0.1, 0.9))
    assert np.all(nf.rhs(U.copy(), case, grid) == 0.0)
    # fluid at rest at the wall temperature between isothermal walls
    c = wl.random_box(3, (10, 12, 8), bc=(P, ("wall", "wall"), P), stretch=("uniform", "tanh2", "uniform"),
                      t_wall=((1.0, 1.0), (1.0, 1.0), (1.0, 1.0)))
    case, grid, U = padded_state(c, uniform=(1.3, 0.0, 0.0, 0.0, 1.3))
    assert np.all(nf.rhs(U.copy(), case, grid) == 0.0)


def test_mirror_symmetry_in_x():
    """Reflecting x (and u) reflects R with the x-momentum component negated."""
    W0 = ("wall", "wall")
    c = wl.random_box(3, (12, 10, 8), bc=(W0, ("periodic", "periodic"), ("periodic", "periodic")),
                      t_wall=((1.1, 1.1), (1, 1), (1, 1)))
    case, grid, U = padded_state(c, seed=2)
    Um = U[:, :, :, ::-1].copy()
    Um[1] = -Um[1]
    R = nf.rhs(U.copy(), case, grid)
    Rm = nf.rhs(Um, case, grid)[:, :, :, ::-1]
    Rm[1] = -Rm[1]
    inner = (slice(None),) + case.interior()
    assert max(rel_err(Rm[inner], R[inner])) < 1e-13


def test_axis_permutation():
    """Relabelling the axes (x, y, z) -> (y, z, x) permutes R accordingly."""
    P = ("periodic", "periodic")
    c = wl.random_box(3, (10, 9, 8), bc=(P, ("wall", "wall"), P), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.2, 0.9),
                      t_wall=((1.0, 1.0), (1.1, 0.9), (1.0, 1.0)))
    case, grid, U = padded_state(c, seed=4)
    R = nf.rhs(U.copy(), case, grid)
    # new axes: x' = y, y' = z, z' = x
    c2 = dict(c)
    perm = (1, 2, 0)
    for key in ("n", "lo", "hi", "bc", "t_wall", "stretch", "beta"):
        c2[key] = tuple(c[key][perm[a]] for a in range(3))
    case2 = nf.Case(c2)
    grid2 = nf.Grid(case2)
    # array axes (z, y, x) -> (z', y', x') = (x, z, y)
    U2 = np.transpose(U, (0, 3, 1, 2))[[0, 2, 3, 1, 4]].copy()
    R2 = nf.rhs(U2, case2, grid2)
    Rb = np.transpose(R2[[0, 3, 1, 2, 4]], (0, 2, 3, 1))
    inner = (slice(None),) + case.interior()
    assert max(rel_err(Rb[inner], R[inner])) < 1e-14


# ---------------------------------------------------------------------------------------------
# boundary conditions
# ---------------------------------------------------------------------------------------------
def test_walls_impose_their_face_values():
    """At an isothermal no-slip wall the face-interpolated velocity is zero and T = T_w; at the
    porous wall with phi = phi0 the wall-normal velocity is the paper's A sin(2 pi kappa x)."""
    par = {k: float(v) for k, v in read_golden("paper_parameters.txt")}
    c = wl.porous_bl_case(nx=64, ny=24)
    assert c["porous"]["A"] == par["disturbance_A"] and c["porous"]["kappa"] == par["disturbance_kappa"]
    case0 = nf.Case(c)
    grid0 = nf.Grid(case0)
    xc0, yc0, _ = [grid0.axes[a].xc[case0.h[a]:case0.h[a] + case0.n[a]] for a in range(3)]
    case, grid, U = padded_state(c, prims=wl.porous_bl_prims(c, xc0, yc0))
    cnt = c["porous"]["count"]
    phi = np.full(cnt, c["porous"]["phi0"])
    inflow = {(0, 0): wl.porous_bl_inflow(c, grid.axes[1].xc)}
    nf.fill_halos(U, case, grid, phi, inflow)
    W, T = nf.cons_to_prim(U, case)
    h = 3
    f = lambda q, o: q[0, h - 1 + o, :]
    interp = lambda q: (9.0 * (f(q, 0) + f(q, 1)) - (f(q, -1) + f(q, 2))) / 16.0
    ix = slice(h, h + case.n[0])
    xc = grid.axes[0].xc[ix]
    b = c["porous"]["begin"]
    expect_v = np.zeros(case.n[0])
    expect_v[b:b + cnt] = par["disturbance_A"] * np.sin(2 * math.pi * par["disturbance_kappa"] * xc[b:b + cnt])
    assert np.max(np.abs(interp(W[2])[ix] - expect_v)) < 1e-15
    assert np.max(np.abs(interp(W[1])[ix])) < 1e-15
    assert np.max(np.abs(interp(T)[ix] - c["t_wall"][1][0])) < 1e-12


def test_periodic_and_zero_gradient_halos():
    P = ("periodic", "periodic")
    c = wl.random_box(3, (8, 7, 6), bc=(P, ("zero_gradient", "zero_gradient"), P))
    case, grid, U = padded_state(c, seed=6)
    nf.fill_halos(U, case, grid)
    h = 3
    assert np.array_equal(U[:, h:-h, h:-h, 0:h], U[:, h:-h, h:-h, 8:8 + h])
    assert np.array_equal(U[:, :, 0, :], U[:, :, h, :])
    assert np.array_equal(U[:, :, -1, :], U[:, :, -h - 1, :])
    assert np.array_equal(U[:, 0:h], U[:, 6:6 + h])       # z pass copies full x-y planes


# ---------------------------------------------------------------------------------------------
# time integration
# ---------------------------------------------------------------------------------------------
def test_rk3_stability_polynomial():
    """For dU/dt = lam U one step multiplies by 1 + z + z^2/2 + z^3/6 (z = lam dt): the three-stage
    third-order Runge-Kutta amplification factor."""
    for z in (-0.3, 0.2, -1.7, 0.05):
        U = np.ones((1, 4))
        out = nf.rk3(U, 1.0, lambda V: z * V, (slice(None),) * 2)
        assert abs(out[0, 0] - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-15


def test_taylor_green_initial_dissipation():
    """-dE_k/dt at t = 0 equals the incompressible closed form (3/4) nu V0^2 / L^2 per unit volume
    (nu = 1/1600), within the discretisation error at 32^3."""
    c = wl.tgv_case(32)
    case = nf.Case(c)
    grid = nf.Grid(case)
    h = case.h
    xs = [grid.axes[a].xc[h[a]:h[a] + 32] for a in range(3)]
    W = wl.tgv_prims(c, *xs)
    Wp = np.pad(W, [(0, 0)] + [(3, 3)] * 3, mode="edge")
    U = nf.prim_to_cons(Wp, case)
    R = nf.rhs(U.copy(), case, grid)
    vol = (2 * math.pi) ** 3
    rate = nf.kinetic_energy_rate(U, R, case, grid) / vol
    assert abs(nf.kinetic_energy(U, case, grid) / vol - 0.125) < 2e-3
    assert abs(-rate - 0.75 / 1600.0) < 0.03 * 0.75 / 1600.0, rate


# ---------------------------------------------------------------------------------------------
# viscosity laws (Sec. 3.2 uses Sutherland's law)
# ---------------------------------------------------------------------------------------------
def _suth_case(mu_ref, T_ref, S):
    return nf.Case(wl.random_box(1, (4, 1, 1), visc="sutherland", mu_ref=mu_ref, suth_S=S) |
                   dict(T_ref=T_ref))


def test_sutherland_reproduces_measured_air_viscosity():
    """Sutherland's law with White's constants for air against measured viscosities of air
    (tests/golden/air_viscosity.txt): within 1 % over 200-400 K.  A wrong exponent (1/2 instead of
    3/2) or the two sums T_ref + S and T + S exchanged misses by 10 % or more."""
    case = _suth_case(1.716e-5, 273.15, 110.4)
    rows = read_golden("air_viscosity.txt")
    T = np.array([float(r[0]) for r in rows])
    ref = np.array([float(r[1]) for r in rows]) * 1e-7
    mu = nf.viscosity(T, case)
    assert np.max(np.abs(mu / ref - 1.0)) < 0.01, mu / ref
    assert nf.viscosity(np.array([273.15]), case)[0] == pytest.approx(1.716e-5, rel=1e-15)


def test_sutherland_log_slope():
    """d ln mu / d ln T = 3/2 - T / (T + S) for Sutherland's law (differentiate
    ln mu = 3/2 ln T - ln(T + S) + const): mu grows like T^(3/2) far below S and like T^(1/2) far
    above it.  Checked by central differences of the oracle's mu in ln T."""
    S = 0.368
    case = _suth_case(0.7, 1.3, S)
    h = 1e-4
    for T in (0.01, 0.2, 1.0, 3.0, 50.0):
        lo, hi = nf.viscosity(np.array([T * math.exp(-h), T * math.exp(h)]), case)
        slope = (math.log(hi) - math.log(lo)) / (2 * h)
        assert abs(slope - (1.5 - T / (T + S))) < 1e-7, (T, slope)


def test_power_law_viscosity():
    """mu = mu_ref (T / T_ref)^e: mu(T_ref) = mu_ref and the log slope is the exponent."""
    case = nf.Case(wl.random_box(1, (4, 1, 1), visc="power", mu_ref=0.3) | dict(T_ref=2.0,
                                                                               visc_exp=0.7))
    assert nf.viscosity(np.array([2.0]), case)[0] == 0.3
    a, b = nf.viscosity(np.array([1.0, 4.0]), case)
    assert math.log(b / a) / math.log(4.0) == pytest.approx(0.7, rel=1e-13)


# ---------------------------------------------------------------------------------------------
# CFL time step: the viscous branch
# ---------------------------------------------------------------------------------------------
def _rest_state(ndim, n, rho, p, mu, Pr, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), stretch=None):
    P = ("periodic", "periodic")
    c = wl.random_box(ndim, (n,) * 3, bc=(P, P, P), visc="constant", mu_ref=mu, lo=lo, hi=hi,
                      stretch=stretch) | dict(Pr=Pr, cfl=0.5)
    return padded_state(c, uniform=(rho, 0.0, 0.0, 0.0, p))


def test_cfl_viscous_branch_worked_examples():
    """Fluid at rest: hand-worked time steps (tests/golden/cfl_worked_examples.txt) where the
    viscous limit binds (with gamma / Pr and with the 4/3 of the normal stress) and where the
    acoustic limit binds."""
    for name, n, rho, p, mu, Pr, dt in read_golden("cfl_worked_examples.txt"):
        for ndim in (1, 2, 3):
            case, grid, U = _rest_state(ndim, int(n), float(rho), float(p), float(mu), float(Pr))
            got = nf.cfl_dt(U, case, grid)
            assert got == pytest.approx(float(dt), rel=1e-14), (name, ndim, got)


def test_cfl_viscous_branch_scaling():
    """The viscous limit scales like dx^2 / nu: halving the spacing quarters it, doubling mu halves
    it, doubling rho doubles it; on a stretched axis the smallest cell decides."""
    base = _rest_state(2, 16, 1.0, 1.0, 2.0, 0.7)
    dt0 = nf.cfl_dt(base[2], base[0], base[1])
    fine = _rest_state(2, 32, 1.0, 1.0, 2.0, 0.7)
    assert nf.cfl_dt(fine[2], fine[0], fine[1]) == pytest.approx(dt0 / 4, rel=1e-13)
    visc = _rest_state(2, 16, 1.0, 1.0, 4.0, 0.7)
    assert nf.cfl_dt(visc[2], visc[0], visc[1]) == pytest.approx(dt0 / 2, rel=1e-13)
    dens = _rest_state(2, 16, 2.0, 2.0, 2.0, 0.7)        # same sound speed, twice the density
    assert nf.cfl_dt(dens[2], dens[0], dens[1]) == pytest.approx(dt0 * 2, rel=1e-13)
    case, grid, U = _rest_state(2, 16, 1.0, 1.0, 2.0, 0.7, lo=(0.0, -1.0, 0.0),
                                stretch=("uniform", "tanh2", "uniform"))
    dy = grid.axes[1].dx[3:3 + 16].min()
    k = 2.0 * max(4.0 / 3.0, 1.4 / 0.7)
    assert nf.cfl_dt(U, case, grid) == pytest.approx(0.5 * dy * dy / (k * 2.0), rel=1e-13)
    assert dy < 2.0 / 16


# ---------------------------------------------------------------------------------------------
# adiabatic wall and Dirichlet inflow halos
# ---------------------------------------------------------------------------------------------
def test_adiabatic_wall_face_values():
    """Adiabatic no-slip wall: at the wall face the interpolated velocity vanishes and so does the
    normal temperature derivative (fourth-order stencils); density and pressure are mirrored."""
    P = ("periodic", "periodic")
    c = wl.random_box(2, (10, 12, 1), bc=(P, ("adiabatic", "adiabatic"), P))
    case, grid, U = padded_state(c, seed=3)
    nf.fill_halos(U, case, grid)
    W, T = nf.cons_to_prim(U, case)
    h, n = 3, 12
    ix = slice(h, h + 10)
    for a in (h - 1, h + n - 1):                     # faces a + 1/2: south and north walls
        f = lambda q, o: q[0, a + o, ix]
        interp = lambda q: (9.0 * (f(q, 0) + f(q, 1)) - (f(q, -1) + f(q, 2))) / 16.0
        dn = lambda q: (f(q, -1) - f(q, 2)) + 27.0 * (f(q, 1) - f(q, 0))
        for comp in (1, 2, 3):
            assert np.max(np.abs(interp(W[comp]))) < 1e-15
        assert np.max(np.abs(dn(T))) < 1e-13 * np.max(np.abs(T))
    for m in range(h):
        for g, s in ((h - 1 - m, h + m), (h + n + m, h + n - 1 - m)):
            assert np.allclose(W[0, 0, g, ix], W[0, 0, s, ix], rtol=1e-15, atol=0)
            assert np.allclose(W[4, 0, g, ix], W[4, 0, s, ix], rtol=1e-15, atol=0)


def test_inflow_halo_layers_hold_the_profile():
    """Dirichlet inflow: every ghost layer of the inflow face converts back to the prescribed
    primitive profile, over the interior tangential range."""
    c = wl.porous_bl_case(nx=16, ny=20)
    case = nf.Case(c)
    grid = nf.Grid(case)
    xc = grid.axes[0].xc[3:3 + 16]
    yc = grid.axes[1].xc[3:3 + 20]
    case, grid, U = padded_state(c, prims=wl.porous_bl_prims(c, xc, yc))
    U[:, :, :, :3] = 7.0                             # stale values that the pass must replace
    prof = wl.porous_bl_inflow(c, grid.axes[1].xc)
    nf.fill_halos(U, case, grid, wl.porous_phi(c), {(0, 0): prof})
    W, _ = nf.cons_to_prim(U, case)
    for g in range(3):
        got = W[:, 0, 3:3 + 20, g]
        assert max(rel_err(got, prof[:, 0, 3:3 + 20])) < 1e-14, g


# ---------------------------------------------------------------------------------------------
# wall heat flux, wall shear and the integrated loss
# ---------------------------------------------------------------------------------------------
def _slab(T_lo, T_hi, prof_u=None, stretch_x=False, visc="power"):
    """2-D fluid between isothermal walls at y = -1 (T_lo) and y = 1 (T_hi): uniform pressure,
    T linear in y (so the wall mirror continues it exactly on a uniform y grid), velocity from
    prof_u(y) or zero."""
    c = wl.random_box(2, (8, 16, 1), bc=(("zero_gradient", "zero_gradient"), ("wall", "wall"),
                                          ("periodic", "periodic")),
                      visc=visc, mu_ref=0.05, t_wall=((1.0, 1.0), (T_lo, T_hi), (1.0, 1.0)),
                      lo=(0.0, -1.0, 0.0), hi=(2.5, 1.0, 1.0),
                      stretch=("tanh1" if stretch_x else "uniform", "uniform", "uniform"),
                      beta=(1.3, 0.0, 0.0))
    case = nf.Case(c)
    grid = nf.Grid(case)
    xc = grid.axes[0].xc[3:11]
    yc = grid.axes[1].xc[3:19]
    y2, x2 = np.meshgrid(yc, xc, indexing="ij")
    T = T_lo + (T_hi - T_lo) * (y2 + 1.0) / 2.0
    p = np.full_like(T, 1.3)
    u = prof_u(y2) if prof_u is not None else 0 * T
    W = np.stack([p / (case.R * T), u, 0 * T, 0 * T, p])[:, None]
    return padded_state(c, prims=W)


def test_wall_heat_flux_of_a_linear_temperature():
    """Fluid at rest with T linear between the walls: q_w = -lambda(T_w) dT/dy on both walls (the
    derivative along +y), exactly, and J = q_w times the wall length, also on a stretched wall
    axis (the cell widths along the wall sum to its length)."""
    T_lo, T_hi = 1.0, 2.2
    for stretch_x in (False, True):
        case, grid, U = _slab(T_lo, T_hi, stretch_x=stretch_x)
        grad = (T_hi - T_lo) / 2.0
        for side, Tw in ((0, T_lo), (1, T_hi)):
            lam = 0.05 * Tw ** 0.7 * case.cp / case.Pr
            qw, tw = nf.wall_fluxes(U, case, grid, 1, side)
            assert qw.shape[-1] == 8
            assert np.max(np.abs(qw + lam * grad)) < 1e-12 * lam * grad, (side, qw)
            assert np.max(np.abs(tw)) < 1e-15
            J = nf.wall_heat_loss(U, case, grid, 1, side)
            assert J == pytest.approx(-lam * grad * 2.5, rel=1e-12)


def test_wall_shear_of_couette_flow():
    """Linear shear u = s (y + 1) vanishes at the south wall, where the no-slip mirror continues it
    exactly: the wall shear is mu(T_w) s, and the heat flux is zero in an isothermal fluid."""
    s = 0.8
    case, grid, U = _slab(1.7, 1.7, prof_u=lambda y: s * (y + 1.0), visc="sutherland")
    qw, tw = nf.wall_fluxes(U, case, grid, 1, 0)
    mu_w = 0.05 * 1.7 ** 1.5 * (1.0 + 0.4) / (1.7 + 0.4)
    assert np.max(np.abs(tw - mu_w * s)) < 1e-13
    assert np.max(np.abs(qw)) < 1e-13


# ---------------------------------------------------------------------------------------------
# stretched-grid geometry and metrics (tanh mappings; Sec. 3.2 gives beta = 2.2)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("stretch,beta", [("tanh1", 2.2), ("tanh2", 2.0), ("uniform", 0.0)])
def test_axis_geometry_and_metrics(stretch, beta):
    """Faces at eta = 0 and 1 land on the domain ends; cell widths sum to the length; centres are
    face midpoints; the centre and face metrics d(index)/dx equal n over the derivative of the
    face mapping taken by fourth-order central differences of x(eta) alone."""
    n, h, lo, hi = 24, 3, -0.3, 1.9
    ax = nf.Axis(n, h, lo, hi, stretch, beta)
    xf_lo = ax.xc[h] - 0.5 * ax.dx[h]
    xf_hi = ax.xc[h + n - 1] + 0.5 * ax.dx[h + n - 1]
    assert xf_lo == pytest.approx(lo, abs=1e-15) and xf_hi == pytest.approx(hi, abs=1e-14)
    assert np.sum(ax.dx[h:h + n]) == pytest.approx(hi - lo, rel=1e-14)
    assert np.all(ax.dx > 0)
    xmap = lambda eta: nf._map(stretch, beta, lo, hi, np.asarray(eta, dtype=np.float64))[0]
    e = 1e-3
    deriv = lambda eta: (-xmap(eta + 2 * e) + 8 * xmap(eta + e) - 8 * xmap(eta - e)
                         + xmap(eta - 2 * e)) / (12 * e)
    a = np.arange(-h, n + h, dtype=np.float64)
    assert np.allclose(ax.mc, n / deriv((a + 0.5) / n), rtol=1e-9, atol=0)
    assert np.allclose(ax.mf, n / deriv((a + 1.0) / n), rtol=1e-9, atol=0)
    xf = xmap(np.arange(-h, n + h + 1) / n)
    assert np.allclose(ax.xc, 0.5 * (xf[1:] + xf[:-1]), rtol=0, atol=1e-15)
    if stretch == "tanh1":
        assert np.all(np.diff(ax.dx[h:h + n]) > 0)               # clustered at the low end
    if stretch == "tanh2":
        assert np.allclose(ax.dx[h:h + n], ax.dx[h:h + n][::-1], rtol=1e-12, atol=0)
        assert ax.dx[h] < ax.dx[h + n // 2] / 3                  # clustered at both ends


def _stretched_visc_error(n):
    """Max error of the dissipative fluxes on the y faces (normal stencils, face metric) and on the
    x faces (tangential y stencils, centre metric) of a smooth 2-D field on a tanh-stretched y axis.
    The field is sampled at the mapped centre positions x(eta_centre), so the uniform-index
    stencils approximate the derivatives in eta to fourth order and the metrics convert them."""
    P = ("periodic", "periodic")
    c = wl.random_box(2, (n, n, 1), bc=(P, P, P), visc="power", mu_ref=0.1,
                      lo=(0.0, -1.0, 0.0), hi=(2 * math.pi, 1.0, 1.0),
                      stretch=("uniform", "tanh2", "uniform"), beta=(0.0, 1.8, 0.0))
    case = nf.Case(c)
    grid = nf.Grid(case)
    h = 3
    ymap = lambda eta: nf._map("tanh2", 1.8, -1.0, 1.0, eta)[0]
    a = np.arange(-h, n + h, dtype=np.float64)
    yc = ymap((a + 0.5) / n)
    yf = ymap((a + 1.0) / n)
    xc = grid.axes[0].xc
    xf = xc + 0.5 * grid.axes[0].dx

    def fields(x, y):
        rho = 1.0 + 0.2 * np.sin(x) * np.cos(y)
        u = np.sin(x) * np.cos(1.3 * y)
        v = 0.5 * np.cos(x) * np.sin(y)
        p = 1.0 + 0.1 * np.cos(x + y)
        return rho, u, v, p

    def exact(x, y, d):
        rho, u, v, p = fields(x, y)
        rx, ry = 0.2 * np.cos(x) * np.cos(y), -0.2 * np.sin(x) * np.sin(y)
        ux, uy = np.cos(x) * np.cos(1.3 * y), -1.3 * np.sin(x) * np.sin(1.3 * y)
        vx, vy = -0.5 * np.sin(x) * np.sin(y), 0.5 * np.cos(x) * np.cos(y)
        px, py = -0.1 * np.sin(x + y), -0.1 * np.sin(x + y)
        T = p / rho
        Tg = ((px * rho - p * rx) / rho ** 2, (py * rho - p * ry) / rho ** 2)
        mu = 0.1 * T ** 0.7
        div = ux + vy
        if d == 0:
            tn = mu * (2 * ux - 2.0 / 3.0 * div)
            tt = mu * (uy + vx)
            return [tn, tt, u * tn + v * tt + mu * case.cp / case.Pr * Tg[0]]
        tt = mu * (uy + vx)
        tn = mu * (2 * vy - 2.0 / 3.0 * div)
        return [tt, tn, u * tt + v * tn + mu * case.cp / case.Pr * Tg[1]]

    y2, x2 = np.meshgrid(yc, xc, indexing="ij")
    rho, u, v, p = fields(x2, y2)
    W = np.stack([rho, u, v, 0 * u, p])[:, None]
    T = W[4] / (W[0] * case.R)
    err = 0.0
    inner_x = (0, slice(h, h + n), slice(None))      # x faces over interior rows
    F = nf.viscous_face_flux(W, T, case, grid, 0)
    ye, xe = np.meshgrid(yc, xf[h - 1:h + n], indexing="ij")
    for got, ex in zip((F[1], F[2], F[4]), exact(xe, ye, 0)):
        err = max(err, np.max(np.abs(got[inner_x] - ex[h:h + n])))
    inner_y = (0, slice(None), slice(h, h + n))      # y faces over interior columns
    F = nf.viscous_face_flux(W, T, case, grid, 1)
    ye, xe = np.meshgrid(yf[h - 1:h + n], xc, indexing="ij")
    for got, ex in zip((F[1], F[2], F[4]), exact(xe, ye, 1)):
        err = max(err, np.max(np.abs(got[inner_y] - ex[:, h:h + n])))
    return err


def test_viscous_flux_fourth_order_on_stretched_grid():
    """Fourth-order convergence of the dissipative fluxes on a tanh-stretched axis: a wrong face or
    centre metric (for instance the cell width in place of the mapping derivative) drops the order
    to two or less."""
    e = [_stretched_visc_error(n) for n in (16, 32, 64)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert orders[-1] > 3.6, (e, orders)


def test_wall_fluxes_agree_with_the_face_flux_on_stretched_walls():
    """On a stretched wall-normal axis (random state, both walls): the wall heat flux is minus the
    energy component of the dissipative face flux at the wall face (the face velocity is zero there)
    and the wall shear is its tangential momentum component, whose metric and stencils the
    stretched-grid convergence test pins."""
    P = ("periodic", "periodic")
    c = wl.random_box(2, (12, 16, 1), bc=(P, ("wall", "wall"), P), visc="sutherland",
                      stretch=("uniform", "tanh2", "uniform"), beta=(0.0, 1.9, 0.0),
                      t_wall=((1.0, 1.0), (1.1, 0.9), (1.0, 1.0)))
    case, grid, U = padded_state(c, seed=11, amp=0.3)
    Uf = U.copy()
    nf.fill_halos(Uf, case, grid)
    W, T = nf.cons_to_prim(Uf, case)
    F = nf.viscous_face_flux(W, T, case, grid, 1)         # faces a + 1/2, a = 2 .. 18
    for side, row in ((0, 0), (1, -1)):
        qw, tw = nf.wall_fluxes(U, case, grid, 1, side)
        assert np.max(np.abs(qw[0, 0] + F[4][0, row, 3:15])) < 1e-13 * np.max(np.abs(qw))
        assert np.max(np.abs(tw[0, 0] - F[1][0, row, 3:15])) < 1e-13 * np.max(np.abs(tw))


def test_wall_heat_loss_weights_by_cell_width():
    """J = sum_i q_w,i dx_i: with a wall-normal temperature gradient g(x) that varies along a
    stretched wall, J is -lambda(T_w) times the width-weighted sum of g over the wall cells."""
    c = wl.random_box(2, (10, 12, 1), bc=(("zero_gradient", "zero_gradient"), ("wall", "wall"),
                                           ("periodic", "periodic")),
                      visc="constant", mu_ref=0.05, t_wall=((1.0, 1.0), (1.0, 1.0), (1.0, 1.0)),
                      lo=(0.0, 0.0, 0.0), hi=(3.0, 1.0, 1.0), stretch=("tanh1", "uniform", "uniform"),
                      beta=(2.0, 0.0, 0.0))
    case = nf.Case(c)
    grid = nf.Grid(case)
    xc = grid.axes[0].xc[3:13]
    yc = grid.axes[1].xc[3:15]
    y2, x2 = np.meshgrid(yc, xc, indexing="ij")
    g = 0.3 + 0.2 * np.sin(x2)
    T = 1.0 + g * y2
    p = np.full_like(T, 1.1)
    W = np.stack([p / (case.R * T), 0 * T, 0 * T, 0 * T, p])[:, None]
    case, grid, U = padded_state(c, prims=W)
    lam = 0.05 * case.cp / case.Pr
    gw = 0.3 + 0.2 * np.sin(xc)
    J = nf.wall_heat_loss(U, case, grid, 1, 0)
    assert J == pytest.approx(-lam * np.sum(gw * grid.axes[0].dx[3:13]), rel=1e-12)
    assert abs(np.sum(gw * grid.axes[0].dx[3:13]) - np.mean(gw) * 3.0) > 1e-3   # weights matter
