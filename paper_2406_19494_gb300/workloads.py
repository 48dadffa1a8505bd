"""Seeded synthetic workloads: case descriptions and initial primitive fields.

This module holds no arithmetic of the method itself (no flux, reconstruction, boundary, time
integration or equation-of-state code): it only describes cases as plain dicts and draws initial
primitive fields (rho, u, v, w, p) at cell-centre coordinates that the caller supplies.  Both the
CUDA path (through the package binding) and the CPU oracle (in the tests) start from these fields,
so both see identical input bits.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) in its counter form: draw i of stream `seed` is mix(seed + (i + 1) * phi64).

Cases (the configurations the solver is exercised and measured on):
  sod          1-D Sod shock tube, 200 cells, WENO5-JS + HLLC, transmissive ends
  tgv          3-D compressible Taylor-Green vortex, 128^3, Ma 0.1, Re 1600, Pr 0.71, power-law mu
  channel      3-D compressible channel, Ma_b 1.5, Re_b 3000, 192x128x128, tanh-stretched walls
  porous_bl    2-D Ma 6 laminar boundary layer, 512x128, disturbance/porous strip on the wall
  e2           2-D Ma 2.25 laminar boundary layer, 300x200, adiabatic wall, similarity inlet
  random_box   small random states on any boundary mix, for parity tests
  serving      a stream of independent solves of uneven sizes (isentropic vortices, four-quadrant
               Riemann problems, Taylor-Green vortices) with Poisson arrival times
"""
import math

import numpy as np

_PHI64 = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, n):
    """n 64-bit outputs of the counter-based SplitMix64 stream `seed`."""
    with np.errstate(over="ignore"):
        x = np.uint64(seed) + (np.arange(1, n + 1, dtype=np.uint64) * _PHI64)
        z = (x ^ (x >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed, n):
    """n doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _base(ndim, n, lo, hi, bc, **kw):
    d = dict(ndim=ndim, n=tuple(n), lo=tuple(lo), hi=tuple(hi), bc=tuple(bc),
             stretch=("uniform",) * 3, beta=(0.0, 0.0, 0.0), t_wall=((0.0, 0.0),) * 3,
             gamma=1.4, R=1.0, Pr=0.72, visc="none", mu_ref=0.0, T_ref=1.0, visc_exp=0.7,
             suth_S=0.0, weno="z", weno_eps=None, body_force=(0.0, 0.0, 0.0), cfl=0.5,
             dt_fixed=0.0, porous=None)
    d.update(kw)
    return d


# ------------------------------------------------------------------------------------------------
# case descriptions
# ------------------------------------------------------------------------------------------------
def sod_case(n=200):
    """Sod shock tube on [0, 1]: gamma 1.4, WENO5-JS + HLLC + TVD-RK3, CFL 0.5, transmissive ends."""
    P = ("periodic", "periodic")
    return _base(1, (n, 1, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0),
                 (("zero_gradient", "zero_gradient"), P, P), weno="js", name="sod%d" % n)


def sod_prims(xc):
    """Left (rho, u, p) = (1, 0, 1) for x < 0.5, right (0.125, 0, 0.1)."""
    left = xc < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    z = np.zeros_like(xc)
    return np.stack([rho, z, z, z, p])


TGV_MA, TGV_RE, TGV_PR = 0.1, 1600.0, 0.71


def tgv_case(n=128, weno="z"):
    """Compressible Taylor-Green vortex on the periodic box [0, 2 pi]^3.

    Nondimensional with rho0 = V0 = L = 1 and R = 1: p0 = 1 / (gamma Ma^2), T0 = p0, viscosity
    mu = (1 / Re) (T / T0)^0.7 (power law), Pr = 0.71, WENO5-Z + HLLC, CFL 0.5.
    """
    g = 1.4
    p0 = 1.0 / (g * TGV_MA ** 2)
    P = ("periodic", "periodic")
    return _base(3, (n, n, n), (0.0,) * 3, (2 * math.pi,) * 3, (P, P, P), gamma=g, R=1.0,
                 Pr=TGV_PR, visc="power", mu_ref=1.0 / TGV_RE, T_ref=p0, visc_exp=0.7, weno=weno,
                 name="tgv%d" % n)


def tgv_prims(case, xc, yc, zc):
    """Taylor-Green initial condition (textbook closed form) at cell centres xc, yc, zc (1-D arrays):
    u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    p = p0 + (cos 2x + cos 2y)(cos 2z + 2) / 16, T uniform = T0 so rho = p / (R T0)."""
    z, y, x = np.meshgrid(zc, yc, xc, indexing="ij")
    p0 = case["T_ref"] * case["R"]            # rho0 = 1 at T0
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p = p0 + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    rho = p / (case["R"] * case["T_ref"])
    return np.stack([rho, u, v, w, p])


CH_MA, CH_RE, CH_PR = 1.5, 3000.0, 0.72


def channel_case(nx=192, ny=128, nz=128, beta=2.0):
    """Compressible channel on [0, 4 pi] x [-1, 1] x [0, 4 pi / 3], Ma_b 1.5, Re_b 3000.

    Nondimensional rho_b = U_b = h = T_w = 1; c_w = 1 / Ma_b gives R = c_w^2 / gamma;
    mu = (1 / Re_b) T^0.7; isothermal no-slip walls at T_w = 1, periodic x and z, tanh
    stretching in y; constant body force f_x = 3 mu_w U_b / h^2 (laminar force balance).
    """
    g = 1.4
    R = (1.0 / CH_MA) ** 2 / g
    mu_w = 1.0 / CH_RE
    P = ("periodic", "periodic")
    return _base(3, (nx, ny, nz), (0.0, -1.0, 0.0), (4 * math.pi, 1.0, 4 * math.pi / 3),
                 (P, ("wall", "wall"), P), stretch=("uniform", "tanh2", "uniform"),
                 beta=(0.0, beta, 0.0), t_wall=((0.0, 0.0), (1.0, 1.0), (0.0, 0.0)), gamma=g, R=R,
                 Pr=CH_PR, visc="power", mu_ref=mu_w, T_ref=1.0, visc_exp=0.7, weno="z",
                 body_force=(3.0 * mu_w, 0.0, 0.0), name="channel%dx%dx%d" % (nx, ny, nz))


def channel_prims(case, xc, yc, zc, seed=0, amp=0.05):
    """Laminar Poiseuille u = 1.5 (1 - y^2), rho = T = 1, plus `amp` (5 %) seeded uniform noise on
    u, v and w (stream `seed`, ordered component-major then z, y, x)."""
    z, y, x = np.meshgrid(zc, yc, xc, indexing="ij")
    N = x.size
    r = uniform01(seed, 3 * N).reshape(3, *x.shape)
    u = 1.5 * (1.0 - y * y) + amp * (2.0 * r[0] - 1.0)
    v = amp * (2.0 * r[1] - 1.0)
    w = amp * (2.0 * r[2] - 1.0)
    rho = np.ones_like(u)
    p = rho * case["R"] * 1.0
    return np.stack([rho, u, v, w, p])


BL_MA, BL_PR, BL_RE_UNIT = 6.0, 0.72, 1.0e4
BL_TWALL = 4.0                 # wall temperature / edge temperature (isothermal porous wall)
BL_TE_KELVIN = 300.0           # dimensional edge temperature for Sutherland's constant


def porous_bl_case(nx=512, ny=128, beta=2.2, porous_count=None):
    """Ma 6 laminar flat-plate boundary layer on [1, 1.5] x [0, 0.4] (the paper's Sec. 3.2 domain).

    Nondimensional rho_e = u_e = T_e = 1, R = 1 / (gamma Ma^2), mu_e = 1 / Re_unit with
    Re_unit = 1e4, Sutherland viscosity (S = 110.4 K / 300 K), Pr = 0.72, y stretched towards the
    wall (tanh, beta = 2.2); west: Dirichlet inflow profile, east and north: zero gradient, south:
    isothermal no-slip wall at T_w = 4 with a porous strip on the middle `porous_count` wall cells
    carrying v_w,i = (A / phi0) phi_i sin(2 pi kappa x_i), A = 0.01, kappa = 10, phi0 = 0.1.
    """
    g = 1.4
    R = 1.0 / (g * BL_MA ** 2)
    cnt = nx // 2 if porous_count is None else porous_count
    P = ("periodic", "periodic")
    return _base(2, (nx, ny, 1), (1.0, 0.0, 0.0), (1.5, 0.4, 1.0),
                 (("inflow", "zero_gradient"), ("porous", "zero_gradient"), P),
                 stretch=("uniform", "tanh1", "uniform"), beta=(0.0, beta, 0.0),
                 t_wall=((0.0, 0.0), (BL_TWALL, 0.0), (0.0, 0.0)), gamma=g, R=R, Pr=BL_PR,
                 visc="sutherland", mu_ref=1.0 / BL_RE_UNIT, T_ref=1.0,
                 suth_S=110.4 / BL_TE_KELVIN, weno="z",
                 porous=dict(axis=1, side=0, begin=(nx - cnt) // 2, count=cnt, A=0.01, kappa=10.0,
                             phi0=0.1),
                 name="porous_bl%dx%d" % (nx, ny))


def porous_phi(case, seed=0, noise=0.1):
    """Per-cell admittances phi_i = phi0 (1 + noise U(-1, 1)) on the porous strip (stream `seed`)."""
    pz = case["porous"]
    r = uniform01(seed + 1000, pz["count"])
    return pz["phi0"] * (1.0 + noise * (2.0 * r - 1.0))


def _blasius(n_eta=4001, eta_max=10.0):
    """Incompressible Blasius profile f'(eta) of f''' + f f'' / 2 = 0 by RK4 shooting on f''(0)."""
    h = eta_max / (n_eta - 1)

    def integrate(s):
        y = np.array([0.0, 0.0, s])
        out = np.zeros(n_eta)
        rhs = lambda y: np.array([y[1], y[2], -0.5 * y[0] * y[2]])
        for k in range(n_eta):
            out[k] = y[1]
            if k == n_eta - 1:
                break
            k1 = rhs(y); k2 = rhs(y + 0.5 * h * k1); k3 = rhs(y + 0.5 * h * k2); k4 = rhs(y + h * k3)
            y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        return out

    lo, hi = 0.2, 0.5
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if integrate(mid)[-1] > 1.0:
            hi = mid
        else:
            lo = mid
    return np.linspace(0.0, eta_max, n_eta), integrate(0.5 * (lo + hi))


def porous_bl_prims(case, xc, yc):
    """Inflow-profile initial state, the same in every column: incompressible Blasius u/u_e with a
    Crocco-Busemann temperature for the isothermal wall (T_w / T_e = 4), mapped to y by the
    Howarth-Dorodnitsyn stretch y = sqrt(2 x / Re_unit) * integral T/T_e d eta at x = 1;
    uniform pressure p = rho_e R T_e, v = w = 0."""
    g = case["gamma"]
    eta, fp = _blasius()
    m2 = 0.5 * (g - 1.0) * BL_MA ** 2
    Tw = case["t_wall"][1][0]
    T = Tw + (1.0 + m2 - Tw) * fp - m2 * fp * fp
    dy = np.concatenate([[0.0], np.cumsum(0.5 * (T[1:] + T[:-1]) * np.diff(eta))])
    ysim = math.sqrt(2.0 * 1.0 / BL_RE_UNIT) * dy
    u1 = np.interp(yc, ysim, fp, right=1.0)
    T1 = np.interp(yc, ysim, T, right=1.0)
    p = case["R"] * 1.0
    y2, x2 = np.meshgrid(yc, xc, indexing="ij")
    u = np.broadcast_to(u1[:, None], y2.shape)
    Tf = np.broadcast_to(T1[:, None], y2.shape)
    rho = p / (case["R"] * Tf)
    z = np.zeros_like(u)
    out = np.stack([rho, u, z, z, np.full_like(u, p)])
    return out[:, None, :, :]


def porous_bl_inflow(case, yc_padded):
    """Inflow profile on the west face plane: primitives shaped (5, 1, py) over padded y."""
    W = porous_bl_prims(case, np.array([case["lo"][0]]), yc_padded)   # (5, 1, py, 1)
    return np.ascontiguousarray(W[:, :, :, 0])


# ------------------------------------------------------------------------------------------------
# compressible laminar boundary layer (Section 3.2's validation case): the similarity solution that
# the inlet imposes and that the outlet profile is compared with
# ------------------------------------------------------------------------------------------------
E2_MA, E2_PR, E2_RE_UNIT, E2_TE_KELVIN = 2.25, 0.72, 1.0e4, 300.0


def similarity_bl(Ma, Pr, gamma=1.4, suth=None, wall="adiabatic", g_wall=None, eta_max=12.0, n=2401):
    """Similarity solution of the compressible laminar flat-plate boundary layer in the
    Illingworth-Levy variables eta = u_e / sqrt(2 rho_e mu_e u_e x) int_0^y rho dy (Section 3.2):

        (C f'')' + f f'' = 0,    (C / Pr g')' + f g' + (gamma - 1) Ma^2 C f''^2 = 0,

    u / u_e = f'(eta), g = T / T_e = rho_e / rho (constant pressure), C = rho mu / (rho_e mu_e) =
    mu(g) / g with Sutherland's law mu / mu_e = g^{3/2} (1 + s) / (g + s), s = S / T_e (suth), or
    C = 1 (suth None).  f(0) = f'(0) = 0, f'(inf) = 1, g(inf) = 1, and at the wall g'(0) = 0
    (adiabatic) or g(0) = g_wall (isothermal).  Shooting on the two unknown wall values (C f''(0)
    and g(0), or C f''(0) and C g'(0) / Pr) with classical RK4 on a uniform eta grid and Newton's
    method with a finite-difference Jacobian.

    Returns a dict of arrays over eta: eta, f, fp (f'), fpp (f''), g, and Y = int_0^eta g, which maps
    eta to the wall distance y = sqrt(2 x / Re_x_unit) Y(eta) in units of the edge state."""
    h = eta_max / (n - 1)
    gm = (gamma - 1.0) * Ma * Ma

    def C(g):
        if suth is None:
            return np.ones_like(g)
        return np.sqrt(g) * (1.0 + suth) / (g + suth)

    def rhs(y):
        f, fp, tau, g, q = y
        c = C(g)
        fpp = tau / c
        gp = q * Pr / c
        return np.array([fp, fpp, -f * fpp, gp, -f * gp - gm * c * fpp * fpp])

    def shoot(u0, u1, record=False):
        # unknowns: tau(0) = C f''(0) and g(0) (adiabatic, q(0) = 0) or q(0) (isothermal)
        u0 = np.atleast_1d(u0).astype(np.float64)
        u1 = np.atleast_1d(u1).astype(np.float64)
        z = np.zeros_like(u0)
        if wall == "adiabatic":
            y = np.array([z, z, u0, u1, z])
        else:
            y = np.array([z, z, u0, np.full_like(u0, g_wall), u1])
        rows = [y.copy()] if record else None
        for _ in range(n - 1):
            k1 = rhs(y)
            k2 = rhs(y + 0.5 * h * k1)
            k3 = rhs(y + 0.5 * h * k2)
            k4 = rhs(y + h * k3)
            y = y + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
            if record:
                rows.append(y.copy())
        return (np.array(rows) if record else y)

    u = np.array([0.47, 1.0 + 0.85 * 0.5 * gm if wall == "adiabatic" else 0.0])
    if wall != "adiabatic":
        u[1] = -0.2 * (g_wall - 1.0)
    for _ in range(40):
        e = 1e-7 * np.maximum(1.0, np.abs(u))
        y = shoot([u[0], u[0] + e[0], u[0]], [u[1], u[1], u[1] + e[1]])
        res = np.array([y[1] - 1.0, y[3] - 1.0])            # f'(inf) - 1, g(inf) - 1 for the 3 runs
        J = np.array([(res[:, 1] - res[:, 0]) / e[0], (res[:, 2] - res[:, 0]) / e[1]]).T
        du = np.linalg.solve(J, -res[:, 0])
        u = u + du
        if np.max(np.abs(res[:, 0])) < 1e-12 and np.max(np.abs(du)) < 1e-12:
            break
    rows = shoot(u[0], u[1], record=True)[:, :, 0]
    eta = np.linspace(0.0, eta_max, n)
    f, fp, tau, g, q = rows.T
    Y = np.concatenate([[0.0], np.cumsum(0.5 * h * (g[1:] + g[:-1]))])
    return dict(eta=eta, f=f, fp=fp, fpp=tau / C(g), g=g, Y=Y)


def e2_case(nx=300, ny=200, beta=2.2):
    """Compressible laminar boundary layer of Section 3.2 (the no-disturbance validation): Ma 2.25,
    Pr 0.72, gamma 1.4, [1, 1.5] x [0, 0.4] with 300 x 200 cells, uniform in x and tanh-stretched
    towards the wall in y (beta = 2.2), adiabatic no-slip wall at the south, zero gradient at the
    north and east, the similarity solution imposed at the west inlet, Re per unit length 1e4,
    Sutherland viscosity (S = 110.4 K over an edge temperature of 300 K, this build's reading).
    Nondimensional rho_e = u_e = T_e = 1, R = 1 / (gamma Ma^2), mu_e = 1 / Re."""
    g = 1.4
    Z = ("zero_gradient", "zero_gradient")
    return _base(2, (nx, ny, 1), (1.0, 0.0, 0.0), (1.5, 0.4, 1.0),
                 (("inflow", "zero_gradient"), ("adiabatic", "zero_gradient"), ("periodic", "periodic")),
                 stretch=("uniform", "tanh1", "uniform"), beta=(0.0, beta, 0.0), gamma=g,
                 R=1.0 / (g * E2_MA ** 2), Pr=E2_PR, visc="sutherland", mu_ref=1.0 / E2_RE_UNIT,
                 T_ref=1.0, suth_S=110.4 / E2_TE_KELVIN, weno="z", name="e2_bl%dx%d" % (nx, ny))


def e2_similarity(case):
    """The similarity solution of the case's edge state (adiabatic wall, its Sutherland constant)."""
    return similarity_bl(E2_MA, case["Pr"], case["gamma"], suth=case["suth_S"])


def similarity_field(case, sim, x, y):
    """Primitives (rho, u, v, w, p) of the self-similar boundary layer at stations x (1-D) and wall
    distances y (1-D), shaped (5, 1, len(y), len(x)): u = f'(eta), T = g(eta), v = (f' Y - g f) /
    sqrt(2 Re_x) (from the stream function sqrt(2 xi) f(eta)), uniform pressure p = R T_e rho_e."""
    Re = 1.0 / case["mu_ref"]
    y2, x2 = np.meshgrid(y, x, indexing="ij")
    scale = np.sqrt(2.0 * x2 / Re)
    Ysim = np.abs(y2) / scale
    eta = np.interp(Ysim, sim["Y"], sim["eta"], right=np.nan)
    far = np.isnan(eta)
    Ymax, eta_max = sim["Y"][-1], sim["eta"][-1]
    eta = np.where(far, eta_max + (Ysim - Ymax), eta)        # beyond the table: g = 1, f' = 1
    fp = np.interp(eta, sim["eta"], sim["fp"], right=1.0)
    g = np.interp(eta, sim["eta"], sim["g"], right=1.0)
    f = np.interp(eta, sim["eta"], sim["f"], right=np.nan)
    f = np.where(np.isnan(f), sim["f"][-1] + (eta - eta_max), f)
    Yv = np.where(far, Ysim, np.interp(eta, sim["eta"], sim["Y"]))
    v = (fp * Yv - g * f) / np.sqrt(2.0 * Re * x2)
    p = case["R"] * 1.0
    rho = p / (case["R"] * g)
    z = np.zeros_like(fp)
    return np.stack([rho, fp, v, z, np.full_like(fp, p)])[:, None]


def e2_inflow(case, sim, yc_padded):
    """Inlet profile on the west face plane (x = lo): primitives shaped (5, 1, py) over padded y
    (ghost rows below the wall take the profile at |y|; the wall map replaces them)."""
    W = similarity_field(case, sim, np.array([case["lo"][0]]), yc_padded)
    return np.ascontiguousarray(W[:, :, :, 0])


def random_box(ndim=3, n=(20, 18, 16), bc=None, visc="power", weno="z", stretch=None,
               body_force=(0.0, 0.0, 0.0), seed=0, **kw):
    """A small case for parity tests; physical parameters of order one, viscosity high enough that
    the dissipative fluxes matter at these resolutions."""
    P = ("periodic", "periodic")
    if bc is None:
        bc = (P, P, P)
    n3 = tuple(n[a] if a < ndim else 1 for a in range(3))
    lo = kw.pop("lo", (0.0, -1.0, 0.0))
    hi = kw.pop("hi", (2.0, 1.0, 1.5))
    st = stretch if stretch is not None else ("uniform",) * 3
    return _base(ndim, n3, lo, hi, bc, stretch=st, beta=kw.pop("beta", (0.0, 1.6, 0.0)),
                 gamma=1.4, R=1.0, Pr=0.72, visc=visc, mu_ref=kw.pop("mu_ref", 0.02),
                 T_ref=1.0, visc_exp=0.7, suth_S=kw.pop("suth_S", 0.4), weno=weno,
                 body_force=body_force, t_wall=kw.pop("t_wall", ((1.0, 1.0),) * 3),
                 name="random%dd" % ndim, **kw)


def random_prims(xc, yc, zc, seed=0, amp=1.0, modes=4, jump=True):
    """Seeded random smooth field plus (optionally) a density/pressure jump, evaluated at the given
    cell-centre coordinates.  rho in about [0.5, 1.6], p in about [0.5, 1.6], |u| up to about 1.6
    (supersonic in places, so every HLLC branch occurs)."""
    z, y, x = np.meshgrid(zc, yc, xc, indexing="ij")
    r = uniform01(seed, 5 * modes * 7).reshape(5, modes, 7)
    out = []
    base = (1.0, 0.0, 0.0, 0.0, 1.0)
    scale = (0.25, 0.8 * amp, 0.8 * amp, 0.8 * amp, 0.25)
    for c in range(5):
        f = np.zeros_like(x)
        for m in range(modes):
            kx, ky, kz = (1 + np.floor(3 * r[c, m, 0:3])).tolist()
            ph = 2 * math.pi * r[c, m, 3:6]
            a = (2.0 * r[c, m, 6] - 1.0) / modes
            f += a * np.sin(kx * 3.1 * x + ph[0]) * np.cos(ky * 2.3 * y + ph[1]) * np.cos(kz * 1.7 * z + ph[2])
        out.append(base[c] + scale[c] * f * modes / 2.0)
    out = np.stack(out)
    if jump:
        sel = (x + 0.3 * y) > 1.1
        out[0] = np.where(sel, out[0] * 0.6, out[0])
        out[4] = np.where(sel, out[4] * 0.7, out[4])
    return out


# ------------------------------------------------------------------------------------------------
# serving stream
# ------------------------------------------------------------------------------------------------
def vortex_case(n):
    """2-D isentropic vortex on the periodic square [0, 10]^2, Euler, WENO5-Z."""
    P = ("periodic", "periodic")
    return _base(2, (n, n, 1), (0.0, 0.0, 0.0), (10.0, 10.0, 1.0), (P, P, P), weno="z",
                 name="vortex%d" % n)


def vortex_prims(xc, yc, strength=5.0, gamma=1.4):
    """Textbook isentropic vortex (free stream rho = u = v = p = 1, R = 1) centred at (5, 5):
    du = -b/(2 pi) e^{(1-r^2)/2} (y - 5), dv = b/(2 pi) e^{(1-r^2)/2} (x - 5),
    T = 1 - (gamma - 1) b^2 / (8 gamma pi^2) e^{1 - r^2}, rho = T^{1/(gamma-1)}, p = rho T."""
    y, x = np.meshgrid(yc, xc, indexing="ij")
    dx, dy = x - 5.0, y - 5.0
    r2 = dx * dx + dy * dy
    f = np.exp(0.5 * (1.0 - r2))
    u = 1.0 - strength / (2 * math.pi) * f * dy
    v = 1.0 + strength / (2 * math.pi) * f * dx
    T = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * math.pi ** 2) * f * f
    rho = T ** (1.0 / (gamma - 1.0))
    z = np.zeros_like(u)
    return np.stack([rho, u, v, z, rho * T])[:, None]


def riemann2d_case(n):
    """2-D four-quadrant Riemann problem on [0, 1]^2 with transmissive boundaries, Euler."""
    Z = ("zero_gradient", "zero_gradient")
    return _base(2, (n, n, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (Z, Z, ("periodic", "periodic")),
                 weno="z", name="riemann%d" % n)


def riemann2d_prims(xc, yc, seed):
    """Seeded moderate four-quadrant data: per quadrant rho in [0.5, 1.5], p in [0.4, 1.2],
    u, v in [-0.3, 0.3] (moderate jumps, no positivity limiter needed), split at (0.5, 0.5)."""
    r = uniform01(seed, 16).reshape(4, 4)
    y, x = np.meshgrid(yc, xc, indexing="ij")
    q = (x >= 0.5).astype(int) + 2 * (y >= 0.5).astype(int)
    rho = 0.5 + r[:, 0][q]
    u = -0.3 + 0.6 * r[:, 1][q]
    v = -0.3 + 0.6 * r[:, 2][q]
    p = 0.4 + 0.8 * r[:, 3][q]
    return np.stack([rho, u, v, np.zeros_like(u), p])[:, None]


def serving_stream(count=512, seed=0, frac_2d=0.7, n2d=(64, 1024), n3d=(32, 160), steps=(100, 2000),
                   rate_hz=None):
    """Requests of the serving workload: dicts with kind, n, nsteps, arrival_s (Poisson process of
    rate `rate_hz`, all at 0 when None) and seed.  2-D grids log-uniform in n2d^2 (half vortices,
    half Riemann problems), 3-D Taylor-Green grids log-uniform in n3d^3, steps uniform."""
    r = uniform01(seed + 77, 6 * count).reshape(count, 6)
    out = []
    t = 0.0
    for i in range(count):
        if rate_hz:
            t += -math.log(1.0 - r[i, 5]) / rate_hz
        if r[i, 0] < frac_2d:
            n = int(round(math.exp(math.log(n2d[0]) + r[i, 1] * (math.log(n2d[1]) - math.log(n2d[0])))))
            kind = "vortex" if r[i, 2] < 0.5 else "riemann"
        else:
            n = int(round(math.exp(math.log(n3d[0]) + r[i, 1] * (math.log(n3d[1]) - math.log(n3d[0])))))
            kind = "tgv"
        ns = int(steps[0] + r[i, 3] * (steps[1] - steps[0]))
        out.append(dict(kind=kind, n=n, nsteps=ns, arrival_s=t, seed=int(seed * 1000 + i)))
    return out


def serving_case_and_prims(req, centres_of):
    """(case, interior primitives) of one serving request; centres_of(case) gives (xc, yc, zc)."""
    if req["kind"] == "vortex":
        c = vortex_case(req["n"])
        xc, yc, _ = centres_of(c)
        return c, vortex_prims(xc, yc)
    if req["kind"] == "riemann":
        c = riemann2d_case(req["n"])
        xc, yc, _ = centres_of(c)
        return c, riemann2d_prims(xc, yc, req["seed"])
    c = tgv_case(req["n"])
    xc, yc, zc = centres_of(c)
    return c, tgv_prims(c, xc, yc, zc)
