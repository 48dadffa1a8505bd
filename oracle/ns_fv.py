"""Plain fp64 oracle of the paper's finite-volume compressible Navier-Stokes solver.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never imports this module.

What it computes (paper sections in brackets):

* conservative state U = (rho, rho u, rho v, rho w, E), E = rho e + |rho u|^2 / (2 rho)  [Sec. 2.1]
* ideal gas p = (gamma - 1) (E - rho |u|^2 / 2), T = p / (rho R)                        [Sec. 2.1, 3.2]
* convective face fluxes F^c, G^c, H^c by WENO5 reconstruction of the primitive variables
  (rho, u, v, w, p) and the HLLC approximate Riemann solver                            [Sec. 2.1, 3.1]
  or, as in the channel computation, TENO6-A with the interpolation limiter (oracle/teno.py)  [Sec. 3.1]
* dissipative face fluxes F^d, G^d, H^d: Newtonian stress with the Stokes hypothesis and
  Fourier heat flux, from fourth- or sixth-order central differences                   [Sec. 2.1, Eq. tau, Sec. 3.1]
* the semi-discrete update R = dU/dt of Eq. ODE, with a body-force source               [Eq. ODE, Eq. NSE]
* halo cells assigned by boundary conditions: periodic, zero-gradient, no-slip walls
  (isothermal, adiabatic), the "Disturbance Wall" transpiration wall, Dirichlet inflow  [Sec. 3.2]
* the explicit TVD Runge-Kutta step (third-order Shu-Osher form) and a CFL time step     [Sec. 2.1]

The paper names the schemes but prints no formula for them (Sec. 2.1, Sec. 3.1); the textbook
definitions used here are: WENO5-JS (Jiang & Shu 1996), WENO5-Z (Borges et al. 2008), HLLC with
Einfeldt/Roe wave-speed bounds (Toro, "Riemann Solvers and Numerical Methods", Ch. 10), Shu-Osher
TVD-RK3.  Every reading taken where the paper is silent is stated at the point of use.

Array layout: U has shape (5, pz, py, px) -- variable, then z, y, x, with x fastest; every active
axis carries H = 3 halo cells on each side (WENO5 needs three), inactive axes have one cell and no
halo.  Spatial axis d (0 = x, 1 = y, 2 = z) is numpy axis 2 - d of a (pz, py, px) field.

All functions are generic over the scalar dtype: with complex128 inputs every non-analytic step
(abs, min, max, branch) decides on the real part, which makes the complex-step derivative exact.
"""
import math

import numpy as np

from . import teno

H = 3                       # halo width
NVAR = 5
BC_KINDS = ("periodic", "zero_gradient", "wall", "adiabatic", "porous", "inflow")


# --------------------------------------------------------------------------------------------
# helpers that keep complex-step differentiation exact
# --------------------------------------------------------------------------------------------
def _re(x):
    return x.real if np.iscomplexobj(x) else x


def _abs(x):
    if np.iscomplexobj(x):
        return np.where(x.real < 0, -x, x)
    return np.abs(x)


def _min(a, b):
    return np.where(_re(a) <= _re(b), a, b)


def _max(a, b):
    return np.where(_re(a) >= _re(b), a, b)


# --------------------------------------------------------------------------------------------
# case description
# --------------------------------------------------------------------------------------------
class Case:
    """Physical and numerical parameters of one solve, read from a plain dict.

    Keys: ndim, n (3-tuple of interior cells), lo, hi (domain), stretch ('uniform' | 'tanh2' |
    'tanh1'), beta, bc (per axis a pair of kinds from BC_KINDS), t_wall (per axis a pair),
    gamma, R, Pr, visc ('none' | 'constant' | 'power' | 'sutherland'), mu_ref, T_ref, visc_exp,
    suth_S, weno ('js' | 'z' | 'teno6a'), weno_eps (None = textbook default), visc_order (4 | 6),
    body_force, cfl, dt_fixed,
    porous (dict: axis, side, begin, count, A, kappa, phi0) or None.
    """

    def __init__(self, d):
        self.ndim = int(d["ndim"])
        self.n = tuple(int(v) for v in d["n"])
        self.lo = tuple(float(v) for v in d["lo"])
        self.hi = tuple(float(v) for v in d["hi"])
        self.stretch = tuple(d.get("stretch", ("uniform",) * 3))
        self.beta = tuple(float(v) for v in d.get("beta", (0.0, 0.0, 0.0)))
        self.bc = tuple(tuple(p) for p in d["bc"])
        self.t_wall = tuple(tuple(float(v) for v in p) for p in d.get("t_wall", ((0, 0),) * 3))
        self.gamma = float(d["gamma"])
        self.R = float(d["R"])
        self.Pr = float(d.get("Pr", 0.72))
        self.visc = d.get("visc", "none")
        self.mu_ref = float(d.get("mu_ref", 0.0))
        self.T_ref = float(d.get("T_ref", 1.0))
        self.visc_exp = float(d.get("visc_exp", 0.7))
        self.suth_S = float(d.get("suth_S", 0.0))
        self.weno = d.get("weno", "z")
        eps = d.get("weno_eps", None)
        # Jiang & Shu use eps = 1e-6; Borges et al. use a tiny eps (1e-40) so that it never masks beta
        self.weno_eps = float(eps) if eps is not None else (1e-6 if self.weno == "js" else 1e-40)
        if self.weno not in ("js", "z", "teno6a", "linear"):
            raise ValueError("unknown reconstruction %r" % (self.weno,))
        # order of the central differences of the dissipative fluxes: 4 (default), or 6 as in the
        # paper's channel computation (Sec. 3.1)
        self.visc_order = int(d.get("visc_order", 4))
        if self.visc_order not in (4, 6):
            raise ValueError("visc_order must be 4 or 6")
        self.body_force = tuple(float(v) for v in d.get("body_force", (0.0, 0.0, 0.0)))
        self.cfl = float(d.get("cfl", 0.5))
        self.dt_fixed = float(d.get("dt_fixed", 0.0))
        self.porous = d.get("porous", None)
        for a in range(3):
            if a >= self.ndim and self.n[a] != 1:
                raise ValueError("inactive axes must have one cell")
            for s in range(2):
                if self.bc[a][s] not in BC_KINDS:
                    raise ValueError("unknown boundary kind %r" % (self.bc[a][s],))
        self.h = tuple(H if a < self.ndim else 0 for a in range(3))
        self.p = tuple(self.n[a] + 2 * self.h[a] for a in range(3))
        self.shape = (NVAR, self.p[2], self.p[1], self.p[0])

    @property
    def cp(self):
        return self.gamma * self.R / (self.gamma - 1.0)

    def interior(self):
        """Slices (z, y, x) selecting the interior of a (pz, py, px) field."""
        return tuple(slice(self.h[a], self.h[a] + self.n[a]) for a in (2, 1, 0))


# --------------------------------------------------------------------------------------------
# grid: uniform or tanh-stretched Cartesian axes (stretched meshes: Sec. 2, Sec. 3.2 beta = 2.2)
# --------------------------------------------------------------------------------------------
def _map(stretch, beta, lo, hi, eta):
    """Face coordinate x(eta) and its derivative dx/deta for eta in [0, 1] (extended outside).

    The paper gives only the stretching parameter; the mapping functions are this oracle's reading:
    'tanh2' clusters cells at both ends (channel walls), 'tanh1' at the low end (boundary-layer wall).
    """
    L = hi - lo
    if stretch == "uniform":
        return lo + L * eta, np.full_like(eta, L)
    tb = math.tanh(beta)
    if stretch == "tanh2":
        t = np.tanh(beta * (2.0 * eta - 1.0))
        return lo + 0.5 * L * (1.0 + t / tb), L * beta * (1.0 - t * t) / tb
    if stretch == "tanh1":
        t = np.tanh(beta * (1.0 - eta))
        return lo + L * (1.0 - t / tb), L * beta * (1.0 - t * t) / tb
    raise ValueError(stretch)


class Axis:
    """1-D geometry of one axis over its padded index range a = 0 .. p-1.

    xc     cell centre (midpoint of the two faces)
    dx     cell width (difference of face coordinates), used by the divergence and the CFL rule
    mc     d(index)/dx at the cell centre   -- metric of the centre derivative stencil
    mf     d(index)/dx at face a+1/2        -- metric of the face-normal derivative stencil
    """

    def __init__(self, n, h, lo, hi, stretch, beta):
        a = np.arange(-h, n + h, dtype=np.float64)
        if stretch == "uniform":
            d = (hi - lo) / n
            self.dx = np.full(a.shape, d)
            self.xc = lo + (a + 0.5) * d
            self.mc = np.full(a.shape, 1.0 / d)
            self.mf = np.full(a.shape, 1.0 / d)
        else:
            xf, _ = _map(stretch, beta, lo, hi, np.arange(-h, n + h + 1, dtype=np.float64) / n)
            self.dx = xf[1:] - xf[:-1]
            self.xc = 0.5 * (xf[1:] + xf[:-1])
            _, dc = _map(stretch, beta, lo, hi, (a + 0.5) / n)
            _, df = _map(stretch, beta, lo, hi, (a + 1.0) / n)
            self.mc = n / dc
            self.mf = n / df


class Grid:
    def __init__(self, case):
        self.axes = [Axis(case.n[a], case.h[a], case.lo[a], case.hi[a], case.stretch[a],
                          case.beta[a]) for a in range(3)]

    def along(self, name, a):
        """1-D metric array of axis a shaped to broadcast against a (pz, py, px) field."""
        v = getattr(self.axes[a], name)
        shp = [1, 1, 1]
        shp[2 - a] = v.size
        return v.reshape(shp)

    def along_inner(self, name, a, case):
        """Like along() but restricted to the interior cells of axis a."""
        h, n = case.h[a], case.n[a]
        v = getattr(self.axes[a], name)[h:h + n]
        shp = [1, 1, 1]
        shp[2 - a] = v.size
        return v.reshape(shp)

    def cell_volume(self):
        return self.along("dx", 0) * self.along("dx", 1) * self.along("dx", 2)

    def inner_volume(self, case):
        return (self.along_inner("dx", 0, case) * self.along_inner("dx", 1, case)
                * self.along_inner("dx", 2, case))


def _sl(a, lo, hi, ndim=3):
    """Index tuple selecting [lo, hi) along spatial axis a of a (pz, py, px) field."""
    s = [slice(None)] * ndim
    s[2 - a] = slice(lo, hi)
    return tuple(s)


# --------------------------------------------------------------------------------------------
# gas model (Sec. 2.1; ideal gas gamma = 1.4 in Sec. 3.2)
# --------------------------------------------------------------------------------------------
def cons_to_prim(U, case):
    """W = (rho, u, v, w, p) and T from U (Sec. 2.1: E = rho e + rho |u|^2 / 2, ideal gas)."""
    rho = U[0]
    u = U[1] / rho
    v = U[2] / rho
    w = U[3] / rho
    p = (case.gamma - 1.0) * (U[4] - 0.5 * rho * (u * u + v * v + w * w))
    T = p / (rho * case.R)
    return np.stack([rho, u, v, w, p]), T


def prim_to_cons(W, case):
    rho, u, v, w, p = W
    E = p / (case.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


def viscosity(T, case):
    """Dynamic viscosity mu(T): constant, power law, or Sutherland (Sec. 3.2 uses Sutherland)."""
    if case.visc == "constant":
        return case.mu_ref * np.ones_like(T)
    if case.visc == "power":
        return case.mu_ref * (T / case.T_ref) ** case.visc_exp
    if case.visc == "sutherland":
        return case.mu_ref * (T / case.T_ref) ** 1.5 * (case.T_ref + case.suth_S) / (T + case.suth_S)
    raise ValueError(case.visc)


# --------------------------------------------------------------------------------------------
# boundary conditions: values assigned to halo cells (Sec. 3.2)
# --------------------------------------------------------------------------------------------
def wall_velocity(case, grid, phi):
    """Wall-normal transpiration velocity v_w on the porous face, indexed by the padded index of the
    first tangential axis.

    Sec. 3.2 (disturbance wall) prescribes v = A sin(2 pi kappa x) with A = 0.01, kappa = 10.  With
    one learnable admittance phi_i per wall cell this oracle reads it as
    v_w,i = (A / phi0) phi_i sin(2 pi kappa x_i), so phi_i = phi0 reproduces the paper's disturbance
    exactly; cells outside the porous strip have v_w = 0.
    """
    pz = case.porous
    t1 = [a for a in range(case.ndim) if a != pz["axis"]][0]
    ax = grid.axes[t1]
    vw = np.zeros(case.p[t1], dtype=np.result_type(phi, np.float64))
    b = case.h[t1] + int(pz["begin"])
    cnt = int(pz["count"])
    vw[b:b + cnt] = (pz["A"] / pz["phi0"]) * phi * np.sin(2.0 * math.pi * pz["kappa"] * ax.xc[b:b + cnt])
    return t1, vw


def fill_halos(U, case, grid, phi=None, inflow=None):
    """Assign all halo cells of U in place.

    Order (this oracle's reading; the paper only says halo cells are assigned values): the x faces
    over the interior (y, z) range, then the y faces over all x and interior z, then the z faces
    over all (x, y).  Each later pass reads cells the earlier passes wrote, which defines the edge
    and corner halos needed by the cross-derivative terms of the viscous stress.
    """
    dt = U.dtype
    for a in range(case.ndim):
        n, h = case.n[a], case.h[a]
        # index ranges of the pass: axes before a in full, axes after a interior
        rng = []
        for b in range(3):
            if b < a:
                rng.append(slice(None))
            elif b > a:
                rng.append(slice(case.h[b], case.h[b] + case.n[b]))
            else:
                rng.append(None)
        for side in (0, 1):
            kind = case.bc[a][side]
            for m in range(h):
                g = h - 1 - m if side == 0 else h + n + m           # ghost layer (padded index)
                if kind == "periodic":
                    src = g + n if side == 0 else g - n
                elif kind == "zero_gradient":
                    src = h if side == 0 else h + n - 1
                else:
                    src = 2 * h - 1 - g if side == 0 else 2 * (h + n) - 1 - g   # mirror image
                idx_g = [slice(None)] + [None] * 3
                idx_s = [slice(None)] + [None] * 3
                for b in range(3):
                    idx_g[3 - b] = g if b == a else rng[b]
                    idx_s[3 - b] = src if b == a else rng[b]
                idx_g, idx_s = tuple(idx_g), tuple(idx_s)
                if kind in ("periodic", "zero_gradient"):
                    U[idx_g] = U[idx_s]
                    continue
                if kind == "inflow":
                    # Dirichlet: fixed primitive profile on the face plane, same in every layer
                    prof = inflow[(a, side)]                           # shape (5, ..tangential..)
                    tsl = tuple([slice(None)] + [rng[b] for b in (2, 1, 0) if b != a])
                    U[idx_g] = prim_to_cons(prof[tsl], case)
                    continue
                Wm, Tm = cons_to_prim(U[idx_s], case)
                Wg = Wm.copy()
                Wg[1:4] = -Wm[1:4]                                     # no-slip: mirror velocity
                if kind == "adiabatic":
                    U[idx_g] = prim_to_cons(Wg, case)
                    continue
                Tw = case.t_wall[a][side]
                Tg = 2.0 * Tw - Tm                                     # T = T_w at the wall face
                if np.any(_re(Tg) <= 0):
                    raise ValueError("isothermal mirror gives non-positive ghost temperature")
                Wg[0] = Wm[4] / (case.R * Tg)                          # p_g = p_m
                if kind == "porous":
                    pz = case.porous
                    if pz["axis"] != a or pz["side"] != side:
                        raise ValueError("porous strip is not on this face")
                    t1, vw = wall_velocity(case, grid, phi)
                    shp = [1, 1]
                    tang = [b for b in (2, 1, 0) if b != a]               # numpy order of tangential
                    vsel = vw[rng[t1]]
                    shp[tang.index(t1)] = vsel.size
                    Wg[1 + a] = 2.0 * vsel.reshape(shp) - Wm[1 + a]     # face normal velocity = v_w
                U[idx_g] = prim_to_cons(Wg, case)
    return U


# --------------------------------------------------------------------------------------------
# WENO5 reconstruction (Jiang & Shu 1996; Borges et al. 2008)
# --------------------------------------------------------------------------------------------
WENO_D = (0.1, 0.6, 0.3)


def weno5(qm2, qm1, q0, qp1, qp2, scheme, eps):
    """Left-biased value at face i+1/2 from the cell values q_{i-2} .. q_{i+2}.

    scheme 'linear' uses the optimal weights d_k (fifth-order upwind, for tests only).
    """
    p0 = (2.0 * qm2 - 7.0 * qm1 + 11.0 * q0) / 6.0
    p1 = (-qm1 + 5.0 * q0 + 2.0 * qp1) / 6.0
    p2 = (2.0 * q0 + 5.0 * qp1 - qp2) / 6.0
    b0 = (13.0 / 12.0) * (qm2 - 2.0 * qm1 + q0) ** 2 + 0.25 * (qm2 - 4.0 * qm1 + 3.0 * q0) ** 2
    b1 = (13.0 / 12.0) * (qm1 - 2.0 * q0 + qp1) ** 2 + 0.25 * (qm1 - qp1) ** 2
    b2 = (13.0 / 12.0) * (q0 - 2.0 * qp1 + qp2) ** 2 + 0.25 * (3.0 * q0 - 4.0 * qp1 + qp2) ** 2
    d0, d1, d2 = WENO_D
    if scheme == "linear":
        a0, a1, a2 = d0, d1, d2
    elif scheme == "js":
        a0 = d0 / (eps + b0) ** 2
        a1 = d1 / (eps + b1) ** 2
        a2 = d2 / (eps + b2) ** 2
    elif scheme == "z":
        tau5 = _abs(b0 - b2)
        a0 = d0 * (1.0 + (tau5 / (b0 + eps)) ** 2)
        a1 = d1 * (1.0 + (tau5 / (b1 + eps)) ** 2)
        a2 = d2 * (1.0 + (tau5 / (b2 + eps)) ** 2)
    else:
        raise ValueError(scheme)
    s = a0 + a1 + a2
    return (a0 * p0 + a1 * p1 + a2 * p2) / s


# --------------------------------------------------------------------------------------------
# HLLC approximate Riemann solver (Toro Ch. 10; paper Sec. 3.1 names HLLC)
# --------------------------------------------------------------------------------------------
def euler_flux(W, d, gamma):
    """Convective flux along axis d of Sec. 2.1 (F^c, G^c, H^c) from primitives."""
    rho, u, v, w, p = W
    vel = (u, v, w)
    un = vel[d]
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    F = [rho * un, rho * un * u, rho * un * v, rho * un * w, un * (E + p)]
    F[1 + d] = F[1 + d] + p
    return F, E


def roe_average(WL, WR, d, gamma):
    """sqrt(rho)-weighted (Roe) averages: velocity vector, total enthalpy H~ and sound speed c~."""
    g = gamma
    rL, pL = WL[0], WL[4]
    rR, pR = WR[0], WR[4]
    _, EL = euler_flux(WL, d, g)
    _, ER = euler_flux(WR, d, g)
    sqL, sqR = np.sqrt(rL), np.sqrt(rR)
    vt = [(sqL * WL[1 + c] + sqR * WR[1 + c]) / (sqL + sqR) for c in range(3)]
    HL = (EL + pL) / rL
    HR = (ER + pR) / rR
    Ht = (sqL * HL + sqR * HR) / (sqL + sqR)
    ct = np.sqrt((g - 1.0) * (Ht - 0.5 * (vt[0] ** 2 + vt[1] ** 2 + vt[2] ** 2)))
    return vt, Ht, ct


def hllc_parts(WL, WR, d, gamma):
    """Wave speeds, star states and fluxes of the HLLC solver along axis d (Toro Ch. 10).

    Wave speeds (reading; the paper is silent): Einfeldt bounds from Roe averages,
    S_L = min(u_L - c_L, u~ - c~), S_R = max(u_R + c_R, u~ + c~); contact speed
    S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R)) / (rho_L (S_L - u_L) - rho_R (S_R - u_R));
    star states U*_K = rho_K (S_K - u_K) / (S_K - S*) [1, S* (normal), tangential velocities,
    E_K / rho_K + (S* - u_K)(S* + p_K / (rho_K (S_K - u_K)))]; F*_K = F_K + S_K (U*_K - U_K).
    """
    g = gamma
    rL, pL = WL[0], WL[4]
    rR, pR = WR[0], WR[4]
    velL = (WL[1], WL[2], WL[3])
    velR = (WR[1], WR[2], WR[3])
    unL, unR = velL[d], velR[d]
    FL, EL = euler_flux(WL, d, g)
    FR, ER = euler_flux(WR, d, g)
    cL = np.sqrt(g * pL / rL)
    cR = np.sqrt(g * pR / rR)
    vt, _, ct = roe_average(WL, WR, d, g)
    SL = _min(unL - cL, vt[d] - ct)
    SR = _max(unR + cR, vt[d] + ct)
    Ss = (pR - pL + rL * unL * (SL - unL) - rR * unR * (SR - unR)) / (rL * (SL - unL) - rR * (SR - unR))

    def star(r, vel, un, p, E, S):
        fac = r * (S - un) / (S - Ss)
        Us = [fac, fac * vel[0], fac * vel[1], fac * vel[2],
              fac * (E / r + (Ss - un) * (Ss + p / (r * (S - un))))]
        Us[1 + d] = fac * Ss
        return Us

    UL = [rL, rL * velL[0], rL * velL[1], rL * velL[2], EL]
    UR = [rR, rR * velR[0], rR * velR[1], rR * velR[2], ER]
    with np.errstate(all="ignore"):                 # the unselected branches may divide by zero
        UsL = star(rL, velL, unL, pL, EL, SL)
        UsR = star(rR, velR, unR, pR, ER, SR)
        FsL = [FL[c] + SL * (UsL[c] - UL[c]) for c in range(NVAR)]
        FsR = [FR[c] + SR * (UsR[c] - UR[c]) for c in range(NVAR)]
    return dict(SL=SL, SR=SR, Ss=Ss, UL=UL, UR=UR, FL=FL, FR=FR, UsL=UsL, UsR=UsR, FsL=FsL, FsR=FsR)


def hllc_flux(WL, WR, d, gamma):
    """HLLC flux along axis d between left and right primitive states.
    Branch order (reading): S_L >= 0 -> F_L; S* >= 0 -> F*_L; S_R > 0 -> F*_R; else F_R."""
    h = hllc_parts(WL, WR, d, gamma)
    SLr, Ssr, SRr = _re(h["SL"]), _re(h["Ss"]), _re(h["SR"])
    out = []
    for c in range(NVAR):
        f = np.where(SLr >= 0, h["FL"][c],
                     np.where(Ssr >= 0, h["FsL"][c], np.where(SRr > 0, h["FsR"][c], h["FR"][c])))
        out.append(f)
    return out


# --------------------------------------------------------------------------------------------
# dissipative fluxes (Sec. 2.1: F^d, G^d, H^d; Newtonian stress, Fourier heat flux)
# --------------------------------------------------------------------------------------------
def _centre_derivative(f, a, grid, order=4):
    """Central derivative along axis a at every cell centre that has order/2 neighbours on both
    sides; other cells are left zero (they are never used).
      order 4: ((f_{j-2} - f_{j+2}) + 8 (f_{j+1} - f_{j-1})) / 12 * (d index/dx)_j
      order 6: (45 (f_{j+1} - f_{j-1}) - 9 (f_{j+2} - f_{j-2}) + (f_{j+3} - f_{j-3})) / 60 * (d index/dx)_j
    """
    out = np.zeros_like(f)
    pa = f.shape[2 - a]
    r = order // 2
    if pa < 2 * r + 1:
        return out
    s = lambda o: _sl(a, r + o, pa - r + o)
    mc = grid.along("mc", a)[s(0)]
    if order == 4:
        out[s(0)] = ((f[s(-2)] - f[s(2)]) + 8.0 * (f[s(1)] - f[s(-1)])) / 12.0 * mc
    else:
        out[s(0)] = (45.0 * (f[s(1)] - f[s(-1)]) - 9.0 * (f[s(2)] - f[s(-2)])
                     + (f[s(3)] - f[s(-3)])) / 60.0 * mc
    return out


def viscous_face_flux(W, T, case, grid, d):
    """F^d at every face a+1/2, a = h-1 .. h+n-1, along axis d, over all tangential cells.

    Reading (the paper uses "central finite-differences", Sec. 2.1, of sixth order in the channel
    computation, Sec. 3.1): case.visc_order 4 or 6,
      order 4: normal derivative ((f_{a-1} - f_{a+2}) + 27 (f_{a+1} - f_a)) / 24 * (d index/dx)_{a+1/2}
               face interpolation (9 (f_a + f_{a+1}) - (f_{a-1} + f_{a+2})) / 16
      order 6: normal derivative (2250 (f_{a+1} - f_a) - 125 (f_{a+2} - f_{a-1})
                                  + 9 (f_{a+3} - f_{a-2})) / 1920 * (d index/dx)_{a+1/2}
               face interpolation (150 (f_a + f_{a+1}) - 25 (f_{a-1} + f_{a+2}) + 3 (f_{a-2} + f_{a+3})) / 256
      tangential derivative: central derivative of the same order at the cell centres of the
      stencil, then face-interpolated.  mu = mu(T_face), lambda = mu c_p / Pr.
    Returns the five components (mass component zero) on faces a = h-1 .. h+n-1 (n+1 faces).
    """
    n, h = case.n[d], case.h[d]
    a0, a1 = h - 1, h + n                          # faces a+1/2 for a in [a0, a1)
    at = lambda f, o: f[_sl(d, a0 + o, a1 + o)]
    mf = grid.along("mf", d)[_sl(d, a0, a1)]
    order = case.visc_order
    if order == 4:
        interp = lambda f: (9.0 * (at(f, 0) + at(f, 1)) - (at(f, -1) + at(f, 2))) / 16.0
        dn = lambda f: ((at(f, -1) - at(f, 2)) + 27.0 * (at(f, 1) - at(f, 0))) / 24.0 * mf
    else:
        interp = lambda f: (150.0 * (at(f, 0) + at(f, 1)) - 25.0 * (at(f, -1) + at(f, 2))
                            + 3.0 * (at(f, -2) + at(f, 3))) / 256.0
        dn = lambda f: (2250.0 * (at(f, 1) - at(f, 0)) - 125.0 * (at(f, 2) - at(f, -1))
                        + 9.0 * (at(f, 3) - at(f, -2))) / 1920.0 * mf

    vel = [W[1], W[2], W[3]]
    vf = [interp(vel[c]) for c in range(3)]
    Tf = interp(T)
    # G[c][b] = d u_c / d x_b at the face
    zero = np.zeros_like(vf[0])
    G = [[zero] * 3 for _ in range(3)]
    for c in range(3):
        G[c][d] = dn(vel[c])
    for b in range(case.ndim):
        if b == d:
            continue
        G[d][b] = interp(_centre_derivative(vel[d], b, grid, order))     # d u_d / d x_b
        G[b][b] = interp(_centre_derivative(vel[b], b, grid, order))     # d u_b / d x_b
    div = G[0][0] + G[1][1] + G[2][2]
    mu = viscosity(Tf, case)
    lam = mu * case.cp / case.Pr
    tau = []
    for c in range(3):
        t = mu * (G[c][d] + G[d][c])
        if c == d:
            t = t - (2.0 / 3.0) * mu * div
        tau.append(t)
    energy = vf[0] * tau[0] + vf[1] * tau[1] + vf[2] * tau[2] + lam * dn(T)
    return [zero, tau[0], tau[1], tau[2], energy]


# --------------------------------------------------------------------------------------------
# right-hand side (Eq. ODE)
# --------------------------------------------------------------------------------------------
def convective_face_flux(W, case, d):
    """WENO5 (or TENO6-A) + HLLC flux at faces a+1/2, a = h-1 .. h+n-1, along axis d, over all
    tangential cells.  Reconstruction is component-wise on the primitive variables (reading; the
    paper is silent).  The right state at a+1/2 is the left-biased value of the mirrored stencil."""
    n, h = case.n[d], case.h[d]
    a0, a1 = h - 1, h + n
    sh = lambda o: _sl(d, a0 + o, a1 + o)
    WL, WR = [], []
    for c in range(NVAR):
        q = W[c]
        if case.weno == "teno6a":
            WL.append(teno.teno6a([q[sh(o)] for o in (-2, -1, 0, 1, 2, 3)]))
            WR.append(teno.teno6a([q[sh(o)] for o in (3, 2, 1, 0, -1, -2)]))
        else:
            WL.append(weno5(q[sh(-2)], q[sh(-1)], q[sh(0)], q[sh(1)], q[sh(2)], case.weno, case.weno_eps))
            WR.append(weno5(q[sh(3)], q[sh(2)], q[sh(1)], q[sh(0)], q[sh(-1)], case.weno, case.weno_eps))
    if case.weno == "teno6a":
        WL, WR = teno.limit_states(WL, WR, [W[c][sh(0)] for c in range(NVAR)],
                                   [W[c][sh(1)] for c in range(NVAR)])
    return hllc_flux(WL, WR, d, case.gamma)


def rhs_filled(U, case, grid):
    """R = dU/dt of Eq. ODE on the interior of U whose halos are already assigned.

    Returns an array shaped like U with the interior filled and the halos zero.
    """
    W, T = cons_to_prim(U, case)
    inner = case.interior()
    R = np.zeros_like(U)
    for d in range(case.ndim):
        Fc = convective_face_flux(W, case, d)
        if case.visc != "none":
            Fd = viscous_face_flux(W, T, case, grid, d)
            F = [Fc[c] - Fd[c] for c in range(NVAR)]
        else:
            F = Fc
        n = case.n[d]
        # restrict the tangential axes to the interior; along d keep the n+1 faces
        tsl = [inner[0], inner[1], inner[2]]
        tsl[2 - d] = slice(None)
        width = grid.along_inner("dx", d, case)
        for c in range(NVAR):
            Fi = F[c][tuple(tsl)]
            diff = Fi[_sl(d, 1, n + 1)] - Fi[_sl(d, 0, n)]
            R[c][inner] = R[c][inner] - diff / width
    f = case.body_force
    if any(v != 0.0 for v in f):
        u = W[1][inner], W[2][inner], W[3][inner]
        for c in range(3):
            R[1 + c][inner] = R[1 + c][inner] + f[c]
        R[4][inner] = R[4][inner] + (f[0] * u[0] + f[1] * u[1] + f[2] * u[2])
    return R


def rhs(U, case, grid, phi=None, inflow=None):
    """R = dU/dt (Eq. ODE) of the interior cells of U; U's halos are overwritten by the BCs."""
    fill_halos(U, case, grid, phi, inflow)
    return rhs_filled(U, case, grid)


# --------------------------------------------------------------------------------------------
# time step and TVD-RK3 (Sec. 2.1 names explicit TVD Runge-Kutta)
# --------------------------------------------------------------------------------------------
def cfl_dt(U, case, grid):
    """CFL time step (reading; the paper is silent):
    dt = CFL * min( min_{cells, axes} dx_d / (|u_d| + c),
                    min_{cells, axes} dx_d^2 / (2 max(4/3, gamma/Pr) mu / rho) )."""
    if case.dt_fixed > 0.0:
        return case.dt_fixed
    W, T = cons_to_prim(U, case)
    inner = case.interior()
    rho, p = W[0][inner], W[4][inner]
    c = np.sqrt(case.gamma * p / rho)
    best = math.inf
    for d in range(case.ndim):
        dx = grid.along_inner("dx", d, case)
        best = min(best, float(np.min(dx / (np.abs(W[1 + d][inner]) + c))))
        if case.visc != "none":
            nu = viscosity(T[inner], case) / rho
            k = 2.0 * max(4.0 / 3.0, case.gamma / case.Pr)
            best = min(best, float(np.min(dx * dx / (k * nu))))
    return case.cfl * best


def rk3(Un, dt, L, inner):
    """Shu-Osher TVD-RK3 (reading of Sec. 2.1's 'explicit TVD Runge-Kutta') for dU/dt = L(U):
    U1 = Un + dt L(Un); U2 = 3/4 Un + 1/4 (U1 + dt L(U1)); Un+1 = 1/3 Un + 2/3 (U2 + dt L(U2)).
    Only the entries selected by `inner` are advanced; L may overwrite the others (halos)."""
    Un = Un.copy()
    U1 = Un.copy()
    L0 = L(Un)
    U1[inner] = Un[inner] + dt * L0[inner]
    L1 = L(U1)
    U2 = U1.copy()
    U2[inner] = 0.75 * Un[inner] + 0.25 * (U1[inner] + dt * L1[inner])
    L2 = L(U2)
    U3 = U2.copy()
    U3[inner] = (1.0 / 3.0) * Un[inner] + (2.0 / 3.0) * (U2[inner] + dt * L2[inner])
    return U3


def rk3_step(U, dt, case, grid, phi=None, inflow=None):
    """One TVD-RK3 step of Eq. ODE with a fixed dt over the three stages; halos of the result are
    not assigned."""
    inner = (slice(None),) + case.interior()
    return rk3(U, dt, lambda V: rhs(V, case, grid, phi, inflow), inner)


def advance(U, case, grid, nsteps, t=0.0, t_end=math.inf, phi=None, inflow=None):
    """Run up to nsteps RK3 steps with the CFL (or fixed) dt; the last step is clipped so that t
    lands on t_end.  Returns (U, t, steps_taken)."""
    taken = 0
    for _ in range(nsteps):
        if t >= t_end:
            break
        dt = cfl_dt(U, case, grid)
        if t + dt > t_end:
            dt = t_end - t
        U = rk3_step(U, dt, case, grid, phi, inflow)
        t = t + dt if t + dt < t_end else t_end
        taken += 1
    return U, t, taken


# --------------------------------------------------------------------------------------------
# diagnostics
# --------------------------------------------------------------------------------------------
def kinetic_energy(U, case, grid):
    """Volume integral of rho |u|^2 / 2 over the interior."""
    inner = case.interior()
    m2 = U[1][inner] ** 2 + U[2][inner] ** 2 + U[3][inner] ** 2
    return np.sum(0.5 * m2 / U[0][inner] * grid.inner_volume(case))


def kinetic_energy_rate(U, R, case, grid):
    """d/dt of the kinetic-energy integral implied by R = dU/dt (chain rule on |m|^2 / (2 rho))."""
    inner = case.interior()
    rho = U[0][inner]
    u = [U[1 + c][inner] / rho for c in range(3)]
    rate = (u[0] * R[1][inner] + u[1] * R[2][inner] + u[2] * R[3][inner]
            - 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) * R[0][inner])
    return np.sum(rate * grid.inner_volume(case))


def wall_fluxes(U, case, grid, axis, side, phi=None, inflow=None):
    """Wall heat flux q_w = -lambda(T_face) dT/dn and wall shear mu(T_face) du_t/dn on the wall face
    (axis, side), from the fourth-order normal stencil across the wall with the halo values; the
    derivative is along +axis.  Returns (q_w, tau_w) over the wall cells of the face plane."""
    Uf = U.copy()
    fill_halos(Uf, case, grid, phi, inflow)
    W, T = cons_to_prim(Uf, case)
    h, n = case.h[axis], case.n[axis]
    a = h - 1 if side == 0 else h + n - 1              # face a+1/2 is the wall face
    mf = grid.axes[axis].mf[a]
    f = lambda q, o: q[_sl(axis, a + o, a + o + 1)]
    dn = lambda q: ((f(q, -1) - f(q, 2)) + 27.0 * (f(q, 1) - f(q, 0))) / 24.0 * mf
    interp = lambda q: (9.0 * (f(q, 0) + f(q, 1)) - (f(q, -1) + f(q, 2))) / 16.0
    Tf = interp(T)
    mu = viscosity(Tf, case)
    lam = mu * case.cp / case.Pr
    t1 = [b for b in range(case.ndim) if b != axis][0]
    inner = list(case.interior())
    inner[2 - axis] = slice(None)
    qw = (-lam * dn(T))[tuple(inner)]
    tw = (mu * dn(W[1 + t1]))[tuple(inner)]
    return qw, tw


def wall_heat_loss(U, case, grid, axis, side, phi=None, inflow=None):
    """J = sum_i q_w,i dx_i over the wall face (the integrated wall heat flux)."""
    qw, _ = wall_fluxes(U, case, grid, axis, side, phi, inflow)
    t1 = [b for b in range(case.ndim) if b != axis][0]
    inner = list(case.interior())
    inner[2 - axis] = slice(0, 1)
    area = 1.0
    for b in range(case.ndim):
        if b != axis:
            area = area * grid.along("dx", b)
    area = area[tuple(inner)] if not np.isscalar(area) else area
    return np.sum(qw * area)
