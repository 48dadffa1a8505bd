"""Exact solution of the Riemann problem of the 1-D Euler equations for an ideal gas.

TEST INFRASTRUCTURE ONLY: used to pin the oracle on the Sod shock tube (the shock-tube validation
named for the WENO5 + HLLC + TVD-RK3 configuration); the product path never imports it.

Method (textbook: the star-region pressure p* is the root of f_L(p) + f_R(p) + u_R - u_L = 0, where
f_K is the shock (Rankine-Hugoniot) branch for p > p_K and the rarefaction (isentropic) branch for
p <= p_K; the root is found by Newton iteration from the two-rarefaction guess, then the self-similar
solution is sampled at x/t).
"""
import math


def _fK(p, rhoK, pK, g):
    """Pressure function f_K and its derivative for one side."""
    cK = math.sqrt(g * pK / rhoK)
    if p > pK:                                  # shock
        A = 2.0 / ((g + 1.0) * rhoK)
        B = (g - 1.0) / (g + 1.0) * pK
        s = math.sqrt(A / (p + B))
        return (p - pK) * s, s * (1.0 - 0.5 * (p - pK) / (B + p))
    # rarefaction
    e = (g - 1.0) / (2.0 * g)
    f = 2.0 * cK / (g - 1.0) * ((p / pK) ** e - 1.0)
    df = (p / pK) ** (-(g + 1.0) / (2.0 * g)) / (rhoK * cK)
    return f, df


def star_state(left, right, g=1.4, tol=1e-14, maxit=100):
    """(p*, u*) for left = (rho, u, p) and right = (rho, u, p)."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    e = (g - 1.0) / (2.0 * g)
    # two-rarefaction initial guess
    p = ((cL + cR - 0.5 * (g - 1.0) * (uR - uL)) / (cL / pL ** e + cR / pR ** e)) ** (1.0 / e)
    p = max(p, 1e-12)
    for _ in range(maxit):
        fl, dl = _fK(p, rL, pL, g)
        fr, dr = _fK(p, rR, pR, g)
        dp = (fl + fr + uR - uL) / (dl + dr)
        pn = max(p - dp, 1e-14)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fK(p, rL, pL, g)
    fr, _ = _fK(p, rR, pR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, s, g=1.4):
    """(rho, u, p) of the self-similar solution at speed s = x / t."""
    rL, uL, pL = left
    rR, uR, pR = right
    ps, us = star_state(left, right, g)
    gm, gp = g - 1.0, g + 1.0
    if s <= us:                                  # left of the contact
        cL = math.sqrt(g * pL / rL)
        if ps > pL:                              # left shock
            SL = uL - cL * math.sqrt(gp / (2 * g) * ps / pL + gm / (2 * g))
            if s <= SL:
                return rL, uL, pL
            r = rL * (ps / pL + gm / gp) / (gm / gp * ps / pL + 1.0)
            return r, us, ps
        cs = cL * (ps / pL) ** (gm / (2 * g))
        if s <= uL - cL:
            return rL, uL, pL
        if s >= us - cs:
            return rL * (ps / pL) ** (1.0 / g), us, ps
        u = 2.0 / gp * (cL + gm / 2.0 * uL + s)
        c = 2.0 / gp * (cL + gm / 2.0 * (uL - s))
        r = rL * (c / cL) ** (2.0 / gm)
        return r, u, pL * (c / cL) ** (2.0 * g / gm)
    cR = math.sqrt(g * pR / rR)
    if ps > pR:                                  # right shock
        SR = uR + cR * math.sqrt(gp / (2 * g) * ps / pR + gm / (2 * g))
        if s >= SR:
            return rR, uR, pR
        r = rR * (ps / pR + gm / gp) / (gm / gp * ps / pR + 1.0)
        return r, us, ps
    cs = cR * (ps / pR) ** (gm / (2 * g))
    if s >= uR + cR:
        return rR, uR, pR
    if s <= us + cs:
        return rR * (ps / pR) ** (1.0 / g), us, ps
    u = 2.0 / gp * (-cR + gm / 2.0 * uR + s)
    c = 2.0 / gp * (cR - gm / 2.0 * (uR - s))
    r = rR * (c / cR) ** (2.0 / gm)
    return r, u, pR * (c / cR) ** (2.0 * g / gm)


def shock_speed(left, right, g=1.4):
    """Speed of the right-moving shock (for a problem with p* > p_R)."""
    ps, _ = star_state(left, right, g)
    rR, uR, pR = right
    cR = math.sqrt(g * pR / rR)
    return uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))


def cell_averages(left, right, x0, t, xf, g=1.4, nsub=64):
    """Cell averages of (rho, u, p) on cells with face coordinates xf (midpoint sub-sampling)."""
    import numpy as np
    n = len(xf) - 1
    out = np.zeros((3, n))
    for i in range(n):
        xs = xf[i] + (np.arange(nsub) + 0.5) / nsub * (xf[i + 1] - xf[i])
        vals = np.array([sample(left, right, (x - x0) / t, g) for x in xs])
        out[:, i] = vals.mean(axis=0)
    return out
