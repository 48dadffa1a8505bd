"""Pins of the compressible boundary-layer similarity solution (workloads.similarity_bl), the inlet
profile and reference of Section 3.2's laminar boundary-layer validation, against what the
mathematics fixes: the Blasius wall shear in the incompressible limit, the Crocco-Busemann
relations for Pr = 1 and C = 1 (adiabatic and isothermal walls), the laminar recovery factor
close to sqrt(Pr), Chapman-Rubesin decoupling, and mass conservation of the self-similar field
(which pins the wall-normal velocity derived from the stream function)."""
import math

import numpy as np
import pytest

from paper_2406_19494_gb300 import workloads as wl

GM = lambda Ma, gamma=1.4: (gamma - 1.0) * Ma * Ma


def test_incompressible_limit_is_blasius():
    """Ma -> 0 with an adiabatic wall: g = 1, C = 1, so f''' + f f'' = 0; in the variable
    eta = y sqrt(U / (2 nu x)) the Blasius wall value is f''(0) = 0.469600 and f' -> 1."""
    s = wl.similarity_bl(1e-4, 0.72, suth=0.368)
    assert s["fpp"][0] == pytest.approx(0.469600, abs=2e-6)
    assert np.max(np.abs(s["g"] - 1.0)) < 1e-7
    # displacement: eta - f(eta) -> 1.2168 (the Blasius displacement thickness in this variable)
    assert s["eta"][-1] - s["f"][-1] == pytest.approx(1.21678, abs=2e-4)


def test_crocco_busemann_adiabatic_pr1():
    """Pr = 1, C = 1, adiabatic wall: g = 1 + (gamma - 1)/2 Ma^2 (1 - f'^2) exactly, so the wall
    temperature is the stagnation temperature."""
    Ma = 2.25
    s = wl.similarity_bl(Ma, 1.0)
    m = 0.5 * GM(Ma)
    assert np.max(np.abs(s["g"] - (1.0 + m * (1.0 - s["fp"] ** 2)))) < 1e-9
    assert s["g"][0] == pytest.approx(1.0 + m, rel=1e-10)


def test_crocco_relation_isothermal_pr1():
    """Pr = 1, C = 1, wall at g_w: g = g_w + (1 + m - g_w) f' - m f'^2, m = (gamma - 1)/2 Ma^2."""
    Ma, gw = 6.0, 4.0
    s = wl.similarity_bl(Ma, 1.0, wall="isothermal", g_wall=gw)
    m = 0.5 * GM(Ma)
    assert np.max(np.abs(s["g"] - (gw + (1.0 + m - gw) * s["fp"] - m * s["fp"] ** 2))) < 1e-8


def test_chapman_rubesin_decouples_and_recovery_factor():
    """C = 1: the momentum equation does not see the temperature, f''(0) = 0.4696 at any Mach
    number; the adiabatic wall recovers r = (g_w - 1) / ((gamma - 1)/2 Ma^2) close to sqrt(Pr)
    (the laminar flat-plate recovery factor, Pr = 0.72)."""
    Ma = 2.25
    s = wl.similarity_bl(Ma, 0.72)
    assert s["fpp"][0] == pytest.approx(0.469600, abs=2e-6)
    r = (s["g"][0] - 1.0) / (0.5 * GM(Ma))
    assert r == pytest.approx(math.sqrt(0.72), rel=3e-3)


def test_sutherland_boundary_layer_is_heated_and_thickened():
    """The Ma 2.25 adiabatic wall with Sutherland viscosity: heated to g_w between 1.7 and 2, and the
    wall shear satisfies the integrated momentum equation C_w f''(0) = int f f'' d eta."""
    c = wl.e2_case()
    s = wl.e2_similarity(c)
    C = lambda g: np.sqrt(g) * (1 + c["suth_S"]) / (g + c["suth_S"])
    assert 1.7 < s["g"][0] < 2.0
    # momentum balance integrated across the layer: C_w f''(0) = int_0^inf f f'' (from (C f'')' = -f f'')
    rhs = np.trapezoid(s["f"] * s["fpp"], s["eta"])
    assert C(s["g"][0]) * s["fpp"][0] == pytest.approx(rhs, rel=1e-5)


def test_self_similar_field_conserves_mass():
    """d(rho u)/dx + d(rho v)/dy = 0 for the field built from the similarity solution (central
    differences at x = 1.25 on a fine grid; the tabulated profile is interpolated linearly, which
    leaves a residual of a few 1e-4 of the terms): pins the wall-normal velocity
    v = (f' Y - g f) / sqrt(2 Re_x) and the mapping of eta to y (v = 0, or a wrong sign in v, leaves
    a residual of the size of the terms)."""
    c = wl.e2_case()
    s = wl.e2_similarity(c)
    y = np.linspace(1e-4, 0.2, 4001)
    hx, hy = 1e-2, y[1] - y[0]
    W = wl.similarity_field(c, s, np.array([1.25 - hx, 1.25, 1.25 + hx]), y)[:, 0]
    mu = W[0] * W[1]
    mv = W[0] * W[2]
    dmu_dx = (mu[:, 2] - mu[:, 0]) / (2 * hx)
    dmv_dy = np.gradient(mv[:, 1], hy)
    scale = np.max(np.abs(dmu_dx))
    assert np.max(np.abs((dmu_dx + dmv_dy)[5:-5])) < 2e-3 * scale
    assert abs(W[1, 0, 1]) < 1e-2 and W[1, -1, 1] == pytest.approx(1.0, abs=1e-6)
