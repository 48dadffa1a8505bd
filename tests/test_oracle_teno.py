"""Pins of the TENO6-A reconstruction and the sixth-order dissipative stencils of the oracle
(the paper's channel scheme, Sec. 3.1) against the mathematics that fixes them: exact
polynomial reproduction, the textbook WENO5 and sixth-order central formulas, the Jiang-Shu
integral evaluated by quadrature, convergence order, the ENO property and the cut-off values."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from conftest import read_golden
from helpers import padded_state
from oracle import ns_fv as nf
from oracle import teno
from paper_2406_19494_gb300 import workloads as wl

GL_X, GL_W = np.polynomial.legendre.leggauss(12)        # exact for degree <= 23 on [-1, 1]


def cell_average(f, o):
    """Average of f over the unit cell centred at o, by Gauss-Legendre quadrature."""
    x = o + 0.5 * GL_X
    return 0.5 * np.sum(GL_W * f(x))


def test_derivation_reproduces_the_weno5_textbook_formulas():
    # candidates of the three-point stencils are WENO5's (Jiang & Shu): S0 is WENO5's p1, S1 its
    # p2 and S2 its p0
    assert teno.CAND[0] == [Fr(-1, 6), Fr(5, 6), Fr(1, 3)]
    assert teno.CAND[1] == [Fr(1, 3), Fr(5, 6), Fr(-1, 6)]
    assert teno.CAND[2] == [Fr(1, 3), Fr(-7, 6), Fr(11, 6)]

    # smoothness measures are WENO5's 13/12 t^2 + 1/4 s^2 forms, expanded into quadratic forms
    def form(t, s):
        return [[Fr(13, 12) * t[j] * t[k] + Fr(1, 4) * s[j] * s[k] for k in range(3)] for j in range(3)]
    assert teno.BETA_M[0] == form((1, -2, 1), (1, 0, -1))
    assert teno.BETA_M[1] == form((1, -2, 1), (3, -4, 1))
    assert teno.BETA_M[2] == form((1, -2, 1), (1, -4, 3))


def test_linear_weights_give_the_sixth_order_central_value():
    # textbook sixth-order value at i+1/2 from cell averages: (1, -8, 37, 37, -8, 1) / 60
    assert teno.FULL_VALUE == [Fr(v, 60) for v in (1, -8, 37, 37, -8, 1)]
    d = teno.D_LIN
    assert sum(d) == 1 and all(x > 0 for x in d)
    for j, o in enumerate(teno.FULL):
        comb = sum(d[k] * teno.CAND[k][s.index(o)] for k, s in enumerate(teno.STENCILS) if o in s)
        assert comb == teno.FULL_VALUE[j]


@pytest.mark.parametrize("k", range(5))
def test_candidates_reproduce_polynomials(k):
    # cell averages (by quadrature) of a polynomial of degree <= stencil size - 1 give its exact
    # value at the face x = 1/2
    rng = np.random.default_rng(k)
    stencils = list(teno.STENCILS) + [teno.FULL]
    weights = list(teno.CAND) + [teno.FULL_VALUE]
    s, v = stencils[k], weights[k]
    c = rng.normal(size=len(s))
    f = lambda x: np.polyval(c, x)
    q = [cell_average(f, o) for o in s]
    got = sum(float(w) * qq for w, qq in zip(v, q))
    assert abs(got - f(0.5)) < 1e-13 * max(1.0, abs(f(0.5)))


@pytest.mark.parametrize("k", range(5))
def test_smoothness_measures_match_the_jiang_shu_integral(k):
    # beta from the rational quadratic form vs. a numerical evaluation of its definition: fit the
    # polynomial to quadrature cell averages, then integrate the squared derivatives by quadrature
    rng = np.random.default_rng(10 + k)
    stencils = list(teno.STENCILS) + [teno.FULL]
    mats = list(teno.BETA_M) + [teno.BETA6_M]
    s, M = stencils[k], mats[k]
    n = len(s)
    q = rng.normal(size=n)
    A = np.array([[cell_average(lambda x, m=m: x ** m, o) for m in range(n)] for o in s])
    a = np.linalg.solve(A, q)                     # P(x) = sum a_m x^m
    P = np.polynomial.Polynomial(a)
    beta = 0.0
    for l in range(1, n):
        dP = P.deriv(l)
        beta += 0.5 * np.sum(GL_W * dP(0.5 * GL_X) ** 2)
    got = teno._quad(M, list(q))
    assert abs(got - beta) < 1e-11 * max(1.0, beta)


def test_teno_worked_examples():
    for name, *rest in read_golden("teno6a_worked_examples.txt"):
        q = [float(x) for x in rest[:6]]
        expected, tol = float(rest[6]), float(rest[7])
        got = teno.teno6a([np.array(x) for x in q])
        assert abs(got - expected) <= tol, (name, got)


def test_teno_smooth_data_keeps_every_stencil_and_converges_at_sixth_order():
    errs = []
    for n in (32, 64):
        h = 2 * np.pi / n
        x = np.arange(n) * h
        qbar = (np.cos(x - h / 2) - np.cos(x + h / 2)) / h       # exact cell averages of sin
        st = [np.roll(qbar, -o) for o in (-2, -1, 0, 1, 2, 3)]
        _, _, _, delta = teno.teno6a_parts(st)
        assert all(np.all(d) for d in delta)
        assert np.all(teno.cutoff(st) == 1e-10)
        val = teno.teno6a(st)
        errs.append(np.max(np.abs(val - np.sin(x + h / 2))))
    order = np.log2(errs[0] / errs[1])
    assert order > 5.7, order


def test_teno_cuts_stencils_across_a_jump_and_does_not_overshoot():
    q = np.array([1.0, 1.0, 1.0, 1.0, 0.2, 0.2, 0.2, 0.2, 0.2])
    vals = []
    for i in range(2, 6):
        st = [np.array(q[i + o]) for o in (-2, -1, 0, 1, 2, 3)]
        p, beta, beta6, delta = teno.teno6a_parts(st)
        # every stencil that crosses the jump (between cells 3 and 4) is cut
        for k, s in enumerate(teno.STENCILS):
            cells = [i + o for o in s]
            crosses = min(cells) <= 3 < max(cells)
            if crosses:
                assert not delta[k], (i, k)
        assert teno.cutoff(st) == 1e-7
        vals.append(float(teno.teno6a(st)))
    assert all(0.2 - 1e-15 <= v <= 1.0 + 1e-15 for v in vals), vals


def test_interpolation_limiter_falls_back_to_the_cell_values():
    WL = [np.array([1.0, -0.1]), np.array([0.1, 0.2]), np.zeros(2), np.zeros(2), np.array([1.0, 1.0])]
    WR = [np.array([1.0, 1.0]), np.array([0.3, 0.4]), np.zeros(2), np.zeros(2), np.array([-1e-3, 2.0])]
    cl = [np.full(2, 7.0)] * 5
    cr = [np.full(2, 9.0)] * 5
    L, R = teno.limit_states(WL, WR, cl, cr)
    # left state of face 1 has rho < 0, right state of face 0 has p < 0: those fall back
    assert [x[1] for x in L] == [7.0] * 5 and [x[0] for x in L] == [1.0, 0.1, 0.0, 0.0, 1.0]
    assert [x[0] for x in R] == [9.0] * 5 and [x[1] for x in R] == [1.0, 0.4, 0.0, 0.0, 2.0]


def test_sixth_order_central_stencils_are_exact_for_quintics():
    # a 1-D velocity field u(x) = quintic, T uniform: the face stress tau_xx = (4/3) mu u'(x_f) and
    # the centre derivative of the sixth-order stencils are exact
    d = wl.tgv_case(12)
    d.update(visc="constant", mu_ref=0.01, visc_order=6)
    case = nf.Case(d)
    grid = nf.Grid(case)
    xc = grid.along("xc", 0).ravel()
    rng = np.random.default_rng(3)
    c = rng.normal(size=6) * 0.05
    u = np.polyval(c, xc)[None, None, :] * np.ones(case.shape[1:])
    W = np.zeros(case.shape)
    W[0] = 1.0
    W[1] = u
    W[4] = 1.0
    T = np.ones(case.shape[1:])
    Fd = nf.viscous_face_flux(W, T, case, grid, 0)
    h = case.h[0]
    xf = [0.5 * (xc[a] + xc[a + 1]) for a in range(h - 1, h + case.n[0])]
    du = np.polyval(np.polyder(c), np.array(xf))
    assert np.allclose(Fd[1][0, 0, :], (4.0 / 3.0) * 0.01 * du, rtol=0, atol=1e-14)
    # centre derivative along y of a field varying along y (degree 6: exact)
    c6 = rng.normal(size=7) * 0.02
    yc = grid.along("xc", 1).ravel()
    f = np.polyval(c6, yc)[None, :, None] * np.ones(case.shape[1:])
    g = nf._centre_derivative(f, 1, grid, 6)
    j = slice(3, case.p[1] - 3)
    assert np.allclose(g[0, j, 0], np.polyval(np.polyder(c6), yc[j]), rtol=1e-12, atol=1e-12)


def _teno_case(n=12, **kw):
    d = wl.tgv_case(n)
    d.update(weno="teno6a", visc_order=6, **kw)
    return d


def test_teno_rhs_conserves_on_a_periodic_box():
    case, grid, U = padded_state(_teno_case(), seed=4)
    R = nf.rhs(U, case, grid)
    inner = case.interior()
    vol = grid.inner_volume(case)
    for v in range(5):
        tot = np.sum(R[v][inner] * vol)
        scale = np.sum(np.abs(R[v][inner]) * vol)
        assert abs(tot) <= 1e-13 * scale, (v, tot, scale)


def test_teno_preserves_a_free_stream_on_a_stretched_grid():
    d = wl.channel_case(nx=8, ny=16, nz=8)
    d.update(weno="teno6a", visc_order=6, bc=(("periodic",) * 2, ("zero_gradient",) * 2, ("periodic",) * 2),
             body_force=(0.0, 0.0, 0.0))
    case, grid, U = padded_state(d, uniform=(1.2, 0.7, -0.1, 0.3, 0.5))
    R = nf.rhs(U, case, grid)
    assert np.max(np.abs(R[(slice(None),) + case.interior()])) < 1e-13


def test_tau6_is_of_higher_order_than_the_smoothness_measures():
    # on smooth data beta_k ~ h^2 while tau6 = |beta6 - (beta1 + beta2 + 4 beta0) / 6| cancels the
    # h^2 and h^4 terms, so gamma_k -> 1 as h -> 0 (the targeting property): tau6 falls by at
    # least 2^5 per halving of h, a beta by 2^2
    taus, betas = [], []
    for n in (64, 128):
        h = 2 * np.pi / n
        x = np.arange(n) * h
        qbar = (np.cos(x - h / 2) - np.cos(x + h / 2)) / h
        st = [np.roll(qbar, -o) for o in (-2, -1, 0, 1, 2, 3)]
        _, beta, beta6, _ = teno.teno6a_parts(st)
        tau = np.abs(beta6 - (beta[1] + beta[2] + 4.0 * beta[0]) / 6.0)
        # points where the leading terms do not vanish (away from the extrema of sin')
        sel = np.abs(np.cos(x)) > 0.5
        taus.append(np.median(tau[sel]))
        betas.append(np.median(beta[0][sel]))
    assert np.log2(betas[0] / betas[1]) == pytest.approx(2.0, abs=0.1)
    assert np.log2(taus[0] / taus[1]) > 5.0, np.log2(taus[0] / taus[1])
