"""Plain fp64 oracle of the channel-flow reconstruction of the paper: TENO6-A with an interpolation
limiter (Sec. 3.1).

TEST INFRASTRUCTURE ONLY: the product path never imports this module.

The paper names the scheme and cites its solver for the definition; it prints no formula.  This
module writes the targeted ENO scheme out from its published definition (Fu, Hu & Adams 2016 for
TENO6; Fu, Hu & Adams 2017 for the adaptive cut-off "-A"), with every constant the paper leaves open
stated as a reading:

* Reconstruction of the left-biased value at face i+1/2 from the six cells i-2 .. i+3 on the
  uniform index grid (the same computational-space reading as WENO5).  Candidate stencils, in the
  TENO order of increasing width: S0 = (i-1, i, i+1), S1 = (i, i+1, i+2), S2 = (i-2, i-1, i),
  S3 = (i, i+1, i+2, i+3).  Each candidate value is that of the polynomial whose cell averages
  match the stencil.  The linear weights d_k are the ones for which sum_k d_k p_k is the value of
  the degree-5 polynomial of the full six-cell stencil (sixth-order linear scheme).
* Smoothness measures: Jiang & Shu's beta = sum_{l>=1} dx^(2l-1) int_{I_i} (d^l P / dx^l)^2 dx of
  each candidate polynomial P over the target cell I_i, and beta6 of the six-cell polynomial.
  tau6 = |beta6 - (beta1 + beta2 + 4 beta0) / 6| (the central stencil weighted four times).
* gamma_k = (1 + tau6 / (beta_k + eps))^6 with eps = 1e-40, chi_k = gamma_k / sum gamma; stencil k
  is kept (delta_k = 1) unless chi_k < C_T; omega_k = d_k delta_k / sum d_j delta_j and the value
  is sum omega_k p_k.
* Adaptive cut-off (TENO-A): the scale sensor of each cell j,
  eta_j = (2 |D_{j+1/2} D_{j-1/2}| + e) / (D_{j+1/2}^2 + D_{j-1/2}^2 + e), D_{j+1/2} = q_{j+1} - q_j,
  e = 0.9 C_r xi^2 / (1 - C_r); eta = min over the cells j = i-1 .. i+2 (every cell whose sensor the
  six-cell stencil determines); m = 1 - min(1, eta / C_r), g = (1 - m)^4 (1 + 4 m),
  betabar = alpha1 - alpha2 (1 - g), C_T = 10^(-floor(betabar)).  Constants (reading; the 2017
  paper's values for its five-point scheme): C_r = 0.25, xi = 1e-3, alpha1 = 10.5, alpha2 = 3.5, so
  C_T = 1e-10 in smooth regions and 1e-7 at discontinuities.
* Interpolation limiter (reading of "enhanced by an interpolation limiter"; the solver's
  positivity-preserving limiter of reconstructed states): when a reconstructed face state has
  rho <= 0 or p <= 0, all five primitives of that state fall back to the first-order value (the
  cell on that side of the face).

The coefficients of the candidates, the linear weights and the quadratic forms of the smoothness
measures are derived here, exactly in rational arithmetic, from the definitions above (cell-average
interpolation and the Jiang-Shu integral), not typed in.  Smoothness measures are evaluated on
differences from the stencil's first cell, which leaves them unchanged (they vanish on constants)
and avoids cancellation between large equal values.
"""
from fractions import Fraction as Fr

import numpy as np

TENO_Q = 6                 # exponent of gamma_k
TENO_C = 1.0               # constant of gamma_k
TENO_EPS = 1e-40
TENO_CR = 0.25
TENO_XI = 1e-3
TENO_ALPHA1 = 10.5
TENO_ALPHA2 = 3.5

# stencils of the left-biased value at i+1/2, as offsets from i
STENCILS = ((-1, 0, 1), (0, 1, 2), (-2, -1, 0), (0, 1, 2, 3))
FULL = (-2, -1, 0, 1, 2, 3)


# --------------------------------------------------------------------------------------------
# exact derivation of the coefficients (definitions written out in rational arithmetic)
# --------------------------------------------------------------------------------------------
def _solve(A, B):
    """Solve A X = B exactly (Gauss-Jordan on Fractions); A n x n, B n x m."""
    n = len(A)
    M = [list(A[r]) + list(B[r]) for r in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [row[n:] for row in M]


def _cell_average_matrix(offsets):
    """A[j][m] = average of x^m over the unit cell centred at offsets[j] (x from the centre of i)."""
    half = Fr(1, 2)
    return [[((o + half) ** (m + 1) - (o - half) ** (m + 1)) / (m + 1) for m in range(len(offsets))]
            for o in offsets]


def poly_coefficients(offsets):
    """C[m][j]: the polynomial P(x) = sum_m a_m x^m with unit-cell averages q_j on `offsets` has
    a_m = sum_j C[m][j] q_j."""
    n = len(offsets)
    eye = [[Fr(int(r == c)) for c in range(n)] for r in range(n)]
    return _solve(_cell_average_matrix(offsets), eye)


def face_value_weights(offsets, x=Fr(1, 2)):
    """v_j with P(x) = sum_j v_j q_j (the value at the right face of cell i by default)."""
    C = poly_coefficients(offsets)
    return [sum(C[m][j] * x ** m for m in range(len(offsets))) for j in range(len(offsets))]


def jiang_shu_matrix(offsets):
    """M with beta = sum_{j,k} M[j][k] q_j q_k = sum_{l>=1} int_{-1/2}^{1/2} (P^(l)(x))^2 dx (unit
    spacing: the dx^(2l-1) factors make beta independent of dx)."""
    n = len(offsets)
    C = poly_coefficients(offsets)
    half = Fr(1, 2)

    def integral(p):          # int_{-1/2}^{1/2} x^p dx
        return (half ** (p + 1) - (-half) ** (p + 1)) / (p + 1)

    M = [[Fr(0)] * n for _ in range(n)]
    for l in range(1, n):
        # l-th derivative: coefficient of x^(m-l) is a_m m!/(m-l)!
        D = []
        for m in range(l, n):
            f = Fr(1)
            for t in range(m - l + 1, m + 1):
                f *= t
            D.append((m - l, [f * C[m][j] for j in range(n)]))
        for pa, ca in D:
            for pb, cb in D:
                w = integral(pa + pb)
                if w == 0:
                    continue
                for j in range(n):
                    for k in range(n):
                        M[j][k] += w * ca[j] * cb[k]
    return M


def linear_weights():
    """d_k such that sum_k d_k p_k equals the six-cell value for all data (unique)."""
    full = face_value_weights(FULL)
    # unknowns d0..d3; one equation per cell of the full stencil
    cand = [face_value_weights(s) for s in STENCILS]
    rows = []
    rhs = []
    for j, o in enumerate(FULL):
        rows.append([cand[k][s.index(o)] if o in s else Fr(0) for k, s in enumerate(STENCILS)])
        rhs.append([full[j]])
    # six equations, four unknowns: solve the first four independent ones, check the rest
    d = _solve([rows[i] for i in (0, 1, 4, 5)], [rhs[i] for i in (0, 1, 4, 5)])
    d = [r[0] for r in d]
    for row, r in zip(rows, rhs):
        assert sum(a * b for a, b in zip(row, d)) == r[0]
    return d


CAND = [face_value_weights(s) for s in STENCILS]
FULL_VALUE = face_value_weights(FULL)
D_LIN = linear_weights()
BETA_M = [jiang_shu_matrix(s) for s in STENCILS]
BETA6_M = jiang_shu_matrix(FULL)


def _quad(M, qs):
    """sum_{j,k} M[j][k] d_j d_k with d_j = q_j - q_0 (M annihilates constants)."""
    ds = [q - qs[0] for q in qs]
    out = 0.0
    for j in range(len(qs)):
        for k in range(len(qs)):
            if M[j][k] != 0:
                out = out + float(M[j][k]) * ds[j] * ds[k]
    return out


def _lin(v, qs):
    out = 0.0
    for w, q in zip(v, qs):
        out = out + float(w) * q
    return out


# --------------------------------------------------------------------------------------------
# TENO6-A
# --------------------------------------------------------------------------------------------
def cutoff(q):
    """Adaptive C_T of the stencil q = (q_{i-2}, ..., q_{i+3}) (arrays broadcast)."""
    e = 0.9 * TENO_CR * TENO_XI ** 2 / (1.0 - TENO_CR)
    eta = None
    for j in range(1, 5):                      # cells i-1 .. i+2
        dp = q[j + 1] - q[j]
        dm = q[j] - q[j - 1]
        ej = (2.0 * np.abs(dp * dm) + e) / (dp * dp + dm * dm + e)
        eta = ej if eta is None else np.minimum(eta, ej)
    m = 1.0 - np.minimum(1.0, eta / TENO_CR)
    g = (1.0 - m) ** 4 * (1.0 + 4.0 * m)
    betabar = TENO_ALPHA1 - TENO_ALPHA2 * (1.0 - g)
    return 10.0 ** (-np.floor(betabar))


def teno6a_parts(q):
    """Candidate values p_k, smoothness measures beta_k, beta6 and the kept-stencil flags delta_k of
    the left-biased value at i+1/2 from q = (q_{i-2}, ..., q_{i+3})."""
    sub = lambda s: [q[o + 2] for o in s]
    p = [_lin(CAND[k], sub(s)) for k, s in enumerate(STENCILS)]
    beta = [_quad(BETA_M[k], sub(s)) for k, s in enumerate(STENCILS)]
    beta6 = _quad(BETA6_M, list(q))
    tau = np.abs(beta6 - (beta[1] + beta[2] + 4.0 * beta[0]) / 6.0)
    gam = [(TENO_C + tau / (b + TENO_EPS)) ** TENO_Q for b in beta]
    tot = gam[0] + gam[1] + gam[2] + gam[3]
    ct = cutoff(q)
    delta = [np.logical_not(g / tot < ct) for g in gam]
    return p, beta, beta6, delta


def teno6a(q):
    """Left-biased TENO6-A value at face i+1/2 from q = (q_{i-2}, ..., q_{i+3})."""
    p, _, _, delta = teno6a_parts(q)
    num = 0.0
    den = 0.0
    for k in range(4):
        w = float(D_LIN[k]) * delta[k]
        num = num + w * p[k]
        den = den + w
    return num / den


def limit_states(WL, WR, W_left_cell, W_right_cell):
    """Interpolation limiter: a face state with rho <= 0 or p <= 0 takes the first-order value of
    the cell on its side (all five primitives).  Arguments are lists of five arrays; returns new
    lists."""
    badL = (WL[0] <= 0.0) | (WL[4] <= 0.0)
    badR = (WR[0] <= 0.0) | (WR[4] <= 0.0)
    L = [np.where(badL, W_left_cell[c], WL[c]) for c in range(5)]
    R = [np.where(badR, W_right_cell[c], WR[c]) for c in range(5)]
    return L, R
