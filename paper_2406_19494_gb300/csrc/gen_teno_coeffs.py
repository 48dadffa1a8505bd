"""Write teno_coeffs.cuh: the rational coefficients of the TENO6 smoothness measures used by the
FP64 kernels, derived symbolically (sympy) from the Jiang-Shu definition.

Not part of the build: the generated header is committed, and this script re-creates it (needs
sympy, available on the development machine only).  Run from this directory:
    python gen_teno_coeffs.py > teno_coeffs.cuh

For a stencil of cells with unit width centred at the integer offsets s (x measured from the centre
of the target cell), the reconstruction polynomial P has the stencil's cell averages, and
beta = sum_{l >= 1} int_{-1/2}^{1/2} (P^(l))^2 dx.  beta vanishes on constants, so it is written as
a quadratic form in the consecutive cell differences of the stencil (the marching kernel carries
them from face to face); the six-cell measures of a window and of its mirror image are emitted as
one pair.  Every emitted form is checked here, exactly, against the definition.  The header also
holds the adaptive cut-off of TENO-A as thresholds on the scale sensor.
"""
import sympy as sp


def beta_matrix(offsets):
    """Symmetric matrix A with beta = q^T A q over the stencil's cell values q (A annihilates
    constants)."""
    x = sp.symbols("x")
    n = len(offsets)
    a = sp.symbols("a0:%d" % n)
    q = sp.symbols("q0:%d" % n)
    P = sum(a[m] * x ** m for m in range(n))
    eqs = [sp.integrate(P, (x, o - sp.Rational(1, 2), o + sp.Rational(1, 2))) - q[j]
           for j, o in enumerate(offsets)]
    Pq = P.subs(sp.solve(eqs, a, dict=True)[0])
    beta = sp.expand(sum(sp.integrate(sp.diff(Pq, x, l) ** 2, (x, -sp.Rational(1, 2), sp.Rational(1, 2)))
                         for l in range(1, n)))
    return sp.Matrix(n, n, lambda i, j: sp.Rational(1, 2) * sp.diff(beta, q[i], q[j])), q, beta


def emit_diff_forms():
    """The four-cell measure and the paired six-cell measures written in the consecutive cell
    differences d_j = q_{j+1} - q_j of the six-cell window q[0..5] (d[0..4]), the form the marching
    kernel carries (one new difference per face).
      * beta4 of cells (0, 1, 2, 3) around target 0 is a form Q in (d_0, d_1, d_2) of those cells;
        the left state's is Q(d2, d3, d4), the right state's (mirror image, cells q3, q2, q1, q0)
        Q(d2, d1, d0) (a quadratic form is even, so the signs of the mirrored differences drop).
      * the reversal of the window maps d_j to -d_{4-j}; with the even combinations
        u0 = d0 + d4, u1 = d1 + d3, u2 = d2 and the odd ones w0 = d0 - d4, w1 = d1 - d3,
        6 beta6 of the window is S + T + 2 X and of its mirror S + T - 2 X (S a form in u, T in w,
        X bilinear).  Both are checked exactly against the row forms above."""
    # beta4 in consecutive differences
    A, q, beta = beta_matrix((0, 1, 2, 3))
    d = sp.symbols("d0:3")
    sub = {q[0]: 0, q[1]: d[0], q[2]: d[0] + d[1], q[3]: d[0] + d[1] + d[2]}
    b4 = sp.expand(beta.subs(sub, simultaneous=True))
    P4 = sp.Poly(b4, *d)
    c4 = {(i, j): P4.coeff_monomial(tuple(int(k == i) + int(k == j) for k in range(3)))
          for i in range(3) for j in range(i, 3)}
    # paired beta6 in consecutive differences
    A6, q6, beta6 = beta_matrix((-2, -1, 0, 1, 2, 3))
    dd = sp.symbols("e0:5")
    sub6 = {q6[0]: 0}
    acc = 0
    for j in range(5):
        acc = acc + dd[j]
        sub6[q6[j + 1]] = acc
    bL = sp.expand(6 * beta6.subs(sub6, simultaneous=True))
    rev = {dd[j]: -dd[4 - j] for j in range(5)}
    bR = sp.expand(bL.subs(rev, simultaneous=True))
    u0, u1, u2, w0, w1 = sp.symbols("u0 u1 u2 w0 w1")
    inv = {dd[0]: (u0 + w0) / 2, dd[4]: (u0 - w0) / 2, dd[1]: (u1 + w1) / 2, dd[3]: (u1 - w1) / 2, dd[2]: u2}
    even = sp.expand(((bL + bR) / 2).subs(inv, simultaneous=True))
    odd = sp.expand(((bL - bR) / 4).subs(inv, simultaneous=True))      # X, with bL = S + T + 2 X
    PE = sp.Poly(even, u0, u1, u2, w0, w1)
    PO = sp.Poly(odd, u0, u1, u2, w0, w1)
    mono = lambda **k: tuple(k.get(n, 0) for n in ("u0", "u1", "u2", "w0", "w1"))
    S = {}
    for i, a in enumerate(("u0", "u1", "u2")):
        for b in ("u0", "u1", "u2")[i:]:
            m = {a: 1}
            m[b] = m.get(b, 0) + 1
            S[(a, b)] = PE.coeff_monomial(mono(**m))
    T = {("w0", "w0"): PE.coeff_monomial(mono(w0=2)), ("w0", "w1"): PE.coeff_monomial(mono(w0=1, w1=1)),
         ("w1", "w1"): PE.coeff_monomial(mono(w1=2))}
    X = {(a, b): PO.coeff_monomial(mono(**{a: 1, b: 1})) for a in ("u0", "u1", "u2") for b in ("w0", "w1")}
    # exact checks against the definitions
    Sv = sum(c * sp.Symbol(a) * sp.Symbol(b) for (a, b), c in S.items())
    Tv = sum(c * sp.Symbol(a) * sp.Symbol(b) for (a, b), c in T.items())
    Xv = sum(c * sp.Symbol(a) * sp.Symbol(b) for (a, b), c in X.items())
    back = {u0: dd[0] + dd[4], u1: dd[1] + dd[3], u2: dd[2], w0: dd[0] - dd[4], w1: dd[1] - dd[3]}
    assert sp.expand((Sv + Tv + 2 * Xv).subs(back, simultaneous=True) - bL) == 0
    assert sp.expand((Sv + Tv - 2 * Xv).subs(back, simultaneous=True) - bR) == 0
    assert sp.expand(sum(c * d[i] * d[j] for (i, j), c in c4.items()) - b4) == 0
    f = lambda c: "%r" % float(c)
    print("// beta4_diff: beta4 of cells (0, 1, 2, 3) around target 0 in the consecutive differences")
    print("// of those cells, d[0..2]; coefficients are the exact rationals rounded to FP64.")
    print("FL_HD double beta4_diff(double d0, double d1, double d2) {")
    print("  const double r0 = fma(%s, d2, fma(%s, d1, %s * d0));" % (f(c4[(0, 2)]), f(c4[(0, 1)]), f(c4[(0, 0)])))
    print("  const double r1 = fma(%s, d2, %s * d1);" % (f(c4[(1, 2)]), f(c4[(1, 1)])))
    print("  return fma(d2, %s * d2, fma(d1, r1, d0 * r0));" % f(c4[(2, 2)]))
    print("}")
    print()
    print("// beta6_pair_diff: 6 beta6 of the window q[0..5] and of its mirror image from the window's")
    print("// consecutive differences d[0..4]: bL = S + T + 2 X, bR = S + T - 2 X with u0 = d0 + d4,")
    print("// u1 = d1 + d3, u2 = d2, w0 = d0 - d4, w1 = d1 - d3 (the reversal keeps u and negates w).")
    print("FL_HD void beta6_pair_diff(const double d[5], double& bL, double& bR) {")
    print("  const double u0 = d[0] + d[4], u1 = d[1] + d[3], u2 = d[2];")
    print("  const double w0 = d[0] - d[4], w1 = d[1] - d[3];")
    print("  const double s0 = fma(%s, u2, fma(%s, u1, %s * u0));" % (f(S[("u0", "u2")]), f(S[("u0", "u1")]), f(S[("u0", "u0")])))
    print("  const double s1 = fma(%s, u2, %s * u1);" % (f(S[("u1", "u2")]), f(S[("u1", "u1")])))
    print("  const double S = fma(u2, %s * u2, fma(u1, s1, u0 * s0));" % f(S[("u2", "u2")]))
    print("  const double T = fma(w1, %s * w1, w0 * fma(%s, w1, %s * w0));" % (f(T[("w1", "w1")]), f(T[("w0", "w1")]), f(T[("w0", "w0")])))
    print("  const double x0 = fma(%s, w1, %s * w0);" % (f(2 * X[("u0", "w1")]), f(2 * X[("u0", "w0")])))
    print("  const double x1 = fma(%s, w1, %s * w0);" % (f(2 * X[("u1", "w1")]), f(2 * X[("u1", "w0")])))
    print("  const double x2 = fma(%s, w1, %s * w0);" % (f(2 * X[("u2", "w1")]), f(2 * X[("u2", "w0")])))
    print("  const double X2 = fma(u2, x2, fma(u1, x1, u0 * x0));")
    print("  const double ST = S + T;")
    print("  bL = ST + X2;")
    print("  bR = ST - X2;")
    print("}")
    print()


def emit_cutoff_thresholds(alpha1=sp.Rational(21, 2), alpha2=sp.Rational(7, 2), cr=sp.Rational(1, 4)):
    """The adaptive cut-off C_T = 10^-floor(alpha1 - alpha2 (1 - g)), g = (1 - m)^4 (1 + 4 m),
    m = 1 - min(1, eta / C_r), as thresholds on the sensor eta.  With t = 1 - m = min(1, eta / C_r),
    g = t^4 (5 - 4 t) increases with t on [0, 1], so floor(...) >= k (k = 8, 9, 10) exactly when
    g >= c_k = 1 - (alpha1 - k) / alpha2, i.e. when eta >= C_r t_k with t_k^4 (5 - 4 t_k) = c_k."""
    t = sp.symbols("t")
    out = []
    for k in (8, 9, 10):
        c = 1 - (alpha1 - k) / alpha2
        roots = [r for r in sp.Poly(t ** 4 * (5 - 4 * t) - c, t).nroots(n=40) if r.is_real and 0 < r < 1]
        assert len(roots) == 1
        out.append((k, c, cr * roots[0]))
    print("// adaptive cut-off as thresholds on the smallest sensor eta: C_T = 10^-k for eta >= eta_k")
    print("// (k = 10, 9, 8; else 10^-7), eta_k = C_r t_k with t_k^4 (5 - 4 t_k) = 1 - (alpha1 - k) / alpha2")
    for k, c, e in out:
        print("constexpr double kCutEta%d = %r;   // g = %s" % (k, float(e), c))
    print()


print("// Generated by gen_teno_coeffs.py (sympy, from the Jiang-Shu definition); do not edit.")
print("#pragma once")
print("#ifndef FL_HD")
print("#define FL_HD __host__ __device__ __forceinline__")
print("#endif")
print("namespace fl {")
print("namespace teno {")
emit_diff_forms()
emit_cutoff_thresholds()
print("}  // namespace teno")
print("}  // namespace fl")
