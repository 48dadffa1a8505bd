"""Write teno_coeffs.cuh: the rational coefficients of the TENO6 smoothness measures used by the
FP64 kernels, derived symbolically (sympy) from the Jiang-Shu definition.

Not part of the build: the generated header is committed, and this script re-creates it (needs
sympy, available on the development machine only).  Run from this directory:
    python gen_teno_coeffs.py > teno_coeffs.cuh

For a stencil of cells with unit width centred at the integer offsets s (x measured from the centre
of the target cell), the reconstruction polynomial P has the stencil's cell averages, and
beta = sum_{l >= 1} int_{-1/2}^{1/2} (P^(l))^2 dx.  beta vanishes on constants, so it is written as
a quadratic form in the differences e_j = q_{s_j} - q_{s_0} (j >= 1): beta = sum_{j<=k} c_jk e_j e_k
/ den with integer c_jk, emitted as a function of the differences.
"""
import sympy as sp


def quadratic_form(offsets):
    x = sp.symbols("x")
    n = len(offsets)
    a = sp.symbols("a0:%d" % n)
    q = sp.symbols("q0:%d" % n)
    P = sum(a[m] * x ** m for m in range(n))
    eqs = [sp.integrate(P, (x, o - sp.Rational(1, 2), o + sp.Rational(1, 2))) - q[j]
           for j, o in enumerate(offsets)]
    sol = sp.solve(eqs, a, dict=True)[0]
    Pq = P.subs(sol)
    beta = sum(sp.integrate(sp.diff(Pq, x, l) ** 2, (x, -sp.Rational(1, 2), sp.Rational(1, 2)))
               for l in range(1, n))
    e = sp.symbols("e1:%d" % n)
    beta = sp.expand(beta.subs({q[j]: q[0] + e[j - 1] for j in range(1, n)}))
    assert beta.free_symbols <= set(e)
    poly = sp.Poly(beta, *e)
    den = sp.ilcm(*[sp.fraction(c)[1] for c in poly.coeffs()])
    terms = []
    for j in range(n - 1):
        for k in range(j, n - 1):
            mono = [0] * (n - 1)
            mono[j] += 1
            mono[k] += 1
            terms.append((j, k, int(poly.coeff_monomial(tuple(mono)) * den)))
    return int(den), terms


def emit(name, offsets):
    den, terms = quadratic_form(offsets)
    n = len(offsets) - 1
    print("// %s: cells %s (offsets from the target cell), e[j-1] = q_{s_j} - q_{s_0}, j = 1 .. %d:"
          % (name, offsets, n))
    print("// beta = sum_{j<=k} c_jk e_j e_k / %d, grouped by rows: sum_j e_j (sum_{k>=j} c_jk e_k / %d)"
          % (den, den))
    print("// (the coefficients c_jk / %d rounded to FP64)." % den)
    print("FL_HD double %s(const double e[%d]) {" % (name, n))
    rows = []
    f = lambda c: "%r" % (float(sp.Rational(c, den)))
    for j in range(n):
        row = [(k, c) for (jj, k, c) in terms if jj == j]
        expr = "%s * e[%d]" % (f(row[0][1]), row[0][0])
        for k, c in row[1:]:
            expr = "fma(%s, e[%d], %s)" % (f(c), k, expr)
        print("  const double r%d = %s;" % (j, expr))
        rows.append(j)
    acc = "e[0] * r0"
    for j in rows[1:]:
        acc = "fma(e[%d], r%d, %s)" % (j, j, acc)
    print("  return %s;" % acc)
    print("}")
    print()


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


def emit_pair(name, offsets, scale=6):
    """Both smoothness measures of a six-cell window and of its mirror image, the form evaluated on
    q and on (q5, .., q0).  With u_j = q_j + q_{5-j} and v_j = q_j - q_{5-j} (j = 0, 1, 2), the
    reversal leaves u and negates v, so beta(q) = S + T + 2 X and beta(Jq) = S + T - 2 X with S a
    form in u, T a form in v and X bilinear; S and X vanish on constants, so they are written in
    a_k = u_k - u_0 (k = 1, 2)."""
    A, q, beta = beta_matrix(offsets)
    n = len(offsets)
    assert n == 6 and all(offsets[j] + offsets[5 - j] == 1 for j in range(3))   # symmetric about the face
    u = sp.symbols("u0:3")
    v = sp.symbols("v0:3")
    sub = {}
    for j in range(3):
        sub[q[j]] = (u[j] + v[j]) / 2
        sub[q[5 - j]] = (u[j] - v[j]) / 2
    bq = sp.expand(beta.subs(sub, simultaneous=True))
    a1, a2 = sp.symbols("a1 a2")
    bq = sp.expand(bq.subs({u[1]: u[0] + a1, u[2]: u[0] + a2}, simultaneous=True))
    assert u[0] not in bq.free_symbols
    poly = sp.Poly(bq, a1, a2, *v)
    coeff = lambda mono: poly.coeff_monomial(mono)
    # S = s11 a1^2 + s12 a1 a2 + s22 a2^2; X = sum x_kj a_k v_j (the part odd in v, halved);
    # T = sum_{i<=j} t_ij v_i v_j
    S = {(1, 1): coeff((2, 0, 0, 0, 0)), (1, 2): coeff((1, 1, 0, 0, 0)), (2, 2): coeff((0, 2, 0, 0, 0))}
    X = {}
    for k in (1, 2):
        for j in range(3):
            mono = [0] * 5
            mono[k - 1] = 1
            mono[2 + j] = 1
            X[(k, j)] = coeff(tuple(mono)) / 2
    T = {}
    for i in range(3):
        for j in range(i, 3):
            mono = [0] * 5
            mono[2 + i] += 1
            mono[2 + j] += 1
            T[(i, j)] = coeff(tuple(mono))
    # exact check: the pair reproduces the form on the window and on its mirror image
    qs = sp.symbols("w0:6")
    us = [qs[j] + qs[5 - j] for j in range(3)]
    vs = [qs[j] - qs[5 - j] for j in range(3)]
    A1, A2 = us[1] - us[0], us[2] - us[0]
    Sv = S[(1, 1)] * A1 ** 2 + S[(1, 2)] * A1 * A2 + S[(2, 2)] * A2 ** 2
    Xv = sum(X[(k, j)] * (A1 if k == 1 else A2) * vs[j] for k in (1, 2) for j in range(3))
    Tv = sum(T[(i, j)] * vs[i] * vs[j] for i in range(3) for j in range(i, 3))
    bL = beta.subs(dict(zip(q, qs)), simultaneous=True)
    bR = beta.subs(dict(zip(q, reversed(qs))), simultaneous=True)
    assert sp.expand(Sv + Tv + 2 * Xv - bL) == 0 and sp.expand(Sv + Tv - 2 * Xv - bR) == 0
    f = lambda c: "%r" % float(scale * c)
    print("// %s: %d times the TENO6 measure of the window q[0..5] (cells %s around the target cell)"
          % (name, scale, offsets))
    print("// and of its mirror image (q[5..0]): bL = S + T + 2 X, bR = S + T - 2 X with u_j = q_j + q_{5-j},")
    print("// v_j = q_j - q_{5-j}, a_k = u_k - u_0; coefficients are %d times the exact rationals, rounded" % scale)
    print("// to FP64 (the factor is the 6 of tau6 = |beta6 - (beta1 + beta2 + 4 beta0) / 6|).")
    print("FL_HD void %s(const double q[6], double& bL, double& bR) {" % name)
    print("  // a_k from differences of neighbouring values, exact for close values, never from the sums u_k")
    print("  const double a1 = (q[1] - q[0]) + (q[4] - q[5]), a2 = (q[2] - q[0]) + (q[3] - q[5]);")
    print("  const double v0 = q[0] - q[5], v1 = q[1] - q[4], v2 = q[2] - q[3];")
    print("  const double S = fma(a1, fma(%s, a2, %s * a1), (%s * a2) * a2);" % (f(S[(1, 2)]), f(S[(1, 1)]), f(S[(2, 2)])))
    print("  const double t0 = fma(%s, v2, fma(%s, v1, %s * v0));" % (f(T[(0, 2)]), f(T[(0, 1)]), f(T[(0, 0)])))
    print("  const double t1 = fma(%s, v2, %s * v1);" % (f(T[(1, 2)]), f(T[(1, 1)])))
    print("  const double T = fma(v2, %s * v2, fma(v1, t1, v0 * t0));" % f(T[(2, 2)]))
    print("  const double x1 = fma(%s, v2, fma(%s, v1, %s * v0));" % (f(2 * X[(1, 2)]), f(2 * X[(1, 1)]), f(2 * X[(1, 0)])))
    print("  const double x2 = fma(%s, v2, fma(%s, v1, %s * v0));" % (f(2 * X[(2, 2)]), f(2 * X[(2, 1)]), f(2 * X[(2, 0)])))
    print("  const double X2 = fma(a2, x2, a1 * x1);")
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
emit("beta4_form", (0, 1, 2, 3))
emit_pair("beta6_pair", (-2, -1, 0, 1, 2, 3))
emit_cutoff_thresholds()
print("}  // namespace teno")
print("}  // namespace fl")
