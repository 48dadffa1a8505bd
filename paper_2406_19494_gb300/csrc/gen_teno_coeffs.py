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
    print("// beta = sum_{j<=k} c_jk e_j e_k / %d, grouped by rows: sum_j e_j (sum_{k>=j} c_jk e_k)." % den)
    print("FL_HD double %s(const double e[%d]) {" % (name, n))
    rows = []
    for j in range(n):
        row = [(k, c) for (jj, k, c) in terms if jj == j]
        expr = "%d.0 * e[%d]" % (row[0][1], row[0][0])
        for k, c in row[1:]:
            expr = "fma(%d.0, e[%d], %s)" % (c, k, expr)
        print("  const double r%d = %s;" % (j, expr))
        rows.append(j)
    acc = "e[0] * r0"
    for j in rows[1:]:
        acc = "fma(e[%d], r%d, %s)" % (j, j, acc)
    print("  return (%s) * (1.0 / %d.0);" % (acc, den))
    print("}")
    print()


print("// Generated by gen_teno_coeffs.py (sympy, from the Jiang-Shu definition); do not edit.")
print("#pragma once")
print("#ifndef FL_HD")
print("#define FL_HD __host__ __device__ __forceinline__")
print("#endif")
print("namespace fl {")
print("namespace teno {")
emit("beta4_form", (0, 1, 2, 3))
emit("beta6_form", (-2, -1, 0, 1, 2, 3))
print("}  // namespace teno")
print("}  // namespace fl")
