// Per-face FP64 arithmetic of the right-hand side, shared by the forward kernels, the adjoint
// kernels and the host-compiled checks of the adjoint: WENO5 reconstruction (Jiang & Shu; Borges
// et al. for the Z weights), the HLLC flux (Toro Ch. 10) and the constants they use.
#pragma once

#include <cmath>

#include "fast_math.cuh"
#include "fluid_internal.cuh"

#ifndef FL_HD
#define FL_HD __host__ __device__ __forceinline__
#endif

namespace fl {

constexpr double kSixth = 1.0 / 6.0;
constexpr double k1312 = 13.0 / 12.0;
constexpr double kTwelfth = 1.0 / 12.0;
constexpr double k24th = 1.0 / 24.0;
constexpr double k16th = 1.0 / 16.0;

// ------------------------------------------------------------------------------------------------
// WENO5 (Jiang & Shu; Borges et al. Z variant): left-biased value at i+1/2 from q_{i-2..i+2}
// ------------------------------------------------------------------------------------------------
// Smoothness indicators of the three-cell stencil (a, b, c) in the three positions WENO5 uses it:
// as the left candidate (A), the centre one (B) and the right one (C) of a left-biased face value.
FL_HD double weno_A(double a, double b, double c) {
  const double t = a - 2.0 * b + c, s = a - 4.0 * b + 3.0 * c;
  return k1312 * t * t + 0.25 * s * s;
}
FL_HD double weno_B(double a, double b, double c) {
  const double t = a - 2.0 * b + c, s = a - c;
  return k1312 * t * t + 0.25 * s * s;
}
FL_HD double weno_C(double a, double b, double c) {
  const double t = a - 2.0 * b + c, s = 3.0 * a - 4.0 * b + c;
  return k1312 * t * t + 0.25 * s * s;
}

// WENO5 face value from the stencil and its three smoothness indicators (beta_0, beta_1, beta_2)
template <int SCHEME>
FL_HD double weno5_beta(double qm2, double qm1, double q0, double qp1, double qp2, double b0,
                        double b1, double b2, double eps) {
  // candidate values times 6
  const double C0 = 2.0 * qm2 - 7.0 * qm1 + 11.0 * q0;
  const double C1 = -qm1 + 5.0 * q0 + 2.0 * qp1;
  const double C2 = 2.0 * q0 + 5.0 * qp1 - qp2;
  // Weights scaled by a common positive factor so that one division remains.  With
  // e_k = beta_k + eps and Q_k = prod_{j != k} e_j:
  //   JS: d_k / e_k^2                  = d_k Q_k^2 / P^2,              P = e0 e1 e2
  //   Z : d_k (1 + (tau5 / e_k)^2)     = d_k (P^2 + tau5^2 Q_k^2) / P^2
  // The common 1/P^2 cancels in omega_k = alpha_k / sum alpha.  Since e_k >= eps the scaled
  // weights stay normal for eps = 1e-40 (P^2 >= 1e-240) and finite while beta_k < 1e50.
  const double e0 = b0 + eps, e1 = b1 + eps, e2 = b2 + eps;
  const double Q0 = e1 * e2, Q1 = e0 * e2, Q2 = e0 * e1;
  double a0, a1, a2;
  if (SCHEME == FLUID_WENO_JS) {
    a0 = 0.1 * (Q0 * Q0); a1 = 0.6 * (Q1 * Q1); a2 = 0.3 * (Q2 * Q2);
  } else {
    const double tau = b0 - b2 < 0.0 ? b2 - b0 : b0 - b2;
    const double P = e0 * Q0;
    const double PP = P * P, tt = tau * tau;
    a0 = 0.1 * (PP + tt * (Q0 * Q0));
    a1 = 0.6 * (PP + tt * (Q1 * Q1));
    a2 = 0.3 * (PP + tt * (Q2 * Q2));
  }
  return (a0 * C0 + a1 * C1 + a2 * C2) * fl_rcp(6.0 * (a0 + a1 + a2));
}

// The same reconstruction split for marching along a grid line.  The indicator set of the
// right-biased value at face a+1/2 is, with the roles of its outer members exchanged, the set of
// the left-biased value at a+3/2; weno_x gives the scaled weights of a set (X_k = alpha_k / d_k
// times the common factor of weno5_beta, which is symmetric under that exchange) so that one set
// serves both faces, and weno_x_value forms the value from the stencil's centre and cell
// differences and the X's, with the linear weights d_k and 1/6 folded into the candidate
// coefficients.

// The scaled weights X_k of an indicator set whose members already include epsilon,
// e_k = beta_k + eps (so that tau = |e0 - e2| = |beta0 - beta2|)
template <int SCHEME>
FL_HD void weno_x(double e0, double e1, double e2, double X[3]) {
  const double Q0 = e1 * e2, Q1 = e0 * e2, Q2 = e0 * e1;
  if (SCHEME == FLUID_WENO_JS) {
    X[0] = Q0 * Q0; X[1] = Q1 * Q1; X[2] = Q2 * Q2;
  } else {
    const double tau = fabs(e0 - e2);
    const double P = e0 * Q0;
    const double PP = P * P;
    const double T0 = tau * Q0, T1 = tau * Q1, T2 = tau * Q2;
    X[0] = fma(T0, T0, PP);
    X[1] = fma(T1, T1, PP);
    X[2] = fma(T2, T2, PP);
  }
}

// The value from the stencil centre q0 and the four cell differences of the stencil,
// dm2 = q_{i-1} - q_{i-2}, dm1 = q_i - q_{i-1}, dp0 = q_{i+1} - q_i, dp1 = q_{i+2} - q_{i+1}:
// with the candidates as offsets from q_i, p0 - q_i = (5 dm1 - 2 dm2) / 6,
// p1 - q_i = (dm1 + 2 dp0) / 6, p2 - q_i = (4 dp0 - dp1) / 6 (d_k / 6 folded in, and both sums
// scaled by 10 so that two coefficients are 1).
FL_HD double weno_x_value(double q0, double dm2, double dm1, double dp0, double dp1, const double X[3]) {
  // d = (1/10, 6/10, 3/10); numerator and denominator both taken times 10
  const double C0 = fma(5.0 / 6.0, dm1, (-1.0 / 3.0) * dm2);
  const double C1 = fma(2.0, dp0, dm1);
  const double C2 = fma(-0.5, dp1, 2.0 * dp0);
  const double num = fma(X[2], C2, fma(X[1], C1, X[0] * C0));
  const double den = fma(3.0, X[2], fma(6.0, X[1], X[0]));
  return fma(num, fl_rcp(den), q0);
}

// WENO5 (Jiang & Shu; Borges et al. Z variant): left-biased value at i+1/2 from q_{i-2..i+2}
template <int SCHEME>
FL_HD double weno5(double qm2, double qm1, double q0, double qp1, double qp2, double eps) {
  return weno5_beta<SCHEME>(qm2, qm1, q0, qp1, qp2, weno_A(qm2, qm1, q0), weno_B(qm1, q0, qp1),
                            weno_C(q0, qp1, qp2), eps);
}

// ------------------------------------------------------------------------------------------------
// HLLC along axis D (Toro Ch. 10) with Einfeldt/Roe wave-speed bounds.  Branch order:
// S_L >= 0 -> F_L; S* >= 0 -> F*_L; S_R > 0 -> F*_R; else F_R.
// ------------------------------------------------------------------------------------------------
template <int D>
FL_HD void hllc(const double wl[5], const double wr[5], const Phys& ph,
                                     double F[5]) {
  const double rL = wl[0], pL = wl[4], rR = wr[0], pR = wr[4];
  const double unL = wl[1 + D], unR = wr[1 + D];
  const double q2L = wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3];
  const double q2R = wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3];
  // 1/sqrt(rho) gives both sqrt(rho) (Roe weights) and 1/rho
  const double qL = fl_rsqrt(rL), qR = fl_rsqrt(rR);
  const double sL = rL * qL, sR = rR * qR;
  const double irL = qL * qL, irR = qR * qR;
  // p / rho and the total enthalpy H = (E + p) / rho = gamma/(gamma-1) p/rho + |u|^2 / 2
  const double gg = ph.gamma * ph.igm1;
  const double pirL = pL * irL, pirR = pR * irR;
  const double HL = fma(pirL, gg, 0.5 * q2L), HR = fma(pirR, gg, 0.5 * q2R);
  const double cL = fl_sqrt(ph.gamma * pirL), cR = fl_sqrt(ph.gamma * pirR);
  // Roe weights sqrt(rho_K) / (sqrt(rho_L) + sqrt(rho_R))
  const double isum = fl_rcp(sL + sR);
  const double aL = sL * isum, aR = sR * isum;
  const double ut0 = fma(aL, wl[1], aR * wr[1]);
  const double ut1 = fma(aL, wl[2], aR * wr[2]);
  const double ut2 = fma(aL, wl[3], aR * wr[3]);
  const double Ht = fma(aL, HL, aR * HR);
  const double ct = fl_sqrt(ph.gm1 * (Ht - 0.5 * (ut0 * ut0 + ut1 * ut1 + ut2 * ut2)));
  const double utn = D == 0 ? ut0 : (D == 1 ? ut1 : ut2);
  const double SL = fmin(unL - cL, utn - ct);
  const double SR = fmax(unR + cR, utn + ct);
  const double mL = rL * (SL - unL), mR = rR * (SR - unR);
  const double Ss = (pR - pL + unL * mL - unR * mR) * fl_rcp(mL - mR);

  const bool left = fl_nonneg(SL) || fl_nonneg(Ss);
  const bool star = left ? !fl_nonneg(SL) : fl_pos(SR);
  const double r = left ? rL : rR;
  const double p = left ? pL : pR;
  const double H = left ? HL : HR;
  const double un = left ? unL : unR;
  const double S = left ? SL : SR;
  const double m = left ? mL : mR;
  const double u0 = left ? wl[1] : wr[1];
  const double u1 = left ? wl[2] : wr[2];
  const double u2 = left ? wl[3] : wr[3];
  // Euler flux of the selected side: (rho u_n, rho u_n u + p n, rho u_n H)
  const double mn = r * un;
  F[0] = mn;
  F[1] = mn * u0;
  F[2] = mn * u1;
  F[3] = mn * u2;
  F[1 + D] += p;
  F[4] = mn * H;
  if (star) {
    // U*_K = m/(S - S*) [1, S* (normal), tangential u, E/rho + (S* - un)(S* + p/m)]
    const double q = fl_rcp(S - Ss);
    const double fac = m * q;
    const double pir = left ? pirL : pirR;
    const double eir = H - pir;                       // E / rho
    const double dU0 = fac - r;
    double dU[3] = {dU0 * u0, dU0 * u1, dU0 * u2};
    dU[D] = fac * Ss - r * un;
    const double Es = fac * eir + (Ss - un) * (fac * Ss + p * q);
    F[0] += S * dU0;
    F[1] += S * dU[0];
    F[2] += S * dU[1];
    F[3] += S * dU[2];
    F[4] += S * (Es - r * eir);
  }
}


// ------------------------------------------------------------------------------------------------
// conservative -> primitive (rho, u, v, w, p, T) with one division
// ------------------------------------------------------------------------------------------------
FL_HD void prim_from_cons(const double U[5], const Phys& ph, double w[6]) {
  const double r = U[0];
  const double ir = fl_rcp(r);
  const double u = U[1] * ir, v = U[2] * ir, ww = U[3] * ir;
  const double p = ph.gm1 * (U[4] - 0.5 * r * (u * u + v * v + ww * ww));
  w[0] = r; w[1] = u; w[2] = v; w[3] = ww; w[4] = p; w[5] = p * ir * ph.iR;
}

// wall halo map of axis a applied to primitives w: velocity mirrored; isothermal T_g = 2 T_w - T,
// p_g = p, rho_g = p / (R T_g); porous adds 2 v_w to the wall-normal component.  Returns false
// when the ghost temperature is not positive.
FL_HD bool wall_map_prim(double w[6], int kind, double Tw, double vw, int a, const Phys& ph) {
  w[1] = -w[1]; w[2] = -w[2]; w[3] = -w[3];
  if (kind == FLUID_BC_ADIABATIC) return true;
  const double Tg = 2.0 * Tw - w[5];
  w[0] = w[4] / (ph.R * Tg);
  w[5] = Tg;
  if (kind == FLUID_BC_POROUS) w[1 + a] = 2.0 * vw + w[1 + a];
  return Tg > 0.0;
}

// ------------------------------------------------------------------------------------------------
// dissipative face flux along D by central differences of order NP (4 or 6 points); the face is
// between cells NP/2 - 1 and NP/2 of the NP-cell stencils: vel[c][k], T[k] at cells
// a-NP/2+1 .. a+NP/2; gd[b][k] = d u_D / d x_b and gb[b][k] = d u_b / d x_b at the same cells for
// tangential axes b (ignored for b == D or b >= ndim); mfa = d(index)/dx at the face.  Returns
// Fd = (tau_0D, tau_1D, tau_2D, energy).
//   4 points: value (9 (f1 + f2) - (f0 + f3)) / 16, derivative ((f0 - f3) + 27 (f2 - f1)) / 24
//   6 points: value (150 (f2 + f3) - 25 (f1 + f4) + 3 (f0 + f5)) / 256,
//             derivative (2250 (f3 - f2) - 125 (f4 - f1) + 9 (f5 - f0)) / 1920
// ------------------------------------------------------------------------------------------------
// the derivatives take m = mfa / 24 (order 4) or mfa / 1920 (order 6), formed once per face
FL_HD double interp4(const double f[4]) { return (9.0 * (f[1] + f[2]) - (f[0] + f[3])) * k16th; }
FL_HD double dnorm4(const double f[4], double m) { return ((f[0] - f[3]) + 27.0 * (f[2] - f[1])) * m; }
FL_HD double interp6(const double f[6]) {
  return (150.0 * (f[2] + f[3]) - 25.0 * (f[1] + f[4]) + 3.0 * (f[0] + f[5])) * (1.0 / 256.0);
}
FL_HD double dnorm6(const double f[6], double m) {
  return (2250.0 * (f[3] - f[2]) - 125.0 * (f[4] - f[1]) + 9.0 * (f[5] - f[0])) * m;
}
template <int NP>
FL_HD double interp_np(const double f[NP]) {
  if constexpr (NP == 4) return interp4(f);
  else return interp6(f);
}
template <int NP>
FL_HD double dnorm_np(const double f[NP], double mfa) {
  if constexpr (NP == 4) return dnorm4(f, mfa);
  else return dnorm6(f, mfa);
}

template <int D, int NP = 4>
FL_HD void visc_face(const double vel[3][NP], const double T[NP], const double gd[3][NP],
                     const double gb[3][NP], int ndim, double mfa, const Phys& ph, double Fd[4]) {
  const double m = mfa * (NP == 4 ? k24th : 1.0 / 1920.0);
  double vf[3], Gf[3][3];
  for (int c = 0; c < 3; ++c) {
    vf[c] = interp_np<NP>(vel[c]);
    Gf[c][D] = dnorm_np<NP>(vel[c], m);
  }
  const double Tf = interp_np<NP>(T);
  const double dT = dnorm_np<NP>(T, m);
  for (int b = 0; b < 3; ++b) {
    if (b == D) continue;
    if (b < ndim) {
      Gf[D][b] = interp_np<NP>(gd[b]);
      Gf[b][b] = interp_np<NP>(gb[b]);
    } else {
      Gf[D][b] = 0.0;
      Gf[b][b] = 0.0;
    }
  }
  const double div = Gf[0][0] + Gf[1][1] + Gf[2][2];
  const double mu = viscosity(Tf, ph);
  const double lam = mu * ph.lam_fac;
  for (int c = 0; c < 3; ++c) {
    if (c == D) Fd[c] = mu * (Gf[D][D] + Gf[D][D]) - (2.0 / 3.0) * mu * div;
    else Fd[c] = mu * (Gf[c][D] + Gf[D][c]);
  }
  Fd[3] = vf[0] * Fd[0] + vf[1] * Fd[1] + vf[2] * Fd[2] + lam * dT;
}

// Dissipative flux of the face a+1/2 along D from the primitives W and centre gradients G, with
// the NP-point stencils; q holds the velocities already loaded for cells a-2 .. a+3 (q[1..3][o],
// o = 0 .. 5).  F -= (0, tau_0D, tau_1D, tau_2D, energy).
#ifdef __CUDACC__
template <int D, int NP>
__device__ __forceinline__ void add_visc_face(const double* __restrict__ W, const double* __restrict__ G, int cell, int s,
                         int a, const Geo& g, const Phys& ph, const double q[5][6], double F[5]) {
  constexpr int o0 = 3 - NP / 2;           // first stencil cell within q: a - NP/2 + 1
  const int nc = g.ncell;
  double vel[3][NP], T[NP], gd[3][NP], gb[3][NP];
#pragma unroll
  for (int o = 0; o < NP; ++o) {
    vel[0][o] = q[1][o0 + o];
    vel[1][o] = q[2][o0 + o];
    vel[2][o] = q[3][o0 + o];
    T[o] = __ldg(W + 5 * nc + cell + (o + o0 - 2) * s);
  }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (b == D || b >= g.ndim) continue;
    const double* pd = G + (D * 3 + b) * nc + cell;   // d u_D / d x_b
    const double* pb = G + (b * 3 + b) * nc + cell;   // d u_b / d x_b
#pragma unroll
    for (int o = 0; o < NP; ++o) {
      gd[b][o] = __ldg(pd + (o + o0 - 2) * s);
      gb[b][o] = __ldg(pb + (o + o0 - 2) * s);
    }
  }
  double Fd[4];
  visc_face<D, NP>(vel, T, gd, gb, g.ndim, g.mf[D][a], ph, Fd);
  F[1] -= Fd[0];
  F[2] -= Fd[1];
  F[3] -= Fd[2];
  F[4] -= Fd[3];
}
#endif

}  // namespace fl
