// Reverse-mode (vector-Jacobian) forms of the per-face and per-cell arithmetic in flux_math.cuh,
// written by hand.  Each *_vjp function recomputes the forward intermediates it needs and returns
// the cotangents of its inputs given the cotangent of its output.  Non-smooth points follow the
// forward's own decisions: the HLLC branch and the Einfeldt min / max take the derivative of the
// selected argument (first argument on ties), |b0 - b2| in WENO5-Z has derivative +1 at zero.
// The WENO weights are differentiated exactly (no frozen weights).
#pragma once

#include "flux_math.cuh"

namespace fl {

// ------------------------------------------------------------------------------------------------
// WENO5: cotangent of the five stencil values q_{i-2..i+2} given the cotangent of the face value
// ------------------------------------------------------------------------------------------------
// With out != nullptr the face value itself (the forward result, q_i plus the offset form) is
// returned too; with g_out = 1 gq is the gradient of the face value.
template <int SCHEME>
FL_HD void weno5_vjp(const double qin[5], double eps, double g_out, double gq[5],
                     double* out_value = nullptr) {
  // WENO5 is translation-equivariant (f(q - c) = f(q) - c), so its Jacobian is that of the data
  // shifted by the centre value.  Working on the shifted data keeps every intermediate -- in
  // particular the weight cotangents, proportional to C_k - 6 f -- free of the cancellation of
  // two O(|q|) numbers, whose rounding the weight derivatives (~1 / spread of the data) would
  // otherwise amplify in nearly uniform regions.
  const double q[5] = {qin[0] - qin[2], qin[1] - qin[2], 0.0, qin[3] - qin[2], qin[4] - qin[2]};
  const double C0 = 2.0 * q[0] - 7.0 * q[1] + 11.0 * q[2];
  const double C1 = -q[1] + 5.0 * q[2] + 2.0 * q[3];
  const double C2 = 2.0 * q[2] + 5.0 * q[3] - q[4];
  const double t0 = q[0] - 2.0 * q[1] + q[2], s0 = q[0] - 4.0 * q[1] + 3.0 * q[2];
  const double t1 = q[1] - 2.0 * q[2] + q[3], s1 = q[1] - q[3];
  const double t2 = q[2] - 2.0 * q[3] + q[4], s2 = 3.0 * q[2] - 4.0 * q[3] + q[4];
  // indicators and epsilon taken times 4 (4 beta = 13/3 t^2 + s^2): the weights of either scheme
  // are homogeneous in (beta + eps, tau), so the value and its gradient are unchanged
  constexpr double K4 = 4.0 * k1312;
  const double b0 = fma(K4 * t0, t0, s0 * s0);
  const double b1 = fma(K4 * t1, t1, s1 * s1);
  const double b2 = fma(K4 * t2, t2, s2 * s2);
  const double eps4 = 4.0 * eps;
  const double e0 = b0 + eps4, e1 = b1 + eps4, e2 = b2 + eps4;
  double a0, a1, a2, ge0, ge1, ge2, gb0 = 0.0, gb2 = 0.0;
  // face value = N / (6 S), N = sum a_k C_k, S = sum a_k
  double r0 = 0.0, r1 = 0.0, r2 = 0.0, sg = 1.0;
  const double i0 = fl_rcp(e0), i1 = fl_rcp(e1), i2 = fl_rcp(e2);
  if (SCHEME == FLUID_WENO_JS) {
    a0 = 0.1 * i0 * i0; a1 = 0.6 * i1 * i1; a2 = 0.3 * i2 * i2;
    r0 = i0; r1 = i1; r2 = i2;
  } else {
    const double tau = b0 - b2 < 0.0 ? b2 - b0 : b0 - b2;
    sg = b0 - b2 < 0.0 ? -1.0 : 1.0;
    r0 = tau * i0; r1 = tau * i1; r2 = tau * i2;
    a0 = 0.1 * fma(r0, r0, 1.0); a1 = 0.6 * fma(r1, r1, 1.0); a2 = 0.3 * fma(r2, r2, 1.0);
  }
  const double S = a0 + a1 + a2;
  const double N = a0 * C0 + a1 * C1 + a2 * C2;
  const double iS6 = fl_rcp(6.0 * S);
  const double out = N * iS6;
  if (out_value) *out_value = out + qin[2];
  const double gN = g_out * iS6;
  const double gS = -6.0 * out * gN;                 // -g_out out / S
  const double ga0 = fma(gN, C0, gS), ga1 = fma(gN, C1, gS), ga2 = fma(gN, C2, gS);
  const double gC0 = gN * a0, gC1 = gN * a1, gC2 = gN * a2;
  if (SCHEME == FLUID_WENO_JS) {
    // a_k = d_k / e_k^2: da/de = -2 a / e
    ge0 = -2.0 * ga0 * a0 * r0;
    ge1 = -2.0 * ga1 * a1 * r1;
    ge2 = -2.0 * ga2 * a2 * r2;
  } else {
    // a_k = d_k (1 + r_k^2), r_k = tau / e_k
    const double gr0 = ga0 * 0.2 * r0, gr1 = ga1 * 1.2 * r1, gr2 = ga2 * 0.6 * r2;
    const double gtau = fma(gr2, i2, fma(gr1, i1, gr0 * i0));
    ge0 = -gr0 * r0 * i0;
    ge1 = -gr1 * r1 * i1;
    ge2 = -gr2 * r2 * i2;
    gb0 = sg * gtau;
    gb2 = -gb0;
  }
  gb0 += ge0;
  const double gb1 = ge1;
  gb2 += ge2;
  // b_k = (13/3) t_k^2 + s_k^2: gt_k = gb_k (26/3) t_k, gs_k = 2 gb_k s_k, folded below as
  // u_k = gb_k t_k and v_k = gb_k s_k with the factors in the coefficients
  const double u0 = gb0 * t0, v0 = gb0 * s0;
  const double u1 = gb1 * t1, v1 = gb1 * s1;
  const double u2 = gb2 * t2, v2 = gb2 * s2;
  constexpr double T = 2.0 * K4;
  gq[0] = fma(2.0, gC0, fma(T, u0, 2.0 * v0));
  gq[1] = fma(-7.0, gC0, -gC1) + fma(-2.0 * T, u0, fma(-8.0, v0, fma(T, u1, 2.0 * v1)));
  gq[3] = fma(2.0, gC1, 5.0 * gC2) + fma(T, u1, fma(-2.0, v1, fma(-2.0 * T, u2, -8.0 * v2)));
  gq[4] = -gC2 + fma(T, u2, 2.0 * v2);
  // translation: f(q + c) = f(q) + c, so the five partial derivatives sum to one and the
  // cotangents to g_out; the centre one follows from the other four
  gq[2] = g_out - ((gq[0] + gq[1]) + (gq[3] + gq[4]));
}

// ------------------------------------------------------------------------------------------------
// Both WENO5 values of one cell and their gradients, sharing the cell's indicator set
// ------------------------------------------------------------------------------------------------
// The left-biased value at face i+1/2 ("up") and the right-biased value at face i-1/2 ("dn") both
// reconstruct in cell i from q_{i-2..i+2}, and their three stencils are the same three cells
// triples with the same target cell: the mirror image of the right-biased stencil set is the
// left-biased one, so the indicators, their reciprocals and the Z ratios r_k = tau / (beta_k + eps)
// are shared and only the linear weights and candidates differ by side (in the up frame:
// d = (1/10, 6/10, 3/10) for up and (3/10, 6/10, 1/10) for dn).  The derivative of tau = |b0 - b2|
// is taken as sign(b0 - b2) in this frame, +1 at zero, for both sides.

// One side from the shared set: the value offset out (= face value - q_i), the cotangents gC of the
// candidates C (times 6, offsets from q_i) and gb of the (times 4) indicators for a unit cotangent.
// rho[k] = r[k] iv[k] (WENO5-Z) is the cell's, shared by both sides.
template <int SCHEME>
FL_HD void weno5_side_vjp(const double f[3], const double r[3], const double iv[3], const double rho[3],
                          double sg, double d0, double d1, double d2, const double C[3], double& out,
                          double gC[3], double gb[3]) {
  const double a0 = d0 * f[0], a1 = d1 * f[1], a2 = d2 * f[2];
  const double S = a0 + a1 + a2;
  const double N = fma(a2, C[2], fma(a1, C[1], a0 * C[0]));
  const double iS6 = fl_rcp(6.0 * S);
  out = N * iS6;
  const double gS = -6.0 * out * iS6;                // -out / S
  const double ga0 = fma(iS6, C[0], gS), ga1 = fma(iS6, C[1], gS), ga2 = fma(iS6, C[2], gS);
  gC[0] = iS6 * a0;
  gC[1] = iS6 * a1;
  gC[2] = iS6 * a2;
  if (SCHEME == FLUID_WENO_JS) {
    // a_k = d_k / e_k^2: da/de = -2 a / e
    gb[0] = -2.0 * ga0 * a0 * r[0];
    gb[1] = -2.0 * ga1 * a1 * r[1];
    gb[2] = -2.0 * ga2 * a2 * r[2];
  } else {
    // a_k = d_k (1 + r_k^2), r_k = tau / e_k: d a_k / d e_k = -2 d_k r_k^2 / e_k, d a_k / d tau =
    // 2 d_k r_k / e_k
    const double gr0 = ga0 * (2.0 * d0) * r[0], gr1 = ga1 * (2.0 * d1) * r[1], gr2 = ga2 * (2.0 * d2) * r[2];
    const double gtau = sg * fma(gr2, iv[2], fma(gr1, iv[1], gr0 * iv[0]));
    gb[0] = fma(-gr0, rho[0], gtau);
    gb[1] = -gr1 * rho[1];
    gb[2] = fma(-gr2, rho[2], -gtau);
  }
}

// up / dn select the values formed; each gradient J (unit cotangent, over q_{i-2..i+2}) sums to
// one, so its centre entry follows from the other four.
//
// With 4 beta_k = (13/3) t_k^2 + s_k^2, d(4 beta_k)/dt_k = T t_k (T = 26/3) and d/ds_k = 2 s_k, and
// t_k, s_k are fixed combinations of the q's, so the indicator part of J is
// sum_k gb_k (T t_k dt_k/dq + 2 s_k ds_k/dq): per stencil point a combination gb_k P_k with
// P_k = T t_k c + 2 s_k c' -- the same six P's for both sides (A: the outer points of stencils 0
// and 2, B: their inner points and stencil 1's two sides), formed once per cell.
template <int SCHEME>
FL_HD void weno5_vjp_cell(const double qin[5], double eps4, bool up, bool dn, double& v_up,
                          double J_up[5], double& v_dn, double J_dn[5]) {
  // shifted by the centre value (see weno5_vjp); q2 = 0
  const double q0 = qin[0] - qin[2], q1 = qin[1] - qin[2], q3 = qin[3] - qin[2], q4 = qin[4] - qin[2];
  // 4 beta_k = (13/3) t_k^2 + s_k^2 of the stencils (i-2..i), (i-1..i+1), (i..i+2) for target i
  const double t0 = fma(-2.0, q1, q0), s0 = fma(-4.0, q1, q0);
  const double t1 = q1 + q3, s1 = q1 - q3;
  const double t2 = fma(-2.0, q3, q4), s2 = fma(-4.0, q3, q4);
  constexpr double K4 = 4.0 * k1312;
  const double b0 = fma(K4 * t0, t0, s0 * s0);
  const double b1 = fma(K4 * t1, t1, s1 * s1);
  const double b2 = fma(K4 * t2, t2, s2 * s2);
  double iv[3], r[3], f[3], rho[3], sg = 1.0;
  iv[0] = fl_rcp(b0 + eps4);
  iv[1] = fl_rcp(b1 + eps4);
  iv[2] = fl_rcp(b2 + eps4);
  if (SCHEME == FLUID_WENO_JS) {
    for (int k = 0; k < 3; ++k) {
      r[k] = iv[k];
      f[k] = iv[k] * iv[k];
      rho[k] = 0.0;
    }
  } else {
    const double db = b0 - b2;
    const double tau = db < 0.0 ? -db : db;
    sg = db < 0.0 ? -1.0 : 1.0;
    for (int k = 0; k < 3; ++k) {
      r[k] = tau * iv[k];
      f[k] = fma(r[k], r[k], 1.0);
      rho[k] = r[k] * iv[k];
    }
  }
  constexpr double T = 2.0 * K4;
  // t0 = q0 - 2 q1, s0 = q0 - 4 q1; t1 = q1 + q3, s1 = q1 - q3; t2 = q4 - 2 q3, s2 = q4 - 4 q3
  const double A0 = fma(T, t0, 2.0 * s0);            // point i-2 (stencil 0)
  const double B0 = fma(-2.0 * T, t0, -8.0 * s0);    // point i-1 (stencil 0)
  const double A1 = fma(T, t1, 2.0 * s1);            // point i-1 (stencil 1)
  const double B1 = fma(T, t1, -2.0 * s1);           // point i+1 (stencil 1)
  const double B2 = fma(-2.0 * T, t2, -8.0 * s2);    // point i+1 (stencil 2)
  const double A2 = fma(T, t2, 2.0 * s2);            // point i+2 (stencil 2)
  if (up) {
    // candidates at i+1/2 times 6: 2 q0 - 7 q1 + 11 q2, -q1 + 5 q2 + 2 q3, 2 q2 + 5 q3 - q4
    const double C[3] = {fma(2.0, q0, -7.0 * q1), fma(2.0, q3, -q1), fma(5.0, q3, -q4)};
    double out, gC[3], gb[3];
    weno5_side_vjp<SCHEME>(f, r, iv, rho, sg, 0.1, 0.6, 0.3, C, out, gC, gb);
    v_up = out + qin[2];
    J_up[0] = fma(2.0, gC[0], gb[0] * A0);
    J_up[1] = fma(-7.0, gC[0], fma(-1.0, gC[1], fma(gb[0], B0, gb[1] * A1)));
    J_up[3] = fma(2.0, gC[1], fma(5.0, gC[2], fma(gb[1], B1, gb[2] * B2)));
    J_up[4] = fma(gb[2], A2, -gC[2]);
    J_up[2] = 1.0 - ((J_up[0] + J_up[1]) + (J_up[3] + J_up[4]));
  }
  if (dn) {
    // candidates at i-1/2 times 6: -q0 + 5 q1 + 2 q2, 2 q1 + 5 q2 - q3, 11 q2 - 7 q3 + 2 q4
    const double C[3] = {fma(5.0, q1, -q0), fma(2.0, q1, -q3), fma(2.0, q4, -7.0 * q3)};
    double out, gC[3], gb[3];
    weno5_side_vjp<SCHEME>(f, r, iv, rho, sg, 0.3, 0.6, 0.1, C, out, gC, gb);
    v_dn = out + qin[2];
    J_dn[0] = fma(gb[0], A0, -gC[0]);
    J_dn[1] = fma(5.0, gC[0], fma(2.0, gC[1], fma(gb[0], B0, gb[1] * A1)));
    J_dn[3] = fma(-7.0, gC[2], fma(-1.0, gC[1], fma(gb[1], B1, gb[2] * B2)));
    J_dn[4] = fma(2.0, gC[2], gb[2] * A2);
    J_dn[2] = 1.0 - ((J_dn[0] + J_dn[1]) + (J_dn[3] + J_dn[4]));
  }
}

// ------------------------------------------------------------------------------------------------
// HLLC along D: cotangents of the left and right primitive states given the flux cotangent
// ------------------------------------------------------------------------------------------------
template <int D>
FL_HD void hllc_vjp(const double wl[5], const double wr[5], const Phys& ph, const double gF[5],
                    double gwl[5], double gwr[5]) {
  // ---- forward (same operations as hllc<D>) ----
  const double rL = wl[0], pL = wl[4], rR = wr[0], pR = wr[4];
  const double unL = wl[1 + D], unR = wr[1 + D];
  const double q2L = wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3];
  const double q2R = wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3];
  const double EL = pL * ph.igm1 + 0.5 * rL * q2L;
  const double ER = pR * ph.igm1 + 0.5 * rR * q2R;
  const double qL = fl_rsqrt(rL), qR = fl_rsqrt(rR);
  const double sL = rL * qL, sR = rR * qR;
  const double irL = qL * qL, irR = qR * qR;
  const double cL = fl_sqrt(ph.gamma * pL * irL), cR = fl_sqrt(ph.gamma * pR * irR);
  const double isum = fl_rcp(sL + sR);
  double ut[3];
  for (int c = 0; c < 3; ++c) ut[c] = (sL * wl[1 + c] + sR * wr[1 + c]) * isum;
  const double HL = (EL + pL) * irL, HR = (ER + pR) * irR;
  const double Ht = (sL * HL + sR * HR) * isum;
  const double ct = fl_sqrt(ph.gm1 * (Ht - 0.5 * (ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2])));
  const double utn = ut[D];
  const double aL = unL - cL, bL = utn - ct;
  const bool selL = aL <= bL;
  const double SL = selL ? aL : bL;
  const double aR = unR + cR, bR = utn + ct;
  const bool selR = aR >= bR;
  const double SR = selR ? aR : bR;
  const double mL = rL * (SL - unL), mR = rR * (SR - unR);
  const double Nn = pR - pL + unL * mL - unR * mR;
  const double Dd = mL - mR;
  const double iDd = fl_rcp(Dd);
  const double Ss = Nn * iDd;
  const bool left = fl_nonneg(SL) || fl_nonneg(Ss);
  const bool star = left ? !fl_nonneg(SL) : fl_pos(SR);
  const double r = left ? rL : rR, p = left ? pL : pR, E = left ? EL : ER;
  const double un = left ? unL : unR, S = left ? SL : SR, m = left ? mL : mR;
  const double ir = left ? irL : irR;
  const double* w = left ? wl : wr;
  const double u[3] = {w[1], w[2], w[3]};
  const double mn = r * un;

  // ---- reverse ----
  // cotangents of the selected side's quantities
  double g_r = 0.0, g_p = 0.0, g_E = 0.0, g_u[3] = {0.0, 0.0, 0.0}, g_S = 0.0, g_m = 0.0;
  double g_ir = 0.0, g_Ss = 0.0;
  // Euler flux of the selected side: F0 = mn, F_c = mn u_c (+ p), F4 = un (E + p)
  double g_mn = gF[0];
  for (int c = 0; c < 3; ++c) {
    g_mn += gF[1 + c] * u[c];
    g_u[c] += gF[1 + c] * mn;
  }
  g_p += gF[1 + D];
  g_u[D] += gF[4] * (E + p);
  g_E += gF[4] * un;
  g_p += gF[4] * un;
  if (star) {
    const double d = S - Ss;
    const double q = fl_rcp(d);
    const double fac = m * q;
    const double A = E * ir, B = Ss - un, Cc = fac * Ss + p * q;
    const double Es = fac * A + B * Cc;
    double dU[5];
    dU[0] = fac - r;
    for (int c = 0; c < 3; ++c) dU[1 + c] = (fac - r) * u[c];
    dU[1 + D] = fac * Ss - r * un;
    dU[4] = Es - E;
    for (int v = 0; v < 5; ++v) g_S += gF[v] * dU[v];
    double g_fac = 0.0;
    // dU0 = fac - r
    g_fac += gF[0] * S;
    g_r -= gF[0] * S;
    for (int c = 0; c < 3; ++c) {
      const double gd = gF[1 + c] * S;
      if (c == D) {
        g_fac += gd * Ss;
        g_Ss += gd * fac;
        g_r -= gd * un;
        g_u[D] -= gd * r;
      } else {
        g_fac += gd * u[c];
        g_r -= gd * u[c];
        g_u[c] += gd * (fac - r);
      }
    }
    const double gEs = gF[4] * S;
    g_E -= gF[4] * S;
    g_fac += gEs * A;
    const double gA = gEs * fac, gB = gEs * Cc, gCc = gEs * B;
    g_fac += gCc * Ss;
    g_Ss += gCc * fac;
    g_p += gCc * q;
    double g_q = gCc * p;
    g_Ss += gB;
    g_u[D] -= gB;
    g_E += gA * ir;
    g_ir += gA * E;
    g_m += g_fac * q;
    g_q += g_fac * m;
    const double g_d = -g_q * q * q;
    g_S += g_d;
    g_Ss -= g_d;
  }
  // mn = r un
  g_r += g_mn * un;
  g_u[D] += g_mn * r;

  // distribute the selected side's cotangents onto L / R intermediates
  double gSL = 0.0, gSR = 0.0, gmL = 0.0, gmR = 0.0, gEL = 0.0, gER = 0.0, girL = 0.0, girR = 0.0;
  for (int v = 0; v < 5; ++v) {
    gwl[v] = 0.0;
    gwr[v] = 0.0;
  }
  double* gw = left ? gwl : gwr;
  gw[0] += g_r;
  gw[4] += g_p;
  for (int c = 0; c < 3; ++c) gw[1 + c] += g_u[c];
  if (left) {
    gEL += g_E; gSL += g_S; gmL += g_m; girL += g_ir;
  } else {
    gER += g_E; gSR += g_S; gmR += g_m; girR += g_ir;
  }
  // Ss = Nn / Dd
  const double gNn = g_Ss * iDd, gDd = -g_Ss * Ss * iDd;
  gwr[4] += gNn;
  gwl[4] -= gNn;
  gwl[1 + D] += gNn * mL;
  gmL += gNn * unL + gDd;
  gwr[1 + D] -= gNn * mR;
  gmR += -gNn * unR - gDd;
  // m = rho (S - un)
  gwl[0] += gmL * (SL - unL);
  gSL += gmL * rL;
  gwl[1 + D] -= gmL * rL;
  gwr[0] += gmR * (SR - unR);
  gSR += gmR * rR;
  gwr[1 + D] -= gmR * rR;
  // Einfeldt bounds
  double gutn = 0.0, gct = 0.0, gcL = 0.0, gcR = 0.0;
  if (selL) { gwl[1 + D] += gSL; gcL -= gSL; } else { gutn += gSL; gct -= gSL; }
  if (selR) { gwr[1 + D] += gSR; gcR += gSR; } else { gutn += gSR; gct += gSR; }
  // ct = sqrt(gm1 (Ht - |ut|^2 / 2))
  double gut[3] = {0.0, 0.0, 0.0};
  gut[D] += gutn;
  const double gX = ct > 0.0 ? 0.5 * gct * fl_rcp(ct) : 0.0;
  const double gHt = ph.gm1 * gX;
  for (int c = 0; c < 3; ++c) gut[c] -= ph.gm1 * gX * ut[c];
  // Ht = (sL HL + sR HR) isum and ut_c = (sL uL_c + sR uR_c) isum: with the weights
  // wL = sL isum, wR = sR isum, d/d sL = isum (HL, uL_c) and d/d isum = (sL + sR) (Ht, ut_c)
  const double wL = sL * isum, wR = sR * isum;
  const double gHL = gHt * wL, gHR = gHt * wR;
  double guL = gHt * HL, guR = gHt * HR, gdot = gHt * Ht;
  for (int c = 0; c < 3; ++c) {
    guL = fma(gut[c], wl[1 + c], guL);
    guR = fma(gut[c], wr[1 + c], guR);
    gdot = fma(gut[c], ut[c], gdot);
    gwl[1 + c] = fma(gut[c], wL, gwl[1 + c]);
    gwr[1 + c] = fma(gut[c], wR, gwr[1 + c]);
  }
  double gsL = guL * isum, gsR = guR * isum;
  const double gisum = gdot * (sL + sR);
  // H = (E + p) ir
  gEL += gHL * irL;
  gwl[4] += gHL * irL;
  girL += gHL * (EL + pL);
  gER += gHR * irR;
  gwr[4] += gHR * irR;
  girR += gHR * (ER + pR);
  // isum = 1 / (sL + sR)
  const double gsum = -gisum * isum * isum;
  gsL += gsum;
  gsR += gsum;
  // c = sqrt(gamma p ir)
  const double gYL = 0.5 * gcL * fl_rcp(cL), gYR = 0.5 * gcR * fl_rcp(cR);
  gwl[4] += gYL * ph.gamma * irL;
  girL += gYL * ph.gamma * pL;
  gwr[4] += gYR * ph.gamma * irR;
  girR += gYR * ph.gamma * pR;
  // s = sqrt(rho), ir = 1 / rho
  gwl[0] += gsL * 0.5 * qL - girL * irL * irL;
  gwr[0] += gsR * 0.5 * qR - girR * irR * irR;
  // E = p / (gamma - 1) + rho |u|^2 / 2
  gwl[4] += gEL * ph.igm1;
  gwl[0] += gEL * 0.5 * q2L;
  gwr[4] += gER * ph.igm1;
  gwr[0] += gER * 0.5 * q2R;
  for (int c = 0; c < 3; ++c) {
    gwl[1 + c] += gEL * rL * wl[1 + c];
    gwr[1 + c] += gER * rR * wr[1 + c];
  }
}

// ------------------------------------------------------------------------------------------------
// dissipative face flux: cotangents of the stencil inputs given the cotangent gFd of
// (tau_0D, tau_1D, tau_2D, energy)
// ------------------------------------------------------------------------------------------------
template <int D>
FL_HD void visc_face_vjp(const double vel[3][4], const double T[4], const double gd[3][4],
                         const double gb[3][4], int ndim, double mfa, const Phys& ph,
                         const double gFd[4], double gvel[3][4], double gT[4], double gGD[3],
                         double gGB[3]) {
  const double ci[4] = {-k16th, 9.0 * k16th, 9.0 * k16th, -k16th};
  const double cn[4] = {k24th * mfa, -27.0 * k24th * mfa, 27.0 * k24th * mfa, -k24th * mfa};
  double vf[3], Gf[3][3];
  for (int c = 0; c < 3; ++c) {
    vf[c] = interp4(vel[c]);
    Gf[c][D] = dnorm4(vel[c], mfa * k24th);
  }
  const double Tf = interp4(T);
  const double dT = dnorm4(T, mfa * k24th);
  bool act[3];
  for (int b = 0; b < 3; ++b) {
    act[b] = b != D && b < ndim;
    if (b == D) continue;
    Gf[D][b] = act[b] ? interp4(gd[b]) : 0.0;
    Gf[b][b] = act[b] ? interp4(gb[b]) : 0.0;
  }
  const double div = Gf[0][0] + Gf[1][1] + Gf[2][2];
  const double mu = viscosity(Tf, ph);
  const double lam = mu * ph.lam_fac;
  double tau[3];
  for (int c = 0; c < 3; ++c) {
    if (c == D) tau[c] = mu * (Gf[D][D] + Gf[D][D]) - (2.0 / 3.0) * mu * div;
    else tau[c] = mu * (Gf[c][D] + Gf[D][c]);
  }
  // reverse
  double gtau[3], gvf[3], gG[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int c = 0; c < 3; ++c) {
    gtau[c] = gFd[c] + gFd[3] * vf[c];
    gvf[c] = gFd[3] * tau[c];
  }
  const double glam = gFd[3] * dT;
  const double gdT = gFd[3] * lam;
  double gmu = glam * ph.lam_fac, gdiv = 0.0;
  for (int c = 0; c < 3; ++c) {
    if (c == D) {
      gmu += gtau[c] * (2.0 * Gf[D][D] - (2.0 / 3.0) * div);
      gG[D][D] += gtau[c] * 2.0 * mu;
      gdiv -= gtau[c] * (2.0 / 3.0) * mu;
    } else {
      gmu += gtau[c] * (Gf[c][D] + Gf[D][c]);
      gG[c][D] += gtau[c] * mu;
      gG[D][c] += gtau[c] * mu;
    }
  }
  for (int c = 0; c < 3; ++c) gG[c][c] += gdiv;
  const double gTf = gmu * viscosity_dT(Tf, mu, ph);
  for (int k = 0; k < 4; ++k) {
    gT[k] = gTf * ci[k] + gdT * cn[k];
    for (int c = 0; c < 3; ++c) gvel[c][k] = gvf[c] * ci[k] + gG[c][D] * cn[k];
  }
  // the tangential gradients enter only through their four-point interpolations Gf[D][b] and
  // Gf[b][b]: their cotangents, which the stencil cells receive times the interpolation weights
  // (-1, 9, 9, -1) / 16
  for (int b = 0; b < 3; ++b) {
    gGD[b] = act[b] ? gG[D][b] : 0.0;
    gGB[b] = act[b] ? gG[b][b] : 0.0;
  }
}

// ------------------------------------------------------------------------------------------------
// conservative -> primitive (rho, u, v, w, p, T): cotangent of U given the cotangent of W
// ------------------------------------------------------------------------------------------------
FL_HD void prim_vjp(const double U[5], const Phys& ph, const double gW[6], double gU[5]) {
  const double r = U[0];
  const double ir = fl_rcp(r);
  const double u[3] = {U[1] * ir, U[2] * ir, U[3] * ir};
  const double p = ph.gm1 * (U[4] - 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  // T = p / (rho R)
  const double gp = gW[4] + gW[5] * ir * ph.iR;
  double gr = gW[0] - gW[5] * p * ir * ir * ph.iR;
  // p = (gamma - 1)(E - |m|^2 / (2 rho))
  gU[4] = ph.gm1 * gp;
  double q2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    gU[1 + c] = gW[1 + c] * ir - ph.gm1 * u[c] * gp;
    gr -= gW[1 + c] * u[c] * ir;
    q2 += u[c] * u[c];
  }
  gr += 0.5 * ph.gm1 * q2 * gp;
  gU[0] = gr;
}

// ------------------------------------------------------------------------------------------------
// wall halo maps of axis a (velocity mirrored; isothermal T_g = 2 T_w - T, p_g = p,
// rho_g = p / (R T_g); porous adds 2 v_w to the wall-normal component): cotangent of the source
// primitives w (rho, u, v, w, p, T) given the ghost cotangent; g_vw receives d/d v_w
// ------------------------------------------------------------------------------------------------
FL_HD void wall_map_vjp(const double w[6], int kind, double Tw, int a, const Phys& ph,
                        const double gg[6], double gw[6], double* g_vw) {
  for (int v = 0; v < 6; ++v) gw[v] = 0.0;
  gw[1] = -gg[1];
  gw[2] = -gg[2];
  gw[3] = -gg[3];
  *g_vw = 0.0;
  if (kind == FLUID_BC_ADIABATIC) {
    gw[0] = gg[0];
    gw[4] = gg[4];
    gw[5] = gg[5];
    return;
  }
  const double Tg = 2.0 * Tw - w[5];
  // rho_g = p / (R Tg): d/dp = 1/(R Tg), d/dT = p / (R Tg^2)
  gw[4] = gg[4] + gg[0] / (ph.R * Tg);
  gw[5] = -gg[5] + gg[0] * w[4] / (ph.R * Tg * Tg);
  if (kind == FLUID_BC_POROUS) *g_vw = 2.0 * gg[1 + a];
}

}  // namespace fl
