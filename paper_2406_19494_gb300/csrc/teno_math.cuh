// TENO6-A reconstruction (the paper's channel scheme, Sec. 3.1), FP64.  The paper names the
// scheme and cites its solver for it; the definition used here is the published one (Fu, Hu &
// Adams 2016 for TENO6, 2017 for the adaptive cut-off):
//   left-biased value at i+1/2 from q_{i-2} .. q_{i+3}; candidate stencils S0 = (i-1, i, i+1),
//   S1 = (i, i+1, i+2), S2 = (i-2, i-1, i), S3 = (i, .., i+3) with the cell-average candidates
//   p_k and the sixth-order linear weights d = (9/20, 3/10, 1/20, 1/5); Jiang-Shu smoothness
//   measures beta_k and beta6 of the six-cell stencil, tau6 = |beta6 - (beta1 + beta2 + 4 beta0)/6|,
//   gamma_k = (1 + tau6 / (beta_k + 1e-40))^6; a stencil is kept unless gamma_k / sum gamma < C_T,
//   and the value is sum d_k p_k over the kept stencils divided by their sum of d_k.
//   Adaptive C_T = 10^-floor(10.5 - 3.5 (1 - g(m))), g = (1 - m)^4 (1 + 4 m),
//   m = 1 - min(1, eta / 0.25), eta the smallest scale sensor
//   (2 |D+ D-| + e) / (D+^2 + D-^2 + e) (D+- the differences to the two neighbours,
//   e = 0.9 * 0.25 * 1e-6 / 0.75) over the cells i-1 .. i+2.
// The right-biased value at i+1/2 is the left-biased value of the mirrored stencil; both use the
// same four cells for the sensor, so one cut-off serves both states of a face.
#pragma once

#include "flux_math.cuh"
#include "teno_coeffs.cuh"

namespace fl {
namespace teno {

constexpr double kEps = 1e-40;
constexpr double kSensorE = 0.9 * 0.25 * 1e-6 / 0.75;

// 1/y for gamma_k, which only decides the cut-off: one second-order Newton step from the hardware
// estimate of rcp.approx.ftz.f64, relative error the square of the estimate's (about 2^-34 or
// smaller; the third-order fl_rcp squares it once more).  A keep decision can differ from exact
// division only where gamma_k / sum gamma is within about 1e-10 relative of C_T.
FL_HD double rcp_decide(double y) {
#ifdef __CUDA_ARCH__
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(y));
  return fma(r, fma(-y, r, 1.0), r);
#else
  return 1.0 / y;
#endif
}

// Cut-off level of a cell from the differences dm, dp to its two neighbours: how many of the
// thresholds kCutEta8 < kCutEta9 < kCutEta10 (teno_coeffs.cuh) its scale sensor
// eta = N / D = (2 |dp dm| + e) / (dp^2 + dm^2 + e) reaches, decided as N >= eta_k D (D > 0)
// without forming the quotient.  The adaptive C_T = 10^-floor(alpha1 - alpha2 (1 - g(m))) of a
// stencil (C_r = 0.25, alpha1 = 10.5, alpha2 = 3.5) is a step function of its smallest sensor,
// since g grows with eta, so it follows from the smallest level of the stencil's cells.
FL_HD int sensor_level(double dm, double dp) {
  const double N = fma(2.0, fabs(dp * dm), kSensorE);
  const double Dn = fma(dp, dp, fma(dm, dm, kSensorE));
  return (fma(-kCutEta8, Dn, N) >= 0.0 ? 1 : 0) + (fma(-kCutEta9, Dn, N) >= 0.0 ? 1 : 0) +
         (fma(-kCutEta10, Dn, N) >= 0.0 ? 1 : 0);
}

// C_T of a level: 1e-7, 1e-8, 1e-9, 1e-10
FL_HD double cutoff_of_level(int level) {
  return level >= 3 ? 1e-10 : (level == 2 ? 1e-9 : (level == 1 ? 1e-8 : 1e-7));
}

// linear weights d_k = (9/20, 3/10, 1/20, 1/5) (sixth-order combination of the four candidates)
FL_HD double lin_weight(int k) { return k == 0 ? 0.45 : (k == 1 ? 0.3 : (k == 2 ? 0.05 : 0.2)); }

// Normalised weights of the kept stencils for each keep mask (bit k set: stencil k kept):
// omega[k][mask] = d_k / sum of the kept d_j, 0 for a cut stencil (mask 0 cannot occur: the
// largest gamma_k / sum gamma is at least 1/4), times the common factor of candidate k's
// coefficients (1/6 for the three-cell candidates, 1/12 for the four-cell one), which the
// candidates below leave out.  Entry i of the 64 is written by call i.
FL_HD void weight_entry(int i, double omega[4][16]) {
  const int k = i >> 4, mask = i & 15;
  double den = 0.0;
  for (int j = 0; j < 4; ++j)
    if ((mask >> j) & 1) den += lin_weight(j);
  omega[k][mask] = ((mask >> k) & 1) ? lin_weight(k) / (den * (k < 3 ? 6.0 : 12.0)) : 0.0;
}

// TENO6 value from the candidates p_k (times 6, the four-cell one times 12), the three-cell
// smoothness measures b_k and i_k = rcp6(b_k) of all four (b6 = 6 beta6): stencil k is kept
// unless gamma_k / sum gamma < C_T, and the value is the kept candidates' combination with the
// normalised weights of omega (weight_entry)
// 1 / (6 (beta + eps)), the factor of tau in gamma_k
FL_HD double rcp6(double beta) { return rcp_decide(fma(6.0, beta, 6.0 * kEps)); }

FL_HD double combine(double p0, double p1, double p2, double p3, double b0, double b1, double b2,
                     double i0, double i1, double i2, double i3, double b6, double ct,
                     const double (*omega)[16]) {
  // b6 is 6 beta6 (beta6_pair), so tau = 6 tau6 and gamma_k = (1 + tau / (6 (beta_k + eps)))^6;
  // i_k = rcp6(beta_k)
  const double tau = fabs(b6 - fma(4.0, b0, b1 + b2));
  double g[4];
  const double ik[4] = {i0, i1, i2, i3};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double x = fma(tau, ik[k], 1.0);
    const double x2 = x * x;
    g[k] = x2 * x2 * x2;
  }
  const double thr = ct * ((g[0] + g[1]) + (g[2] + g[3]));
  const int mask = (g[0] < thr ? 0 : 1) | (g[1] < thr ? 0 : 2) | (g[2] < thr ? 0 : 4) | (g[3] < thr ? 0 : 8);
  return fma(omega[3][mask], p3, fma(omega[2][mask], p2, fma(omega[1][mask], p1, omega[0][mask] * p0)));
}

// Both states of the face a+1/2 from q[0..5] = q_{a-2} .. q_{a+3} and the window's consecutive
// differences d[0..4] (d_j = q[j+1] - q[j]; the march carries d[0..3] and forms d[4]) while
// marching along +D.
//   * the candidates are written as offsets from 6 q_a (6 q_{a+1} for the mirrored stencil), the
//     smoothness measures in the differences (beta4_diff, beta6_pair_diff);
//   * the left state's central and downwind candidates are the right state's downwind and central
//     ones (the same quadratics through cells a-1..a+1 and a..a+2, at the same point);
//   * the right state's three-cell measures (B of the stencil centred at a+1, A at a, C at a+2) are
//     the next face's left-state measures (B at a+1, C at a+2, A at a): b3c carries them as
//     (beta0, beta1, beta2) of that next left state, and kk the 13/12 t^2 parts of the stencils
//     centred at a and a+1.
// On entry b3c holds this face's left-state (beta0, beta1, beta2) and i3c their rcp6; on exit the
// next face's.
FL_HD void face_states(const double q[6], const double d[5], double ct, double b3c[3], double i3c[3],
                       double kk[2], const double (*omega)[16], double& wl, double& wr) {
  // candidates times 6 (three cells) and 12 (four cells); the factors are in omega
  const double q6 = 6.0 * q[2], r6 = 6.0 * q[3];
  const double pc = fma(2.0, d[2], d[1]) + q6;                  // cells a-1..a+1
  const double pd = fma(4.0, d[2], -d[3]) + q6;                 // cells a..a+2
  const double pu = fma(5.0, d[1], -2.0 * d[0]) + q6;
  const double p4 = fma(9.0, d[2], fma(-4.0, d[3], d[4])) + 2.0 * q6;
  // 6 beta6 of the window and of its mirror image together (the reversal negates the odd part)
  double b6l, b6r;
  beta6_pair_diff(d, b6l, b6r);
  wl = combine(pc, pd, pu, p4, b3c[0], b3c[1], b3c[2], i3c[0], i3c[1], i3c[2],
               rcp6(beta4_diff(d[2], d[3], d[4])), b6l, ct, omega);
  // right state: the mirrored stencil q'_j = q[5 - j]
  const double ru = fma(-5.0, d[3], 2.0 * d[4]) + r6;
  const double r4 = fma(-9.0, d[2], fma(4.0, d[1], -d[0])) + 2.0 * r6;
  // three-cell measures K + s^2 / 4 with K = 13/12 t^2 of the stencil: K of the stencils centred at
  // a and a+1 carry over from the previous face (kk), the one centred at a+2 is new
  const double t2 = d[4] - d[3];
  const double K2 = k1312 * t2 * t2;
  const double sB = d[2] + d[3], sC = fma(3.0, d[2], -d[1]), sA = fma(-3.0, d[3], d[4]);
  const double rb0 = fma(0.25 * sB, sB, kk[1]);             // B of (q2, q3, q4)
  const double rb1 = fma(0.25 * sC, sC, kk[0]);             // C of (q1, q2, q3)
  const double rb2 = fma(0.25 * sA, sA, K2);                // A of (q3, q4, q5)
  kk[0] = kk[1];
  kk[1] = K2;
  const double ib0 = rcp6(rb0), ib1 = rcp6(rb1), ib2 = rcp6(rb2);
  wr = combine(pd, pc, ru, r4, rb0, rb1, rb2, ib0, ib1, ib2, rcp6(beta4_diff(d[2], d[1], d[0])), b6r,
               ct, omega);
  // next face's left state: beta0 = B at a+1 (rb0), beta1 = C at a+2 (rb2's stencil), beta2 = A at
  // a (rb1's), with their reciprocal factors
  b3c[0] = rb0;
  b3c[1] = rb2;
  b3c[2] = rb1;
  i3c[0] = ib0;
  i3c[1] = ib2;
  i3c[2] = ib1;
}

}  // namespace teno
}  // namespace fl
