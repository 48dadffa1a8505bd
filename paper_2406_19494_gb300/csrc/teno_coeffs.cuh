// Generated by gen_teno_coeffs.py (sympy, from the Jiang-Shu definition); do not edit.
#pragma once
#ifndef FL_HD
#define FL_HD __host__ __device__ __forceinline__
#endif
namespace fl {
namespace teno {
// beta4_diff: beta4 of cells (0, 1, 2, 3) around target 0 in the consecutive differences
// of those cells, d[0..2]; coefficients are the exact rationals rounded to FP64.
FL_HD double beta4_diff(double d0, double d1, double d2) {
  const double r0 = fma(7.725, d2, fma(-21.616666666666667, d1, 8.779166666666667 * d0));
  const double r1 = fma(-11.616666666666667, d2, 15.45 * d1);
  return fma(d2, 2.279166666666667 * d2, fma(d1, r1, d0 * r0));
}

// beta6_pair_diff: 6 beta6 of the window q[0..5] and of its mirror image from the window's
// consecutive differences d[0..4]: bL = S + T + 2 X, bR = S + T - 2 X with u0 = d0 + d4,
// u1 = d1 + d3, u2 = d2, w0 = d0 - d4, w1 = d1 - d3 (the reversal keeps u and negates w).
FL_HD void beta6_pair_diff(const double d[5], double& bL, double& bR) {
  const double u0 = d[0] + d[4], u1 = d[1] + d[3], u2 = d[2];
  const double w0 = d[0] - d[4], w1 = d[1] - d[3];
  const double s0 = fma(98.2734126984127, u2, fma(-65.48214285714286, u1, 8.147718253968254 * u0));
  const double s1 = fma(-426.59603174603177, u2, 139.74007936507937 * u1);
  const double S = fma(u2, 333.02261904761906 * u2, fma(u1, s1, u0 * s0));
  const double T = fma(w1, 11.023809523809524 * w1, w0 * fma(-8.623809523809523, w1, 2.0559523809523808 * w0));
  const double x0 = fma(-6.854861111111111, w1, 3.2774305555555556 * w0);
  const double x1 = fma(25.044444444444444, w1, -10.172222222222222 * w0);
  const double x2 = fma(-32.37916666666667, w1, 13.289583333333333 * w0);
  const double X2 = fma(u2, x2, fma(u1, x1, u0 * x0));
  const double ST = S + T;
  bL = ST + X2;
  bR = ST - X2;
}

// adaptive cut-off as thresholds on the smallest sensor eta: C_T = 10^-k for eta >= eta_k
// (k = 10, 9, 8; else 10^-7), eta_k = C_r t_k with t_k^4 (5 - 4 t_k) = 1 - (alpha1 - k) / alpha2
constexpr double kCutEta8 = 0.1422785499942228;   // g = 2/7
constexpr double kCutEta9 = 0.18020361976189328;   // g = 4/7
constexpr double kCutEta10 = 0.2155369674668411;   // g = 6/7

}  // namespace teno
}  // namespace fl
