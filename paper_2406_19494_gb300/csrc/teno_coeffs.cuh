// Generated by gen_teno_coeffs.py (sympy, from the Jiang-Shu definition); do not edit.
#pragma once
#ifndef FL_HD
#define FL_HD __host__ __device__ __forceinline__
#endif
namespace fl {
namespace teno {
// beta4_form: cells (0, 1, 2, 3) (offsets from the target cell), e[j-1] = q_{s_j} - q_{s_0}, j = 1 .. 3:
// beta = sum_{j<=k} c_jk e_j e_k / 240, grouped by rows: sum_j e_j (sum_{k>=j} c_jk e_k / 240)
// (the coefficients c_jk / 240 rounded to FP64).
FL_HD double beta4_form(const double e[3]) {
  const double r0 = fma(19.341666666666665, e[2], fma(-71.85833333333333, e[1], 45.84583333333333 * e[0]));
  const double r1 = fma(-16.175, e[2], 29.345833333333335 * e[1]);
  const double r2 = 2.279166666666667 * e[2];
  return fma(e[2], r2, fma(e[1], r1, e[0] * r0));
}

// beta6_pair: 6 times the TENO6 measure of the window q[0..5] (cells (-2, -1, 0, 1, 2, 3) around the target cell)
// and of its mirror image (q[5..0]): bL = S + T + 2 X, bR = S + T - 2 X with u_j = q_j + q_{5-j},
// v_j = q_j - q_{5-j}, a_k = u_k - u_0; coefficients are 6 times the exact rationals, rounded
// to FP64 (the factor is the 6 of tau6 = |beta6 - (beta1 + beta2 + 4 beta0) / 6|).
FL_HD void beta6_pair(const double q[6], double& bL, double& bR) {
  // a_k from differences of neighbouring values, exact for close values, never from the sums u_k
  const double a1 = (q[1] - q[0]) + (q[4] - q[5]), a2 = (q[2] - q[0]) + (q[3] - q[5]);
  const double v0 = q[0] - q[5], v1 = q[1] - q[4], v2 = q[2] - q[3];
  const double S = fma(a1, fma(-30.67142857142857, a2, 21.70357142857143 * a1), (11.023809523809524 * a2) * a2);
  const double t0 = fma(163.75555555555556, v2, fma(-81.77757936507936, v1, 8.147718253968254 * v0));
  const double t1 = fma(-869.831746031746, v2, 213.36994047619046 * v1);
  const double T = fma(v2, 899.3587301587302 * v2, fma(v1, t1, v0 * t0));
  const double x1 = fma(-80.88541666666667, v2, fma(45.348958333333336, v1, -10.132291666666667 * v0));
  const double x2 = fma(57.423611111111114, v2, fma(-31.899305555555557, v1, 6.854861111111111 * v0));
  const double X2 = fma(a2, x2, a1 * x1);
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
