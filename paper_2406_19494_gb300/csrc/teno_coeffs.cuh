// Generated by gen_teno_coeffs.py (sympy, from the Jiang-Shu definition); do not edit.
#pragma once
#ifndef FL_HD
#define FL_HD __host__ __device__ __forceinline__
#endif
namespace fl {
namespace teno {
// beta4_form: cells (0, 1, 2, 3) (offsets from the target cell), e[j-1] = q_{s_j} - q_{s_0}, j = 1 .. 3:
// beta = sum_{j<=k} c_jk e_j e_k / 240, grouped by rows: sum_j e_j (sum_{k>=j} c_jk e_k).
FL_HD double beta4_form(const double e[3]) {
  const double r0 = fma(4642.0, e[2], fma(-17246.0, e[1], 11003.0 * e[0]));
  const double r1 = fma(-3882.0, e[2], 7043.0 * e[1]);
  const double r2 = 547.0 * e[2];
  return (fma(e[2], r2, fma(e[1], r1, e[0] * r0))) * (1.0 / 240.0);
}

// beta6_form: cells (-2, -1, 0, 1, 2, 3) (offsets from the target cell), e[j-1] = q_{s_j} - q_{s_0}, j = 1 .. 5:
// beta = sum_{j<=k} c_jk e_j e_k / 120960, grouped by rows: sum_j e_j (sum_{k>=j} c_jk e_k).
FL_HD double beta6_form(const double e[5]) {
  const double r0 = fma(1325006.0, e[4], fma(-7727988.0, e[3], fma(17905032.0, e[2], fma(-20427884.0, e[1], 5653317.0 * e[0]))));
  const double r1 = fma(-2792660.0, e[4], fma(15929912.0, e[3], fma(-35817664.0, e[2], 19510972.0 * e[1])));
  const double r2 = fma(2863984.0, e[4], fma(-15880404.0, e[3], 17195652.0 * e[2]));
  const double r3 = fma(-1429976.0, e[4], 3824847.0 * e[3]);
  const double r4 = 139633.0 * e[4];
  return (fma(e[4], r4, fma(e[3], r3, fma(e[2], r2, fma(e[1], r1, e[0] * r0))))) * (1.0 / 120960.0);
}

// beta6_pair: the TENO6 measure of the window q[0..5] (cells (-2, -1, 0, 1, 2, 3) around the target cell)
// and of its mirror image (q[5..0]): bL = S + T + 2 X, bR = S + T - 2 X with u_j = q_j + q_{5-j},
// v_j = q_j - q_{5-j}, a_k = u_k - u_0; coefficients are the exact rationals rounded to FP64.
FL_HD void beta6_pair(const double q[6], double& bL, double& bR) {
  // a_k from differences of neighbouring values, exact for close values, never from the sums u_k
  const double a1 = (q[1] - q[0]) + (q[4] - q[5]), a2 = (q[2] - q[0]) + (q[3] - q[5]);
  const double v0 = q[0] - q[5], v1 = q[1] - q[4], v2 = q[2] - q[3];
  const double S = fma(a1, fma(-5.1119047619047615, a2, 3.6172619047619046 * a1), (1.8373015873015872 * a2) * a2);
  const double t0 = fma(27.29259259259259, v2, fma(-13.629596560846561, v1, 1.3579530423280424 * v0));
  const double t1 = fma(-144.97195767195768, v2, 35.561656746031744 * v1);
  const double T = fma(v2, 149.89312169312169 * v2, fma(v1, t1, v0 * t0));
  const double x1 = fma(-13.480902777777779, v2, fma(7.558159722222222, v1, -1.6887152777777779 * v0));
  const double x2 = fma(9.570601851851851, v2, fma(-5.316550925925926, v1, 1.1424768518518518 * v0));
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
