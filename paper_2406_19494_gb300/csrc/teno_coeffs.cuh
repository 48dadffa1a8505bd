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

}  // namespace teno
}  // namespace fl
