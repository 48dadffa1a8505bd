// Host build of the TENO6-A face arithmetic of the FP64 kernels (teno_math.cuh and the generated
// teno_coeffs.cuh), for a CPU check against the oracle: reads six-cell windows q[0..5] from stdin,
// forms the cut-off from the sensor levels of cells 1..4 as the face kernel does, and prints the left-
// and right-biased states of the face between cells 2 and 3.
#include <cmath>
#include <algorithm>
#include <cstdio>

#include "../../paper_2406_19494_gb300/csrc/teno_math.cuh"

int main() {
  double omega[4][16];
  for (int i = 0; i < 64; ++i) fl::teno::weight_entry(i, omega);
  double q[6];
  while (std::scanf("%lf %lf %lf %lf %lf %lf", q, q + 1, q + 2, q + 3, q + 4, q + 5) == 6) {
    int level = 3;
    for (int j = 1; j <= 4; ++j) level = std::min(level, fl::teno::sensor_level(q[j] - q[j - 1], q[j + 1] - q[j]));
    const double ct = fl::teno::cutoff_of_level(level);
    double b3c[3] = {fl::weno_B(q[1], q[2], q[3]), fl::weno_C(q[2], q[3], q[4]), fl::weno_A(q[0], q[1], q[2])};
    // 13/12 t^2 of the three-cell stencils centred at cells 2 and 3, as the march carries them
    const double ta = std::fma(-2.0, q[2], q[1]) + q[3], tb = std::fma(-2.0, q[3], q[2]) + q[4];
    double kk[2] = {fl::k1312 * ta * ta, fl::k1312 * tb * tb};
    double wl, wr;
    double i3c[3] = {fl::teno::rcp6(b3c[0]), fl::teno::rcp6(b3c[1]), fl::teno::rcp6(b3c[2])};
    const double d[5] = {q[1] - q[0], q[2] - q[1], q[3] - q[2], q[4] - q[3], q[5] - q[4]};
    fl::teno::face_states(q, d, ct, b3c, i3c, kk, omega, wl, wr);
    std::printf("%.17g %.17g %.17g\n", wl, wr, ct);
  }
  return 0;
}
