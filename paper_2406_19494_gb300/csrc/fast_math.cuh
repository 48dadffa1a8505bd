// Reciprocal, reciprocal square root and square root as the FP64 kernels compute them: one
// Newton-Raphson step of third order from the hardware estimate, checked on the GPU against CUDA's
// IEEE division and square root (fluid_check_rcp, fluid_check_sqrt).  Host code (the
// host-compiled checks of the adjoint) uses the C library.
#pragma once

#include <cmath>

#ifndef FL_HD
#define FL_HD __host__ __device__ __forceinline__
#endif

namespace fl {

// Reciprocal square root by one step of the third-order iteration for x^{-1/2} from the hardware
// estimate of the PTX instruction rsqrt.approx.ftz.f64: with e = 1 - x y^2 the exact value is
// y (1 - e)^{-1/2} = y (1 + e/2 + 3 e^2/8 + O(e^3)), so the step cubes the relative error.  For
// positive normal x the result is within a few ulp of 1/sqrt(x) (checked against CUDA's square
// root by fluid_check_sqrt).  Host code divides.
FL_HD double fl_rsqrt(double x) {
#ifdef __CUDA_ARCH__
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-(x * y), y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
#else
  return 1.0 / std::sqrt(x);
#endif
}

// Square root as x * x^{-1/2} for positive normal finite x (high word in [2^20, 0x7ff00000));
// zero, negative, denormal or non-finite x take the library square root.
FL_HD double fl_sqrt(double x) {
#ifdef __CUDA_ARCH__
  const int hw = __double2hiint(x);
  if (hw >= 0x00100000 && hw < 0x7ff00000) return x * fl_rsqrt(x);
  return sqrt(x);
#else
  return std::sqrt(x);
#endif
}

// Reciprocal by Newton-Raphson iteration for 1/y (one step with its second-order term,
// r' = r + r (e + e^2), e = 1 - y r, which cubes the relative error) from the hardware estimate of
// the PTX instruction rcp.approx.ftz.f64.  For positive normal y the result is within a few ulp of
// 1/y (checked against CUDA's division by fluid_check_math).  Host code divides.
FL_HD double fl_rcp(double y) {
#ifdef __CUDA_ARCH__
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(y));
  const double e = fma(-y, r, 1.0);
  return fma(r, fma(e, e, e), r);
#else
  return 1.0 / y;
#endif
}


}  // namespace fl
