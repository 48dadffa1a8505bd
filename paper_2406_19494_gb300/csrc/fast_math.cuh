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

// x^n for a small positive integer n by binary powering (n - 1 + number of bits of n multiplies at
// most; x^7 and x^10 take four).
FL_HD double fl_ipow(double x, int n) {
  double r = x, b = x;
  bool have = false;
  while (true) {
    if (n & 1) {
      r = have ? r * b : b;
      have = true;
    }
    n >>= 1;
    if (!n) break;
    b = b * b;
  }
  return r;
}

// x^(p/q) for 0 < p, q <= 16 and x in [2^-B, 2^B): y = x^(p/q) is the positive root of y^q = a,
// a = x^p.  B (at most 49, and such that the FP32 estimate and x^p stay normal: |(p/q) log2 x| <
// 125, |p log2 x| < 1021) is set on the host (set_power_law) as the high-word bounds hw_lo, hw_hi:
// the high word of a positive double orders like the number, so the range test, the conversion of
// x to FP32 (truncated: the estimate needs only its leading bits) and the exact conversion of the
// estimate back to FP64 are integer operations.  An FP32 estimate y0 = 2^(e log2 x) from the
// hardware approximations (ex2.approx, lg2.approx; relative error below about 3e-6 on this range)
// takes one step of Halley's method for y^q = a,
// y1 = y0 ((q + 1) a + (q - 1) y0^q) / ((q - 1) a + (q + 1) y0^q), whose error is about
// (q^2 - 1) / 12 times the cube of y0's, below FP64 rounding.  The step is written as the
// correction y1 = y0 + 2 y0 (a - y0^q) / ((q + 1) y0^q + (q - 1) a), of relative size about 1e-6,
// so that its own rounding stays far below an ulp of y1.  Other x take the library
// exp(e log x).  e32 is p/q in FP32.  Checked on the GPU against x^(p/q) (fluid_check_pow).
FL_HD double fl_pow_rational(double x, int p, int q, float e32, int hw_lo, int hw_hi) {
#ifdef __CUDA_ARCH__
  const int hw = __double2hiint(x);
  if (hw >= hw_lo && hw < hw_hi) {
    // exponent rebiased from 1023 to 127, the top 23 fraction bits
    const float xf = __int_as_float(((hw - ((1023 - 127) << 20)) << 3) |
                                    (int)((unsigned)__double2loint(x) >> 29));
    float l, y32;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(xf));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y32) : "f"(e32 * l));
    const int yb = __float_as_int(y32);
    const double y0 = __hiloint2double((yb >> 3) + ((1023 - 127) << 20), yb << 29);
    const double a = fl_ipow(x, p), yq = fl_ipow(y0, q);
    const double den = fma(0.5 * (double)(q + 1), yq, (0.5 * (double)(q - 1)) * a);
    return fma(y0 * (a - yq), fl_rcp(den), y0);
  }
#endif
  return exp(((double)p / (double)q) * log(x));
}

// x >= 0 and x > 0 from the sign and magnitude bits (integer operations in device code; -0 >= 0
// holds and -0 > 0 does not; a NaN counts by its sign bit)
FL_HD bool fl_nonneg(double x) {
#ifdef __CUDA_ARCH__
  const int hw = __double2hiint(x);
  return hw >= 0 || ((hw & 0x7fffffff) | __double2loint(x)) == 0;
#else
  return x >= 0.0;
#endif
}
FL_HD bool fl_pos(double x) {
#ifdef __CUDA_ARCH__
  const int hw = __double2hiint(x);
  return hw >= 0 && (hw | __double2loint(x)) != 0;
#else
  return x > 0.0;
#endif
}

// FP32 -> FP64 widening assembled from the bit fields with integer operations.  The conversion is
// exact, so the result is the same double the conversion instruction gives: a normal number
// re-biases its exponent (127 -> 1023) and keeps its 23 fraction bits at the top of the 52; a
// subnormal number is normalised by the position of its leading one; zeros keep their sign;
// infinities and NaNs take the all-ones exponent with their fraction bits (a NaN stays a NaN).
// On this GPU a 64-bit conversion issues to the FP64 pipe, at the rate of an FP64 FMA; these
// integer operations do not.  Checked against the conversion instruction (fluid_check_widen).
FL_HD double fl_widen(float x) {
#ifdef __CUDA_ARCH__
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  unsigned m = u & 0x7fffffu;
  unsigned ef;
  if (e == 0xffu) {
    ef = 0x7ffu;
  } else if (e != 0u) {
    ef = e + (1023u - 127u);
  } else if (m == 0u) {
    ef = 0u;
  } else {
    const int sh = __clz((int)m) - 8;               // 1 .. 23: moves the leading one to bit 23
    m = (m << sh) & 0x7fffffu;
    ef = (unsigned)(1023 - 126 - sh);                // the value is 1.fraction x 2^(-126 - sh)
  }
  return __hiloint2double((int)((u & 0x80000000u) | (ef << 20) | (m >> 3)), (int)(m << 29));
#else
  return (double)x;
#endif
}

}  // namespace fl
