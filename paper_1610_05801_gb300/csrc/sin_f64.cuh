// FP64 sine of the FP64 kick, written for the scarce FP64 pipe of GB300 (2 DFMA per
// clock per SM).
//
// Method: Cody-Waite argument reduction x = q pi/2 + r (Cody & Waite, "Software Manual
// for the Elementary Functions", 1980), done with fused multiply-adds so a two-part
// pi/2 suffices, then one polynomial on |r| <= pi/4 whose coefficient set (sine or
// cosine) is selected per lane by the quadrant parity:
//     sin r = r + r^3 S(r^2),   cos r = 1 - r^2/2 + r^4 C(r^2),   deg S = deg C = 5,
// fitted by Chebyshev interpolation at 60 digits (gen_sin_coeffs.py; polynomial error
// 2e-17 relative for S, 1.3e-18 for C).  11 FP64 operations per call, no branches and
// no local memory on the path; the quadrant is found in FP32 and the range check on the
// integer pipe.  |x| > 1e5 (far outside any RF bucket) falls back to CUDA's sin().
// Accuracy: a few ulp on |x| <= 1e5 (checked against CUDA's sin and mpmath in the
// tests through phtl_eval_sin).
#pragma once

#include <cuda_runtime.h>

#include "dfloat.cuh"

namespace phtl {
namespace detail {

constexpr double kTwoOverPi = 0.63661977236758134308;
constexpr double kPio2Hi = 1.5707963267948966;      // nearest double to pi/2
constexpr double kPio2Lo = 6.123233995736766e-17;   // pi/2 - kPio2Hi

__device__ __forceinline__ double sc_coef(bool odd, double s, double c) { return odd ? c : s; }

}  // namespace detail

__device__ __forceinline__ double sin_f64(double x)
{
    using namespace detail;
    // |x| >= 1e5 (high word of 1e5 is 0x40f86a00): library sine
    if ((__double2hiint(x) & 0x7fffffff) >= 0x40f86a00) return sin(x);
    // quadrant q = nearest integer to x * 2/pi, found in FP32 from the top 24 bits of x
    // (integer split: no FP64 instruction).  Near a half-integer q may be off by one,
    // which only moves |r| a hair past pi/4, inside the polynomials' accuracy.
    const float xf = split_bits(x).h;
    const float tf = __fmaf_rn(xf, 0.6366197466850281f, 12582912.0f);
    const int qi = __float_as_int(tf);         // q mod 2^22 in the low mantissa bits
    const double q = widen_float_bits(__fsub_rn(tf, 12582912.0f));
    double r = fma(-q, kPio2Hi, x);
    r = fma(-q, kPio2Lo, r);
    const double r2 = r * r;
    const bool odd = (qi & 1) != 0;
    double p = sc_coef(odd, 1.5918129294866608e-10, -1.1382632425521717e-11);
    p = fma(p, r2, sc_coef(odd, -2.5051131845003624e-08, 2.08761462684032e-09));
    p = fma(p, r2, sc_coef(odd, 2.755731610255244e-06, -2.7557317271729793e-07));
    p = fma(p, r2, sc_coef(odd, -0.00019841269836758574, 2.480158729876569e-05));
    p = fma(p, r2, sc_coef(odd, 0.008333333333330948, -0.0013888888888887398));
    p = fma(p, r2, sc_coef(odd, -0.16666666666666666, 0.041666666666666664));
    const double m = (odd ? r2 : r) * r2;                 // r^3 or r^4
    const double a = odd ? fma(-0.5, r2, 1.0) : r;        // r or 1 - r^2/2
    const double res = fma(m, p, a);
    // quadrants 2 and 3 flip the sign: an integer XOR of the sign bit, not an FP64 negate
    return __longlong_as_double(__double_as_longlong(res) ^ (static_cast<long long>(qi & 2) << 62));
}

}  // namespace phtl
