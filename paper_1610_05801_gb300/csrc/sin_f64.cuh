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
//
// sin_kz(k, z) = sin(k z) is the kick's phase for phi_s = 0 with the product folded into
// the reduction: r = (k z - q H) - q L with H = 3217/2048 (12 significant bits, so q H is
// an integer times 2^-11, formed exactly for |q| < 2^16) and L = pi/2 - H rounded to FP64.
// The first step is one FMA on the exact k z, the second one FMA, so the phase costs no
// separate FP64 operation and r is rounded relative to itself rather than to k z: 11 FP64
// operations for sin(k z), against 12 for the phase product followed by sin_f64.
#pragma once

#include <cuda_runtime.h>

#include "dfloat.cuh"

namespace phtl {
namespace detail {

constexpr double kTwoOverPi = 0.63661977236758134308;
constexpr double kPio2Hi = 1.5707963267948966;      // nearest double to pi/2
constexpr double kPio2Lo = 6.123233995736766e-17;   // pi/2 - kPio2Hi
constexpr float kPio2H12 = 1.57080078125f;          // 3217 / 2048
constexpr double kPio2L12 = -4.454455103380769e-06; // pi/2 - 3217/2048
constexpr float kMagic = 12582912.0f;               // 1.5 * 2^23: rounds to an integer

// sin r = r + r^3 S(r^2), cos r = 1 - r^2/2 + r^4 C(r^2): coefficients of S and C from the
// highest degree down (Chebyshev fits, gen_sin_coeffs.py)
__host__ __device__ constexpr double kS(int i)
{
    return i == 0 ? 1.5918129294866608e-10 : i == 1 ? -2.5051131845003624e-08
         : i == 2 ? 2.755731610255244e-06  : i == 3 ? -0.00019841269836758574
         : i == 4 ? 0.008333333333330948   : -0.16666666666666666;
}
__host__ __device__ constexpr double kC(int i)
{
    return i == 0 ? -1.1382632425521717e-11 : i == 1 ? 2.08761462684032e-09
         : i == 2 ? -2.7557317271729793e-07 : i == 3 ? 2.480158729876569e-05
         : i == 4 ? -0.0013888888888887398  : 0.041666666666666664;
}
constexpr double kTwoPi = 6.283185307179586;

__device__ __forceinline__ double sc_coef(bool odd, double s, double c) { return odd ? c : s; }

// sin(q pi/2 + r) for |r| <= pi/4 (a hair more when q came out one off), given the low
// bits qi of q.
__device__ __forceinline__ double sin_quadrant(double r, int qi)
{
    const double r2 = r * r;
    const bool odd = (qi & 1) != 0;
    double p = sc_coef(odd, kS(0), kC(0));
#pragma unroll
    for (int i = 1; i < 6; ++i) p = fma(p, r2, sc_coef(odd, kS(i), kC(i)));
    const double m = (odd ? r2 : r) * r2;                 // r^3 or r^4
    const double a = odd ? fma(-0.5, r2, 1.0) : r;        // r or 1 - r^2/2
    const double res = fma(m, p, a);
    // quadrants 2 and 3 flip the sign: an integer XOR of the sign bit, not an FP64 negate
    return __longlong_as_double(__double_as_longlong(res) ^ (static_cast<long long>(qi & 2) << 62));
}

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
    const float tf = __fmaf_rn(xf, 0.6366197466850281f, kMagic);
    const int qi = __float_as_int(tf);         // q mod 2^22 in the low mantissa bits
    const double q = widen_float_bits(__fsub_rn(tf, kMagic));
    double r = fma(-q, kPio2Hi, x);
    r = fma(-q, kPio2Lo, r);
    return sin_quadrant(r, qi);
}

namespace detail {

// -q H = -q 3217 / 2048 as a double, exactly, for |q| < 2^16: the integer product m = q 3217
// (|m| < 2^28) placed into the significand with integer operations (no FP64 or conversion
// instruction).  Within |q| < 4096 it equals the FP32 product q H, which is exact there.
__device__ __forceinline__ double neg_q_h(int q)
{
    const int m = -q * 3217;
    const unsigned a = static_cast<unsigned>(m < 0 ? -m : m);
    const int p = 31 - __clz(static_cast<int>(a | 1u));            // leading bit of |m|
    const unsigned long long mant = (static_cast<unsigned long long>(a) << (52 - p)) &
                                    0x000FFFFFFFFFFFFFull;
    const unsigned long long bits = (static_cast<unsigned long long>(m < 0 ? 1u : 0u) << 63) |
                                    (static_cast<unsigned long long>(1023 - 11 + p) << 52) | mant;
    return a == 0u ? -0.0 : __longlong_as_double(static_cast<long long>(bits));  // q = 0: -0 * H
}

}  // namespace detail

// sin(k z); k2opi = k * 2/pi rounded to FP32.  The fused form holds for |k z| up to ~1e5
// (the quadrant q below 2^16): it covers the bucket and the particles that leave it for
// ~1e6 turns, so a warp does not split between two sine paths when one of its particles
// drifts away.  Beyond, and for Inf and NaN: sin_f64(k * z).
__device__ __forceinline__ double sin_kz(double k, float k2opi, double z)
{
    using namespace detail;
    const float xq = __fmul_rn(split_bits(z).h, k2opi);   // ~ k z * 2/pi
    if (!(fabsf(xq) < 65536.0f)) return sin_f64(k * z);
    const float tf = __fadd_rn(xq, kMagic);
    const int qi = __float_as_int(tf);
    const float qf = __fsub_rn(tf, kMagic);
    const double mqh = neg_q_h(qi - __float_as_int(kMagic));         // -q H, exact
    double r = fma(k, z, mqh);
    r = fma(widen_float_bits(qf), -kPio2L12, r);
    return sin_quadrant(r, qi);
}

// sin and cos of 2 pi a, a in turns (the chromatic phase advance).  Quarter-turn
// reduction a = n/4 + f: f = a - n/4 is exact (Sterbenz; n from FP32, so |f| may exceed
// 1/8 by a hair), r = 2 pi f is rounded once, then both polynomials of sin_quadrant on r
// and the quadrant's swap and signs as integer selects.  19 FP64 operations for the pair.
// |a| >= 2^20 turns falls back to CUDA's sin and cos.
__device__ __forceinline__ void sincos_turns(double a, double& s, double& c)
{
    using namespace detail;
    const float af = split_bits(a).h;
    if (!(fabsf(af) < 1048576.0f)) {
        s = sin(kTwoPi * a);
        c = cos(kTwoPi * a);
        return;
    }
    const float tf = __fmaf_rn(af, 4.0f, kMagic);
    const int ni = __float_as_int(tf);                       // n mod 2^22
    const float nf = __fsub_rn(tf, kMagic);
    const double r = (a - widen_float_bits(__fmul_rn(nf, 0.25f))) * kTwoPi;
    const double r2 = r * r;
    double ps = kS(0), pc = kC(0);
#pragma unroll
    for (int i = 1; i < 6; ++i) {
        ps = fma(ps, r2, kS(i));
        pc = fma(pc, r2, kC(i));
    }
    const double sr = fma(r * r2, ps, r);
    const double cr = fma(r2 * r2, pc, fma(-0.5, r2, 1.0));
    const bool swap = (ni & 1) != 0;
    // n mod 4 = 0: (sr, cr); 1: (cr, -sr); 2: (-sr, -cr); 3: (-cr, sr)
    s = __longlong_as_double(__double_as_longlong(swap ? cr : sr) ^
                             (static_cast<long long>(ni & 2) << 62));
    c = __longlong_as_double(__double_as_longlong(swap ? sr : cr) ^
                             (static_cast<long long>((ni + 1) & 2) << 62));
}

}  // namespace phtl
