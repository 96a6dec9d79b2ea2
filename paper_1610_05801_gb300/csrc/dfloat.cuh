// Double-float (FP32 pair) helpers for work that must keep ~48 bits but should not
// run on the FP64 pipe (2 operations per clock per SM on GB300, against 128 for FP32).
//
// A value is the unevaluated sum h + l of two floats.  split_bits() turns a double into
// such a pair with integer operations only (no FP64 or conversion instruction: the
// double <-> float conversions run at the FP64 pipe's rate on this GPU), the products use
// the exact FP32 product error from fmaf (Dekker / Knuth), and sums use TwoSum followed
// by Fast2Sum renormalisation.  Explicit _rn intrinsics keep the compiler from
// contracting or reassociating.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace phtl {

struct DF2 {
    float h, l;
};

// x ~ h + l with |x - (h + l)| <= 2^-47 |x|: h holds the top 24 significant bits of x
// (truncated), l the next 24 (truncated).  |x| below 2^-126 (and the low part below
// float range) is flushed to zero; Inf / NaN give a NaN high part.
__device__ __forceinline__ DF2 split_bits(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned hi32 = static_cast<unsigned>(b >> 32), lo32 = static_cast<unsigned>(b);
    const unsigned sign = hi32 & 0x80000000u;
    const int e = static_cast<int>((hi32 >> 20) & 0x7ffu);  // biased FP64 exponent
    const int ef = e - 896;                                  // biased FP32 exponent
    DF2 r;
    if (e == 0x7ff) {
        r.h = __int_as_float(0x7fc00000);
        r.l = 0.0f;
        return r;
    }
    if (ef <= 0) {
        r.h = 0.0f;
        r.l = 0.0f;
        return r;
    }
    if (ef > 254) {
        r.h = __int_as_float(static_cast<int>(sign | 0x7f800000u));
        r.l = 0.0f;
        return r;
    }
    const unsigned mant_hi = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
    r.h = __int_as_float(static_cast<int>(sign | (static_cast<unsigned>(ef) << 23) | mant_hi));
    const unsigned m29 = lo32 & 0x1fffffffu;  // remaining bits: value m29 * 2^(e - 1075)
    const int p = 31 - __clz(static_cast<int>(m29 | 1u));     // MSB position (0 if m29 == 0)
    const unsigned mant = p > 23 ? (m29 >> (p - 23)) : (m29 << (23 - p));
    const int el = e - 1075 + p + 127;                          // biased FP32 exponent of l
    const bool keep = m29 != 0u && el > 0;
    r.l = keep ? __int_as_float(static_cast<int>(sign | (static_cast<unsigned>(el) << 23) | (mant & 0x7fffffu)))
               : 0.0f;
    return r;
}

// float -> double with integer operations (the F2F instruction runs at the FP64 pipe's
// rate on this GPU).  Subnormal floats become zero; Inf / NaN use the conversion.
__device__ __forceinline__ double widen_float_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0xffu) return static_cast<double>(f);
    const unsigned sign = u & 0x80000000u;
    if (e == 0u) return __hiloint2double(static_cast<int>(sign), 0);
    const unsigned m = u & 0x7fffffu;
    return __hiloint2double(static_cast<int>(sign | ((e + 896u) << 20) | (m >> 3)),
                            static_cast<int>(m << 29));
}

// Cheaper forms of the two for the RF phase argument of the FP32C kernels (k z + phi_s
// formed in FP64 from a coordinate's two floats), where a term below 2^-126 in magnitude
// changes nothing.
//
// widen_float_phase: exact for normal floats and +-0 (a particle at z = 0 keeps the phase 0
// exactly); subnormals become values of magnitude in [2^-127, 2^-126); Inf / NaN become
// finite values of magnitude >= 2^128 (a lost particle's phase, which the sine's
// wide-range path takes).
__device__ __forceinline__ double widen_float_phase(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned mag = u & 0x7fffffffu;
    const unsigned hi = mag != 0u ? (mag >> 3) + (896u << 20) : 0u;
    return __hiloint2double(static_cast<int>((u & 0x80000000u) | hi), static_cast<int>(u << 29));
}

// split_phase: split_bits's high part; the low part is the remaining 29 bits rounded to
// nearest (one integer-to-float conversion) instead of truncated, so
// |x - (h + l)| <= 2^-48 |x|.  For 2^-74 <= |x| < 2^128 (both parts normal or zero);
// other magnitudes, Inf and NaN take split_bits.
__device__ __forceinline__ DF2 split_phase(double x)
{
    const unsigned hi32 = static_cast<unsigned>(__double2hiint(x));
    const unsigned lo32 = static_cast<unsigned>(__double2loint(x));
    const unsigned e = (hi32 >> 20) & 0x7ffu;
    if (e - 949u > 201u) return split_bits(x);
    const unsigned sign = hi32 & 0x80000000u;
    const unsigned t = (hi32 & 0x7fffffffu) - (896u << 20);  // FP32 biased exponent at bit 20
    DF2 r;
    r.h = __uint_as_float(sign | __funnelshift_l(lo32, t, 3));
    const float m = __uint2float_rn(lo32 & 0x1fffffffu);      // the remaining bits, rounded
    r.l = __uint_as_float(sign | __float_as_uint(__fmul_rn(m, __uint_as_float((e - 948u) << 23))));
    return r;
}

__device__ __forceinline__ DF2 df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF2{s, e};
}

__device__ __forceinline__ DF2 df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return DF2{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF2 df_add(DF2 a, DF2 b)
{
    DF2 s = df_two_sum(a.h, b.h);
    const float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return df_fast_two_sum(s.h, e);
}

// a + b when |a| >= |b| is known (e.g. a constant term of a Horner step and a small
// product): Fast2Sum on the heads is then exact, which saves the three operations of
// TwoSum; the result is the same as df_add's.
__device__ __forceinline__ DF2 df_add_dominant(DF2 a, DF2 b)
{
    const float s = __fadd_rn(a.h, b.h);
    const float e = __fadd_rn(__fadd_rn(__fsub_rn(a.h, s), b.h), __fadd_rn(a.l, b.l));
    return df_fast_two_sum(s, e);
}

// a * b for a float b (a pair times a single float).
__device__ __forceinline__ DF2 df_mul_f(DF2 a, float b)
{
    const float p = __fmul_rn(a.h, b);
    const float e = __fmaf_rn(a.l, b, __fmaf_rn(a.h, b, -p));
    return df_fast_two_sum(p, e);
}

// -a when the integer flag has bit 31 set, +a when it is 0 (sign flip by XOR).
__device__ __forceinline__ DF2 df_xor_sign(DF2 a, unsigned sign_bit)
{
    return DF2{__uint_as_float(__float_as_uint(a.h) ^ sign_bit),
               __uint_as_float(__float_as_uint(a.l) ^ sign_bit)};
}

// a * b with the exact FP32 product error and the cross terms (the l*l term, 2^-48
// relative, is dropped).
__device__ __forceinline__ DF2 df_mul(DF2 a, DF2 b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ double df_to_double(DF2 a)
{
    return static_cast<double>(a.h) + static_cast<double>(a.l);
}

__device__ __forceinline__ DF2 df_shfl_xor(DF2 a, int o)
{
    return DF2{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}

}  // namespace phtl
