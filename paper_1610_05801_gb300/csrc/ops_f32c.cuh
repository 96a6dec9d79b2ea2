// FP32-compensated per-particle operations shared by the FP32C kernels (single bunch
// and batched).  Every coordinate is an unevaluated sum hi + comp of two floats; see
// track_f32c.cu for the arithmetic model.  One thread owns P = 4 particles.
#pragma once

#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "internal.h"
#include "monitor.cuh"
#include "sin_f64.cuh"

namespace phtl {
namespace f32c {

constexpr int P = 4;

// Register budgets of the FP32-compensated kernels, as resident 256-thread blocks per SM asked
// of the compiler.  The kernels are issue-bound with few resident warps (116-160 registers:
// 12-16 warps per SM), so more blocks per SM (fewer registers, some spill) pays where it was
// measured to (1e6 particles, transverse planes, a monitor row every turn):
//   - linear map: 4 blocks (at most 64 registers: 32 warps) for FP32C (+3.8 % over 3 blocks,
//     all three schemes); 3 blocks (at most 85 registers) for FP32CS (-2.5 % at 4) and the Ruth4
//     FP32CD kernel (-7 % at 4); the FP32CD Euler-Cromer and leap-frog kernels ran slower at 3
//     and keep the compiler's choice (1);
//   - widened map and RK4 / double RF (general kernels): 3 blocks for FP32C (-4 % time over the
//     three symplectic schemes, -34 % for RK4 on the double-RF ring), FP32CS (-29 %) and FP32CD
//     RK4 (-24 %); 2 blocks (at most 128 registers) for the FP32CD symplectic schemes (-2 %;
//     3 blocks was 1 % slower than the compiler's choice);
//   - batched kernels: 3 blocks (the batched FP32C kernel spills 2 KB a thread at 64 registers
//     for +1.2 %); the widened map's batched kernels (16 bunches of 2.5e5 particles, 500
//     turns): 2 blocks for FP32C and FP32CD (FP32CD leap-frog -17 %, Ruth4 -47 %), 3 for FP32CS
//     (-37 %);
//   - ramp programme: 3 blocks for FP32C (-6.6 %), the compiler's choice for FP32CD and FP32CS
//     (track_ramp.cu).
// Build options PHTL_F32C_GEN_MIN_BLOCKS, PHTL_F32C_GEN_BATCHED_MIN_BLOCKS (general kernels) and
// PHTL_F32C_MAXNREG (one register cap for all of them) override these, for measuring.
constexpr int f32c_general_min_blocks(int scheme, int dtype)
{
#ifdef PHTL_F32C_GEN_MIN_BLOCKS
    return (void)scheme, (void)dtype, PHTL_F32C_GEN_MIN_BLOCKS;
#else
    return dtype == PHTL_F32CD && scheme != PHTL_RK4 ? 2 : 3;
#endif
}
constexpr int f32c_track_min_blocks(int scheme, int dtype, bool general)
{
    return general ? f32c_general_min_blocks(scheme, dtype)
                   : dtype == PHTL_F32C ? 4 : (dtype == PHTL_F32CD && scheme != PHTL_RUTH4 ? 1 : 3);
}
constexpr int f32c_batched_min_blocks(int dtype, bool general)
{
#ifdef PHTL_F32C_GEN_BATCHED_MIN_BLOCKS
    return general ? ((void)dtype, PHTL_F32C_GEN_BATCHED_MIN_BLOCKS) : 3;
#else
    return general ? (dtype == PHTL_F32CS ? 3 : 2) : 3;
#endif
}
#ifdef PHTL_F32C_MAXNREG
#define PHTL_F32C_RAMP_BOUNDS(S, DT) __maxnreg__(PHTL_F32C_MAXNREG)
#define PHTL_F32C_RAMP_BOUNDS_C __maxnreg__(PHTL_F32C_MAXNREG)
#define PHTL_F32C_TRACK_BOUNDS(S, DT, G) __maxnreg__(PHTL_F32C_MAXNREG)
#define PHTL_F32C_BATCHED_BOUNDS(DT, G) __maxnreg__(PHTL_F32C_MAXNREG)
#else
#define PHTL_F32C_RAMP_BOUNDS(S, DT) __launch_bounds__(256)
#define PHTL_F32C_RAMP_BOUNDS_C __launch_bounds__(256, 3)
#define PHTL_F32C_TRACK_BOUNDS(S, DT, G) __launch_bounds__(256, f32c::f32c_track_min_blocks(S, DT, G))
#define PHTL_F32C_BATCHED_BOUNDS(DT, G) __launch_bounds__(256, f32c::f32c_batched_min_blocks(DT, G))
#endif
constexpr float kTwoPiHi = 6.28318548202514648438f;     // float(2 pi)
constexpr float kTwoPiLo = -1.74845553146951715e-07f;    // 2 pi - kTwoPiHi
constexpr float kInvTwoPi = 0.159154943091895335769f;

struct DF {
    float hi, c;
};

// (hi, c) += inc, with the rounding error of hi + inc kept in c (TwoSum), then
// renormalised so |c| <= ulp(hi)/2 (Fast2Sum).  Explicit _rn intrinsics keep the
// compiler from contracting or reassociating.
__device__ __forceinline__ void acc(DF& a, float inc)
{
    const float s = __fadd_rn(a.hi, inc);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(inc, bb));
    const float c = __fadd_rn(a.c, err);
    const float t = __fadd_rn(s, c);
    a.c = __fsub_rn(c, __fsub_rn(t, s));
    a.hi = t;
}

// Double-float product m * u (m = mh + ml, u = uh + uc) as (p, e): p + e ~ m u.
__device__ __forceinline__ void df_mul(float mh, float ml, const DF& u, float& p, float& e)
{
    p = __fmul_rn(mh, u.hi);
    e = __fmaf_rn(mh, u.hi, -p);                 // exact error of the FP32 product
    e = __fmaf_rn(mh, u.c, __fmaf_rn(ml, u.hi, e));
}

// Double-float rotation [u; v] <- [[m0, m1], [m2, m3]] [u; v].
__device__ __forceinline__ void df_rotate(DF& u, DF& v, const float (&mh)[4], const float (&ml)[4])
{
    float p1, e1, p2, e2, p3, e3, p4, e4;
    df_mul(mh[0], ml[0], u, p1, e1);
    df_mul(mh[1], ml[1], v, p2, e2);
    df_mul(mh[2], ml[2], u, p3, e3);
    df_mul(mh[3], ml[3], v, p4, e4);
    // un = p1 + p2 + (e1 + e2) via TwoSum + Fast2Sum
    {
        const float s = __fadd_rn(p1, p2);
        const float bb = __fsub_rn(s, p1);
        const float err = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
        const float lo = __fadd_rn(err, __fadd_rn(e1, e2));
        const float t = __fadd_rn(s, lo);
        u.c = __fsub_rn(lo, __fsub_rn(t, s));
        u.hi = t;
    }
    {
        const float s = __fadd_rn(p3, p4);
        const float bb = __fsub_rn(s, p3);
        const float err = __fadd_rn(__fsub_rn(p3, __fsub_rn(s, bb)), __fsub_rn(p4, bb));
        const float lo = __fadd_rn(err, __fadd_rn(e3, e4));
        const float t = __fadd_rn(s, lo);
        v.c = __fsub_rn(lo, __fsub_rn(t, s));
        v.hi = t;
    }
}

// ---------------------------------------------------------------------------------------
// Arithmetic of PHTL_F32C / PHTL_F32CD: double-float (FP32 pair, ~48 bits) throughout.
// Increments are double-float products and are added with TwoSum + Fast2Sum, the sine is
// a double-float polynomial, so each turn's relative error stays near 1e-14: over 1e6 turns
// particles near the separatrix (where the tune varies steeply with amplitude) keep their
// phases, and bunch moments follow the FP64 result.

__device__ __forceinline__ DF2 as2(const DF& a) { return DF2{a.hi, a.c}; }
__device__ __forceinline__ DF2 neg2(DF2 a) { return DF2{-a.h, -a.l}; }

__device__ __forceinline__ void acc2(DF& a, DF2 inc)
{
    const DF2 s = df_add(as2(a), inc);
    a.hi = s.h;
    a.c = s.l;
}

__device__ __forceinline__ double widen_bits(float f) { return widen_float_bits(f); }

// Phase argument phi = phi_s + k z as a double-float pair.  PHTL_F32C forms it in FP64 from
// hi + comp (exact in double) with one DFMA and splits it with the phase forms of the
// integer widening and split; PHTL_F32CD in double-float arithmetic.
// ZS: phi_s == 0, so the phase is k z alone (chosen once, outside the turn loop).
template <int DT, bool ZS>
__device__ __forceinline__ DF2 phase_df(const MapConsts& c, const DF& z)
{
    if (DT == PHTL_F32C) {
        const double zd = widen_float_phase(z.hi) + widen_float_phase(z.c);
        return split_phase(ZS ? c.k * zd : fma(c.k, zd, c.phis));
    }
    const DF2 kz = df_mul(DF2{c.k_hi, c.k_lo}, as2(z));
#ifdef PHTL_F32CD_PHASE_F32
    // build option, for the accuracy comparison of the FP32 variants: the PHTL_F32CD phase
    // rounded to one float (double-float state, increments and sine otherwise)
    if (DT == PHTL_F32CD) {
        const DF2 ph = ZS ? kz : df_add(kz, DF2{c.phis_hi, c.phis_lo});
        return DF2{__fadd_rn(ph.h, ph.l), 0.0f};
    }
#endif
    return ZS ? kz : df_add(kz, DF2{c.phis_hi, c.phis_lo});
}

// Double-float split of an FP64 constant at compile time.
struct DFC {
    float h, l;
    __host__ __device__ constexpr DFC(double v) : h(static_cast<float>(v)), l(static_cast<float>(v - static_cast<double>(static_cast<float>(v)))) {}
};

// Double-float sine, absolute error ~1e-12 on the kick's range (a per-kick force error
// far below what moves a particle's phase measurably in 1e6 turns).
// Reduction x = q pi/2 + r with pi/2 = P1 + P2 + P3: q P1 is formed exactly (two_prod),
// x.h - q P1 exactly as a TwoSum pair (its low part is zero whenever Sterbenz applies), and
// the small remainder (x.l - e1 - q P2 - q P3, each ~1e-7) is summed in FP32 and
// renormalised.  Then on |r| <= pi/4 one polynomial chosen per lane by the
// quadrant parity, sin r = r + r^3 S(r^2), cos r = 1 - r^2/2 + r^4 C(r^2), with the
// coefficients of the FP64 sine (sin_f64.cuh): the two leading Horner steps in
// double-float, the four trailing terms (|t^2 S_2| <= 8e-5, |t^2 C_2| <= 1e-5) in FP32.
// Every double-float addition after the reduction adds a smaller term to a larger one
// (Horner constant vs product, r vs r^3 S, 1 - t/2 vs r^4 C), so it uses Fast2Sum on the
// heads.  |x| >= 1e4 falls back to the FP64 sine.
__device__ __forceinline__ DF2 sin_df(DF2 x)
{
    if (!(fabsf(x.h) < 1.0e4f)) return split_bits(sin_f64(widen_bits(x.h) + widen_bits(x.l)));
    const float magic = 12582912.0f;
    const float t0 = __fmaf_rn(x.h, 0.6366197466850281f, magic);
    const float q = __fsub_rn(t0, magic);
    const int qi = __float_as_int(t0);
    const float p1 = __fmul_rn(q, 1.5707963705062866f);
    const float e1 = __fmaf_rn(q, 1.5707963705062866f, -p1);
    const DF2 hd = df_two_sum(x.h, -p1);  // exact as a pair (Sterbenz makes hd.l ~0)
    float rest = __fadd_rn(__fsub_rn(x.l, e1), hd.l);
    rest = __fmaf_rn(-q, -4.371138828673793e-08f, rest);
    rest = __fmaf_rn(-q, -1.7151245100058819e-15f, rest);
    const DF2 r = df_fast_two_sum(hd.h, rest);
    const DF2 t = df_mul(r, r);
    const bool odd = (qi & 1) != 0;
    // trailing terms in FP32: C_5..C_2 / S_5..S_2
    float tail = odd ? -1.1382632425521717e-11f : 1.5918129294866608e-10f;
    tail = __fmaf_rn(tail, t.h, odd ? 2.08761462684032e-09f : -2.5051131845003624e-08f);
    tail = __fmaf_rn(tail, t.h, odd ? -2.7557317271729793e-07f : 2.755731610255244e-06f);
    tail = __fmaf_rn(tail, t.h, odd ? 2.480158729876569e-05f : -0.00019841269836758574f);
    // leading Horner steps in double-float
    constexpr DFC s1(0.008333333333330948), s0(-0.16666666666666666);
    constexpr DFC c1(-0.0013888888888887398), c0(0.041666666666666664);
    DF2 u = df_add_dominant(odd ? DF2{c1.h, c1.l} : DF2{s1.h, s1.l}, df_mul_f(t, tail));
    u = df_add_dominant(odd ? DF2{c0.h, c0.l} : DF2{s0.h, s0.l}, df_mul(t, u));
    const DF2 m = df_mul(odd ? t : r, t);                                  // r^3 or r^4
    const DF2 a = odd ? df_add_dominant(DF2{1.0f, 0.0f}, DF2{-0.5f * t.h, -0.5f * t.l}) : r;
    const DF2 res = df_add_dominant(a, df_mul(m, u));
    return df_xor_sign(res, static_cast<unsigned>(qi & 2) << 30);      // quadrants 2, 3: -res
}

// ---------------------------------------------------------------------------------------
// Arithmetic of PHTL_F32CS: FP32 increments and the SFU sine (fast, less accurate).

// Phase argument rounded to FP32 (double-float formation, then rounded).  Build option
// PHTL_F32CS_PHASE_FP64: formed in FP64 from hi + comp instead (the same value after the
// rounding to FP32, up to ties), for the accuracy comparison of the FP32CS variants.
template <bool ZS>
__device__ __forceinline__ float phase_f(const MapConsts& c, const DF& z)
{
#ifdef PHTL_F32CS_PHASE_FP64
    const double zd = widen_bits(z.hi) + widen_bits(z.c);
    const double ph = ZS ? c.k * zd : fma(c.k, zd, c.phis);
    const DF2 p2 = split_bits(ph);
    return __fadd_rn(p2.h, p2.l);
#else
    const DF2 ph = phase_df<PHTL_F32CD, ZS>(c, z);
    return __fadd_rn(ph.h, ph.l);
#endif
}

// Build option PHTL_F32CS_SINE_DF: the double-float sine of the FP32 phase instead of the
// SFU (rounded to FP32), for the accuracy comparison of the FP32CS variants.
__device__ __forceinline__ float sin_sfu(float x)
{
#ifdef PHTL_F32CS_SINE_DF
    const DF2 s = sin_df(DF2{x, 0.0f});
    return __fadd_rn(s.h, s.l);
#else
    const float nq = rintf(x * kInvTwoPi);
    return __sinf(__fmaf_rn(-nq, kTwoPiLo, __fmaf_rn(-nq, kTwoPiHi, x)));
#endif
}

// ---------------------------------------------------------------------------------------
// kick: delta += kw * (sin(phi) - sin(phi_s)), kw = kh + kl (the FP64 weight as a pair);
// ZS: phi_s == 0, no subtraction
template <int DT, bool ZS>
__device__ __forceinline__ void kick(const DF (&z)[P], DF (&d)[P], float kh, float kl,
                                     const MapConsts& c)
{
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (DT == PHTL_F32CS) {
            float f;
            if (c.linear) {
                f = c.lin_hi * (z[p].hi + z[p].c);
            } else {
                f = sin_sfu(phase_f<ZS>(c, z[p]));
                if (!ZS) f -= c.sinphis_hi;
            }
            acc(d[p], __fmaf_rn(kh, f, __fmul_rn(kl, f)));
        } else {
            DF2 f;
            if (c.linear) {
                f = df_mul(DF2{c.lin_hi, c.lin_lo}, as2(z[p]));
            } else {
                f = sin_df(phase_df<DT, ZS>(c, z[p]));
                if (!ZS) f = df_add(f, DF2{-c.sinphis_hi, -c.sinphis_lo});
            }
            acc2(d[p], df_mul(DF2{kh, kl}, f));
        }
    }
}

// drift: z -= dc * delta, dc = dh + dl
template <int DT>
__device__ __forceinline__ void drift(DF (&z)[P], const DF (&d)[P], float dh, float dl)
{
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (DT == PHTL_F32CS) {
            const float inc = __fmaf_rn(dh, d[p].hi, __fmaf_rn(dl, d[p].hi, __fmul_rn(dh, d[p].c)));
            acc(z[p], -inc);
        } else {
            acc2(z[p], neg2(df_mul(DF2{dh, dl}, as2(d[p]))));
        }
    }
}

// dh, dl, kh, kl: the drift and kick weights of this bunch's scheme split into FP32
// hi + lo (the single-bunch kernel passes the MapConsts copies, the batched kernel the
// job table's).
template <int SCHEME, int DT, bool ZS>
__device__ __forceinline__ void long_turn(DF (&z)[P], DF (&d)[P], const MapConsts& c,
                                          const float* dh, const float* dl, const float* kh,
                                          const float* kl)
{
    if (SCHEME == PHTL_EULER_CROMER) {
        kick<DT, ZS>(z, d, kh[0], kl[0], c);
        drift<DT>(z, d, dh[0], dl[0]);
    } else if (SCHEME == PHTL_LEAPFROG) {
        drift<DT>(z, d, dh[0], dl[0]);
        kick<DT, ZS>(z, d, kh[0], kl[0], c);
        drift<DT>(z, d, dh[1], dl[1]);
    } else {
        drift<DT>(z, d, dh[0], dl[0]);
        kick<DT, ZS>(z, d, kh[0], kl[0], c);
        drift<DT>(z, d, dh[1], dl[1]);
        kick<DT, ZS>(z, d, kh[1], kl[1], c);
        drift<DT>(z, d, dh[2], dl[2]);
        kick<DT, ZS>(z, d, kh[2], kl[2], c);
        drift<DT>(z, d, dh[3], dl[3]);
    }
}

// ---- widened map: nonlinear slippage and chromaticity -------------------------------

// Drift with the slippage expansion, z -= (dc + g1 d + g2 d^2) d (each coefficient a
// float pair: dc = w eta0 C, g1 = w eta1 C, g2 = w eta2 C).
template <int DT>
__device__ __forceinline__ void drift_nl(DF (&z)[P], const DF (&d)[P], float dh, float dl,
                                         float g1h, float g1l, float g2h, float g2l)
{
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (DT == PHTL_F32CS) {
            const float e = __fmul_rn(__fmaf_rn(g2h, d[p].hi, g1h), d[p].hi);  // (g1 + g2 d) d
            const float inc = __fmaf_rn(dh + e, d[p].hi, __fmaf_rn(dl, d[p].hi, __fmul_rn(dh, d[p].c)));
            acc(z[p], -inc);
        } else {
            const DF2 dd = as2(d[p]);
            DF2 e = df_add(df_mul(DF2{g2h, g2l}, dd), DF2{g1h, g1l});
            e = df_add(df_mul(e, dd), DF2{dh, dl});
            acc2(z[p], neg2(df_mul(e, dd)));
        }
    }
}

// ---- second RF system (double RF) and classic RK4 ----------------------------------

// Force of the second RF system per unit weight, sin(phi2 + k2 z) - sin(phi2) (rf_linear:
// cos(phi2) k2 z), as a pair: the phase in FP64 for PHTL_F32C, in double-float for
// PHTL_F32CD, and the double-float sine.
template <int DT>
__device__ __forceinline__ DF2 force2_df(const MapConsts& c, DF2 z)
{
    if (c.linear) return df_mul(DF2{c.lin2_hi, c.lin2_lo}, z);
    DF2 ph;
    if (DT == PHTL_F32C) {
        const double zd = widen_float_phase(z.h) + widen_float_phase(z.l);
        ph = split_phase(fma(c.k2, zd, c.phi2));
    } else {
        ph = df_add(df_mul(DF2{c.k2_hi, c.k2_lo}, z), DF2{c.phi2_hi, c.phi2_lo});
    }
    return df_add(sin_df(ph), DF2{-c.sinphi2_hi, -c.sinphi2_lo});
}

// The same for PHTL_F32CS: the phase rounded to FP32 and the SFU sine.
__device__ __forceinline__ float force2_f(const MapConsts& c, DF2 z)
{
    if (c.linear) return c.lin2_hi * (z.h + z.l);
    const DF2 ph = df_add(df_mul(DF2{c.k2_hi, c.k2_lo}, z), DF2{c.phi2_hi, c.phi2_lo});
    return sin_sfu(__fadd_rn(ph.h, ph.l)) - c.sinphi2_hi;
}

// Force of the main RF system per unit weight at a pair z (the bracket of kick()).
template <int DT, bool ZS>
__device__ __forceinline__ DF2 force1_df(const MapConsts& c, DF2 z)
{
    if (c.linear) return df_mul(DF2{c.lin_hi, c.lin_lo}, z);
    const DF2 f = sin_df(phase_df<DT, ZS>(c, DF{z.h, z.l}));
    return ZS ? f : df_add(f, DF2{-c.sinphis_hi, -c.sinphis_lo});
}

template <bool ZS>
__device__ __forceinline__ float force1_f(const MapConsts& c, DF2 z)
{
    if (c.linear) return c.lin_hi * (z.h + z.l);
    const float f = sin_sfu(phase_f<ZS>(c, DF{z.h, z.l}));
    return ZS ? f : f - c.sinphis_hi;
}

// Kick of the widened map: the main system (kick()), then the second one when it is on
// (k2h + k2l: this stage's w_j A2), each increment added on its own.
template <int DT, bool ZS>
__device__ __forceinline__ void kick_gen(const DF (&z)[P], DF (&d)[P], float kh, float kl, float k2h,
                                         float k2l, const MapConsts& c, bool dual)
{
    kick<DT, ZS>(z, d, kh, kl, c);
    if (!dual) return;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (DT == PHTL_F32CS) {
            const float f = force2_f(c, as2(z[p]));
            acc(d[p], __fmaf_rn(k2h, f, __fmul_rn(k2l, f)));
        } else {
            acc2(d[p], df_mul(DF2{k2h, k2l}, force2_df<DT>(c, as2(z[p]))));
        }
    }
}

// Right-hand side of the smooth motion per turn as pairs: dz/dn = -(dc + g1 d + g2 d^2) d,
// dd/dn = kw F1(z) + kw2 F2(z) (dc = eta0 C, g1 = eta1 C, g2 = eta2 C, kw = A, kw2 = A2).
template <int DT, bool ZS>
__device__ __forceinline__ void rk4_rhs_df(DF2 z, DF2 d, const MapConsts& c, DF2 dc, DF2 g1, DF2 g2,
                                           DF2 kw, DF2 kw2, bool dual, DF2& fz, DF2& fd)
{
    DF2 e = df_add(df_mul(g2, d), g1);
    e = df_add(df_mul(e, d), dc);
    fz = neg2(df_mul(e, d));
    fd = df_mul(kw, force1_df<DT, ZS>(c, z));
    if (dual) fd = df_add(fd, df_mul(kw2, force2_df<DT>(c, z)));
}

__device__ __forceinline__ DF2 df_scale2(DF2 a, float s) { return DF2{s * a.h, s * a.l}; }  // s = 2^k: exact

// One classic RK4 step of one turn.  PHTL_F32C / PHTL_F32CD: every stage in double-float,
// the weighted sum (k1 + 2 k2 + 2 k3 + k4) / 6 added to the state with TwoSum.
// PHTL_F32CS: the stages in FP32 (the state's comp folded into the stage arguments), the
// weighted sum added with TwoSum.
template <int DT, bool ZS>
__device__ __forceinline__ void rk4_turn(DF (&z)[P], DF (&d)[P], const MapConsts& c, float dh,
                                         float dl, float kh, float kl, float k2h, float k2l,
                                         float g1h, float g1l, float g2h, float g2l, bool dual)
{
    constexpr DFC sixth(1.0 / 6.0);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (DT == PHTL_F32CS) {
            const float z0 = z[p].hi, d0 = d[p].hi, zc = z[p].c, dcmp = d[p].c;
            float kz[4], kd[4];
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                const float w = st == 0 ? 0.0f : (st == 3 ? 1.0f : 0.5f);
                const float zs = st == 0 ? z0 : __fadd_rn(z0, __fmaf_rn(w, kz[st - 1], zc));
                const float ds = st == 0 ? d0 : __fadd_rn(d0, __fmaf_rn(w, kd[st - 1], dcmp));
                const float e = __fmaf_rn(__fmaf_rn(g2h, ds, g1h), ds, dh);
                kz[st] = -__fmul_rn(e, ds);
                const DF2 zz{zs, 0.0f};
                const float f1 = force1_f<ZS>(c, zz);
                float fd = __fmaf_rn(kh, f1, __fmul_rn(kl, f1));
                if (dual) fd = __fmaf_rn(k2h, force2_f(c, zz), fd);
                kd[st] = fd;
            }
            const float sz = __fmaf_rn(2.0f, __fadd_rn(kz[1], kz[2]), __fadd_rn(kz[0], kz[3]));
            const float sd = __fmaf_rn(2.0f, __fadd_rn(kd[1], kd[2]), __fadd_rn(kd[0], kd[3]));
            acc(z[p], __fmul_rn(sz, 0.166666671633720398f));
            acc(d[p], __fmul_rn(sd, 0.166666671633720398f));
        } else {
            const DF2 dc{dh, dl}, g1{g1h, g1l}, g2{g2h, g2l}, kw{kh, kl}, kw2{k2h, k2l};
            const DF2 z0 = as2(z[p]), d0 = as2(d[p]);
            DF2 k1z, k1d, k2z, k2d, k3z, k3d, k4z, k4d;
            rk4_rhs_df<DT, ZS>(z0, d0, c, dc, g1, g2, kw, kw2, dual, k1z, k1d);
            rk4_rhs_df<DT, ZS>(df_add(z0, df_scale2(k1z, 0.5f)), df_add(d0, df_scale2(k1d, 0.5f)), c,
                               dc, g1, g2, kw, kw2, dual, k2z, k2d);
            rk4_rhs_df<DT, ZS>(df_add(z0, df_scale2(k2z, 0.5f)), df_add(d0, df_scale2(k2d, 0.5f)), c,
                               dc, g1, g2, kw, kw2, dual, k3z, k3d);
            rk4_rhs_df<DT, ZS>(df_add(z0, k3z), df_add(d0, k3d), c, dc, g1, g2, kw, kw2, dual, k4z, k4d);
            const DF2 sz = df_add(df_add(k1z, k4z), df_scale2(df_add(k2z, k3z), 2.0f));
            const DF2 sd = df_add(df_add(k1d, k4d), df_scale2(df_add(k2d, k3d), 2.0f));
            acc2(z[p], df_mul(sz, DF2{sixth.h, sixth.l}));
            acc2(d[p], df_mul(sd, DF2{sixth.h, sixth.l}));
        }
    }
}

// One turn of the widened map: slippage expansion (g1*, g2*: stage i's w_i eta1 C,
// w_i eta2 C), second RF system (k2h, k2l: stage j's w_j A2) and, for RK4, the classic
// Runge-Kutta step.
template <int SCHEME, int DT, bool ZS>
__device__ __forceinline__ void long_turn_nl(DF (&z)[P], DF (&d)[P], const MapConsts& c,
                                             const float* dh, const float* dl, const float* kh,
                                             const float* kl, const float* k2h, const float* k2l,
                                             const float (&g1h)[4], const float (&g1l)[4],
                                             const float (&g2h)[4], const float (&g2l)[4], bool dual)
{
    if (SCHEME == PHTL_RK4) {
        rk4_turn<DT, ZS>(z, d, c, dh[0], dl[0], kh[0], kl[0], k2h[0], k2l[0], g1h[0], g1l[0],
                         g2h[0], g2l[0], dual);
    } else if (SCHEME == PHTL_EULER_CROMER) {
        kick_gen<DT, ZS>(z, d, kh[0], kl[0], k2h[0], k2l[0], c, dual);
        drift_nl<DT>(z, d, dh[0], dl[0], g1h[0], g1l[0], g2h[0], g2l[0]);
    } else if (SCHEME == PHTL_LEAPFROG) {
        drift_nl<DT>(z, d, dh[0], dl[0], g1h[0], g1l[0], g2h[0], g2l[0]);
        kick_gen<DT, ZS>(z, d, kh[0], kl[0], k2h[0], k2l[0], c, dual);
        drift_nl<DT>(z, d, dh[1], dl[1], g1h[1], g1l[1], g2h[1], g2l[1]);
    } else {
        drift_nl<DT>(z, d, dh[0], dl[0], g1h[0], g1l[0], g2h[0], g2l[0]);
        kick_gen<DT, ZS>(z, d, kh[0], kl[0], k2h[0], k2l[0], c, dual);
        drift_nl<DT>(z, d, dh[1], dl[1], g1h[1], g1l[1], g2h[1], g2l[1]);
        kick_gen<DT, ZS>(z, d, kh[1], kl[1], k2h[1], k2l[1], c, dual);
        drift_nl<DT>(z, d, dh[2], dl[2], g1h[2], g1l[2], g2h[2], g2l[2]);
        kick_gen<DT, ZS>(z, d, kh[2], kl[2], k2h[2], k2l[2], c, dual);
        drift_nl<DT>(z, d, dh[3], dl[3], g1h[3], g1l[3], g2h[3], g2l[3]);
    }
}

// Stage constants w_i eta1 C and w_i eta2 C of this scheme as float pairs (loop-invariant).
template <int SCHEME>
__device__ __forceinline__ void slip_stages(const MapConsts& c, float (&g1h)[4], float (&g1l)[4],
                                            float (&g2h)[4], float (&g2l)[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const DF2 a = split_bits(drift_weight(SCHEME, i) * c.eta1C);
        const DF2 b = split_bits(drift_weight(SCHEME, i) * c.eta2C);
        g1h[i] = a.h;
        g1l[i] = a.l;
        g2h[i] = b.h;
        g2l[i] = b.l;
    }
}

// sin and cos of 2 pi a, a in turns as a float pair (the chromatic phase advance):
// quarter-turn reduction a = n/4 + f with a.h - n/4 exact (Sterbenz), r = 2 pi f in
// double-float, then the sine and cosine polynomials of sin_df on r (the two leading
// Horner steps in double-float, the trailing terms in FP32) and the quadrant's swap and
// signs.  |a| >= 1e4 turns takes the FP64 form.
__device__ __forceinline__ void sincos_df_turns(DF2 a, DF2& s, DF2& c)
{
    if (!(fabsf(a.h) < 1.0e4f)) {
        double sd, cd;
        sincos_turns(widen_bits(a.h) + widen_bits(a.l), sd, cd);
        s = split_bits(sd);
        c = split_bits(cd);
        return;
    }
    const float magic = 12582912.0f;
    const float tf = __fmaf_rn(a.h, 4.0f, magic);
    const int ni = __float_as_int(tf);
    const float nq = __fmul_rn(__fsub_rn(tf, magic), 0.25f);
    const DF2 hd = df_two_sum(a.h, -nq);
    const DF2 f = df_fast_two_sum(hd.h, __fadd_rn(hd.l, a.l));
    constexpr DFC tp(6.283185307179586);
    const DF2 r = df_mul(f, DF2{tp.h, tp.l});
    const DF2 t = df_mul(r, r);
    float ts = 1.5918129294866608e-10f, tc = -1.1382632425521717e-11f;
    ts = __fmaf_rn(ts, t.h, -2.5051131845003624e-08f);
    tc = __fmaf_rn(tc, t.h, 2.08761462684032e-09f);
    ts = __fmaf_rn(ts, t.h, 2.755731610255244e-06f);
    tc = __fmaf_rn(tc, t.h, -2.7557317271729793e-07f);
    ts = __fmaf_rn(ts, t.h, -0.00019841269836758574f);
    tc = __fmaf_rn(tc, t.h, 2.480158729876569e-05f);
    constexpr DFC s1(0.008333333333330948), s0(-0.16666666666666666);
    constexpr DFC c1(-0.0013888888888887398), c0(0.041666666666666664);
    DF2 us = df_add_dominant(DF2{s1.h, s1.l}, df_mul_f(t, ts));
    us = df_add_dominant(DF2{s0.h, s0.l}, df_mul(t, us));
    DF2 uc = df_add_dominant(DF2{c1.h, c1.l}, df_mul_f(t, tc));
    uc = df_add_dominant(DF2{c0.h, c0.l}, df_mul(t, uc));
    const DF2 sr = df_add_dominant(r, df_mul(df_mul(r, t), us));
    const DF2 cr = df_add_dominant(df_add_dominant(DF2{1.0f, 0.0f}, DF2{-0.5f * t.h, -0.5f * t.l}),
                                   df_mul(df_mul(t, t), uc));
    const bool swap = (ni & 1) != 0;
    // n mod 4 = 0: (sr, cr); 1: (cr, -sr); 2: (-sr, -cr); 3: (-cr, sr)
    s = df_xor_sign(swap ? cr : sr, static_cast<unsigned>(ni & 2) << 30);
    c = df_xor_sign(swap ? sr : cr, static_cast<unsigned>((ni + 1) & 2) << 30);
}

// Chromatic rotation of one plane, each particle by 2 pi (q + xi d) with its own d.
// PHTL_F32C / PHTL_F32CD: angle, sine and cosine and the rotation in double-float;
// PHTL_F32CS: the angle in FP32, the SFU's sine and cosine, the rotation in double-float.
template <int DT>
__device__ __forceinline__ void rotate_chroma(DF (&u)[P], DF (&v)[P], const DF (&d)[P], float qh,
                                              float ql, float xh, float xl, float bh, float bl,
                                              float ibh, float ibl)
{
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (DT == PHTL_F32CS) {
            float a = __fmaf_rn(xh, d[p].hi, qh);
            a = __fsub_rn(a, rintf(a));
            float sn, cs;
            __sincosf(6.28318530717958647692f * a, &sn, &cs);
            const float mh[4] = {cs, bh * sn, -(sn * ibh), cs};
            const float ml[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            df_rotate(u[p], v[p], mh, ml);
        } else {
            DF2 sn, cs;
            sincos_df_turns(df_add(DF2{qh, ql}, df_mul(DF2{xh, xl}, as2(d[p]))), sn, cs);
            const DF2 bs = df_mul(DF2{bh, bl}, sn);
            const DF2 sib = df_mul(DF2{ibh, ibl}, sn);
            const DF2 un = df_add(df_mul(cs, as2(u[p])), df_mul(bs, as2(v[p])));
            const DF2 vn = df_add(df_mul(cs, as2(v[p])), neg2(df_mul(sib, as2(u[p]))));
            u[p] = DF{un.h, un.l};
            v[p] = DF{vn.h, vn.l};
        }
    }
}

// The transverse step of the general loop: chromatic where xi != 0, else the one matrix.
template <int DT>
__device__ __forceinline__ void transverse_gen(DF (&x)[P], DF (&xp)[P], DF (&y)[P], DF (&yp)[P],
                                               const DF (&d)[P], bool hx, bool hy,
                                               const MapConsts& c)
{
    if (hx) {
        if (c.chroma_x) {
            rotate_chroma<DT>(x, xp, d, c.qx_hi, c.qx_lo, c.xi_x_hi, c.xi_x_lo, c.bx_hi, c.bx_lo,
                              c.ibx_hi, c.ibx_lo);
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) df_rotate(x[p], xp[p], c.mx_hi, c.mx_lo);
        }
    }
    if (hy) {
        if (c.chroma_y) {
            rotate_chroma<DT>(y, yp, d, c.qy_hi, c.qy_lo, c.xi_y_hi, c.xi_y_lo, c.by_hi, c.by_lo,
                              c.iby_hi, c.iby_lo);
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) df_rotate(y[p], yp[p], c.my_hi, c.my_lo);
        }
    }
}

__device__ __forceinline__ void pair_sums(const DF (&a)[P], const DF (&b)[P], float* f)
{
    f[0] = a[0].hi;
    f[1] = b[0].hi;
    f[2] = a[0].hi * a[0].hi;
    f[3] = b[0].hi * b[0].hi;
    f[4] = a[0].hi * b[0].hi;
#pragma unroll
    for (int p = 1; p < P; ++p) {
        f[0] += a[p].hi;
        f[1] += b[p].hi;
        f[2] = fmaf(a[p].hi, a[p].hi, f[2]);
        f[3] = fmaf(b[p].hi, b[p].hi, f[3]);
        f[4] = fmaf(a[p].hi, b[p].hi, f[4]);
    }
}

// FP32 warp reduce-scatter (same butterfly as the FP64 one in monitor.cuh).
template <int NF>
__device__ __forceinline__ float warp_reduce_scatter_f(float (&f)[NF], int lane)
{
#pragma unroll
    for (int o = 16; o >= (NF == 16 ? 2 : 4); o >>= 1) {
        const int h = (NF == 16) ? (o >> 1) : (o >> 2);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < NF / 2; ++i) {
            if (i < h) {
                float send = upper ? f[i] : f[i + h];
                float keep = upper ? f[i + h] : f[i];
                f[i] = keep + __shfl_xor_sync(kFullMask, send, o);
            }
        }
    }
    float v = f[0];
    if (NF == 8) v += __shfl_xor_sync(kFullMask, v, 2);
    v += __shfl_xor_sync(kFullMask, v, 1);
    return v;
}

template <bool TRANS>
__device__ __forceinline__ void record(const DF (&z)[P], const DF (&d)[P], const DF (&x)[P],
                                       const DF (&xp)[P], const DF (&y)[P], const DF (&yp)[P],
                                       float cnt, bool hx, bool hy, double* smem, int parity,
                                       double* rows, int64_t row)
{
    constexpr int NF = TRANS ? 16 : 8;
    float f[NF];
    f[0] = cnt;
    pair_sums(z, d, f + 1);
    if constexpr (TRANS) {
        if (hx) {
            pair_sums(x, xp, f + 6);
        } else {
#pragma unroll
            for (int j = 6; j < 11; ++j) f[j] = 0.0f;
        }
        if (hy) {
            pair_sums(y, yp, f + 11);
        } else {
#pragma unroll
            for (int j = 11; j < 16; ++j) f[j] = 0.0f;
        }
    } else {
        f[6] = 0.0f;
        f[7] = 0.0f;
    }
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const float v = warp_reduce_scatter_f<NF>(f, lane);
    double* buf = smem + parity * (nwarps * 16);
    constexpr int kShift = (NF == 16) ? 1 : 2;
    if ((lane & ((1 << kShift) - 1)) == 0) buf[warp * 16 + (lane >> kShift)] = static_cast<double>(v);
    __syncthreads();
    const int nvalid = TRANS ? 16 : 6;
    if (warp == 0 && lane < nvalid) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += buf[w * 16 + lane];
        atomicAdd(rows + row * PHTL_MON_FIELDS + lane, s);
    }
}

// 128-bit accesses only where the host allowed them (vec) AND both the hi and the comp
// addresses really are 16-byte aligned; anything else takes the scalar path.
__device__ __forceinline__ bool aligned16_pair(const float* a, const float* b)
{
    return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
}

__device__ __forceinline__ void load4(const float* __restrict__ g, int64_t base, int64_t n,
                                      bool vec, DF (&v)[P])
{
    if (vec && base + P <= n && aligned16_pair(g + base, g + n + base)) {
        const float4 h = __ldcs(reinterpret_cast<const float4*>(g + base));
        const float4 c = __ldcs(reinterpret_cast<const float4*>(g + n + base));
        v[0] = {h.x, c.x};
        v[1] = {h.y, c.y};
        v[2] = {h.z, c.z};
        v[3] = {h.w, c.w};
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const bool ok = base + p < n;
            v[p].hi = ok ? g[base + p] : 0.0f;
            v[p].c = ok ? g[n + base + p] : 0.0f;
        }
    }
}

__device__ __forceinline__ void store4(float* __restrict__ g, int64_t base, int64_t n, bool vec,
                                       const DF (&v)[P])
{
    if (vec && base + P <= n && aligned16_pair(g + base, g + n + base)) {
        __stcs(reinterpret_cast<float4*>(g + base), make_float4(v[0].hi, v[1].hi, v[2].hi, v[3].hi));
        __stcs(reinterpret_cast<float4*>(g + n + base), make_float4(v[0].c, v[1].c, v[2].c, v[3].c));
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            if (base + p < n) {
                g[base + p] = v[p].hi;
                g[n + base + p] = v[p].c;
            }
        }
    }
}

}  // namespace f32c
}  // namespace phtl
