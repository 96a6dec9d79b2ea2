// FP32-compensated per-particle operations shared by the FP32C kernels (single bunch
// and batched).  Every coordinate is an unevaluated sum hi + comp of two floats; see
// track_f32c.cu for the arithmetic model.  One thread owns P = 4 particles.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "monitor.cuh"

namespace phtl {
namespace f32c {

constexpr int P = 4;
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

// Phase argument phi = phi_s + k z rounded to FP32 and reduced to [-pi, pi].
template <int DT>
__device__ __forceinline__ float phase(const MapConsts& c, const DF& z)
{
    float ph;
    if (DT == PHTL_F32C) {
        // FP64: hi + comp is exact in double; one DFMA, then round to FP32
        const double zd = static_cast<double>(z.hi) + static_cast<double>(z.c);
        ph = static_cast<float>(fma(c.k, zd, c.phis));
    } else {
        // double-float: exact FP32 product k_hi * z_hi plus the cross terms, plus phi_s
        const float p = __fmul_rn(c.k_hi, z.hi);
        float e = __fmaf_rn(c.k_hi, z.hi, -p);
        e = __fmaf_rn(c.k_hi, z.c, __fmaf_rn(c.k_lo, z.hi, e));
        const float s = __fadd_rn(p, c.phis_hi);
        const float bb = __fsub_rn(s, p);
        const float err = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.phis_hi, bb));
        ph = __fadd_rn(s, __fadd_rn(err, __fadd_rn(e, c.phis_lo)));
    }
    // reduce by 2 pi (two-part constant) so the SFU sine sees |arg| <= ~pi
    const float nq = rintf(ph * kInvTwoPi);
    return __fmaf_rn(-nq, kTwoPiLo, __fmaf_rn(-nq, kTwoPiHi, ph));
}

template <int DT>
__device__ __forceinline__ float rf_force(const MapConsts& c, const DF& z)
{
    if (c.linear) return c.lin_f * (z.hi + z.c);
    return __sinf(phase<DT>(c, z)) - c.sinphis_f;
}

template <int DT>
__device__ __forceinline__ void kick(const DF (&z)[P], DF (&d)[P], float kw, const MapConsts& c)
{
#pragma unroll
    for (int p = 0; p < P; ++p) acc(d[p], __fmul_rn(kw, rf_force<DT>(c, z[p])));
}

__device__ __forceinline__ void drift(DF (&z)[P], const DF (&d)[P], float dc)
{
#pragma unroll
    for (int p = 0; p < P; ++p) acc(z[p], __fmul_rn(-dc, d[p].hi));
}

// dc, kw: FP32 drift and kick weights of this bunch's scheme (the single-bunch kernel
// passes c.dc_hi, c.kw_hi, the batched kernel the job table's copies).
template <int SCHEME, int DT>
__device__ __forceinline__ void long_turn(DF (&z)[P], DF (&d)[P], const MapConsts& c,
                                          const float* dc, const float* kw)
{
    if (SCHEME == PHTL_EULER_CROMER) {
        kick<DT>(z, d, kw[0], c);
        drift(z, d, dc[0]);
    } else if (SCHEME == PHTL_LEAPFROG) {
        drift(z, d, dc[0]);
        kick<DT>(z, d, kw[0], c);
        drift(z, d, dc[1]);
    } else {
        drift(z, d, dc[0]);
        kick<DT>(z, d, kw[0], c);
        drift(z, d, dc[1]);
        kick<DT>(z, d, kw[1], c);
        drift(z, d, dc[2]);
        kick<DT>(z, d, kw[2], c);
        drift(z, d, dc[3]);
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
    if (TRANS) {
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
