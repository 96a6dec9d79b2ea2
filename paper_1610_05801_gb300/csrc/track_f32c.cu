// FP32-compensated persistent multi-turn tracking kernel (PHTL_F32C, PHTL_F32CD).
//
// Same structure as the FP64 kernel (Sec. 2.3: turn loop inside the kernel, state in
// registers), but every coordinate is an unevaluated sum hi + comp of two floats:
//   - each drift/kick increment is computed in FP32 and added with Knuth's TwoSum, the
//     rounding error going into comp, followed by a Fast2Sum renormalisation;
//   - the RF phase argument k z is formed from hi + comp either in FP64 (PHTL_F32C) or
//     in double-float FP32-pair arithmetic (PHTL_F32CD), reduced to [-pi, pi] and
//     rounded to FP32 for the SFU sine (__sinf);
//   - the transverse matrix (Sec. 1.1.1) is applied in double-float arithmetic (exact
//     FP32 products by fmaf, TwoSum of the two terms), so the rotation keeps ~48 bits;
//   - per-turn moment sums are FP32 per thread and across the warp (<= 128 particles),
//     then FP64 across warps and blocks.
// Each thread owns P = 4 particles (one 128-bit load of hi and one of comp per
// coordinate).  This kernel is FP32-pipe / issue bound; the FP64 variant of the phase
// argument adds a handful of FP64-pipe operations per kick.
#include <cuda_runtime.h>

#include "internal.h"
#include "monitor.cuh"

namespace phtl {
namespace {

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

template <int SCHEME, int DT>
__device__ __forceinline__ void long_turn(DF (&z)[P], DF (&d)[P], const MapConsts& c)
{
    if (SCHEME == PHTL_EULER_CROMER) {
        kick<DT>(z, d, c.kw_hi[0], c);
        drift(z, d, c.dc_hi[0]);
    } else if (SCHEME == PHTL_LEAPFROG) {
        drift(z, d, c.dc_hi[0]);
        kick<DT>(z, d, c.kw_hi[0], c);
        drift(z, d, c.dc_hi[1]);
    } else {
        drift(z, d, c.dc_hi[0]);
        kick<DT>(z, d, c.kw_hi[0], c);
        drift(z, d, c.dc_hi[1]);
        kick<DT>(z, d, c.kw_hi[1], c);
        drift(z, d, c.dc_hi[2]);
        kick<DT>(z, d, c.kw_hi[2], c);
        drift(z, d, c.dc_hi[3]);
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

__device__ __forceinline__ void load4(const float* __restrict__ g, int64_t base, int64_t n,
                                      bool vec, DF (&v)[P])
{
    if (vec && base + P <= n) {
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
    if (vec && base + P <= n) {
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

template <int SCHEME, int DT, bool TRANS, bool MON>
__global__ void __launch_bounds__(256) k_track_f32c(LaunchDesc L, MapConsts c, MonitorArgs m)
{
    extern __shared__ double smem[];
    float* g[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = static_cast<float*>(L.c[i]);
    const bool hx = TRANS && g[2] != nullptr;
    const bool hy = TRANS && g[4] != nullptr;
    const bool vec = L.vec != 0;
    const int64_t chunk = static_cast<int64_t>(blockDim.x) * P;
    const int64_t nchunks = (L.n + chunk - 1) / chunk;
    int parity = 0;

    for (int64_t ci = blockIdx.x; ci < nchunks; ci += gridDim.x) {
        const int64_t base = ci * chunk + static_cast<int64_t>(threadIdx.x) * P;
        DF z[P], d[P], x[P], xp[P], y[P], yp[P];
        load4(g[0], base, L.n, vec, z);
        load4(g[1], base, L.n, vec, d);
#pragma unroll
        for (int p = 0; p < P; ++p) x[p] = xp[p] = y[p] = yp[p] = DF{0.0f, 0.0f};
        if (hx) {
            load4(g[2], base, L.n, vec, x);
            load4(g[3], base, L.n, vec, xp);
        }
        if (hy) {
            load4(g[4], base, L.n, vec, y);
            load4(g[5], base, L.n, vec, yp);
        }
        const int64_t left = L.n - base;
        const float cnt = left >= P ? static_cast<float>(P) : (left > 0 ? static_cast<float>(left) : 0.0f);

        int64_t until = m.until, row = m.row;
        if (MON && m.initial) {
            record<TRANS>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, m.rows, 0);
            parity ^= 1;
        }
        for (int t = 0; t < L.nturns; ++t) {
            long_turn<SCHEME, DT>(z, d, c);
            if (TRANS) {
                if (hx) {
#pragma unroll
                    for (int p = 0; p < P; ++p) df_rotate(x[p], xp[p], c.mx_hi, c.mx_lo);
                }
                if (hy) {
#pragma unroll
                    for (int p = 0; p < P; ++p) df_rotate(y[p], yp[p], c.my_hi, c.my_lo);
                }
            }
            if (MON) {
                if (--until == 0) {
                    record<TRANS>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, m.rows, row);
                    parity ^= 1;
                    ++row;
                    until = m.stride;
                }
            }
        }
        store4(g[0], base, L.n, vec, z);
        store4(g[1], base, L.n, vec, d);
        if (hx) {
            store4(g[2], base, L.n, vec, x);
            store4(g[3], base, L.n, vec, xp);
        }
        if (hy) {
            store4(g[4], base, L.n, vec, y);
            store4(g[5], base, L.n, vec, yp);
        }
    }
}

template <int S, int D, bool T, bool M>
const void* kptr()
{
    return reinterpret_cast<const void*>(&k_track_f32c<S, D, T, M>);
}

template <int S, int D>
const void* sel_tm(bool trans, bool mon)
{
    if (trans) return mon ? kptr<S, D, true, true>() : kptr<S, D, true, false>();
    return mon ? kptr<S, D, false, true>() : kptr<S, D, false, false>();
}

template <int S>
const void* sel_d(int dtype, bool trans, bool mon)
{
    if (dtype == PHTL_F32C) return sel_tm<S, PHTL_F32C>(trans, mon);
    if (dtype == PHTL_F32CD) return sel_tm<S, PHTL_F32CD>(trans, mon);
    return nullptr;
}

const void* select_kernel(int scheme, int dtype, bool trans, bool mon)
{
    if (scheme == PHTL_EULER_CROMER) return sel_d<PHTL_EULER_CROMER>(dtype, trans, mon);
    if (scheme == PHTL_LEAPFROG) return sel_d<PHTL_LEAPFROG>(dtype, trans, mon);
    if (scheme == PHTL_RUTH4) return sel_d<PHTL_RUTH4>(dtype, trans, mon);
    return nullptr;
}

}  // namespace

int occupancy_f32c(int scheme, bool trans, bool mon, int dtype, int block)
{
    const void* k = select_kernel(scheme, dtype, trans, mon);
    if (!k) return 0;
    int nb = 0;
    const size_t smem = mon ? 2u * (block / 32) * 16 * sizeof(double) : 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_track_f32c(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                              int dtype, cudaStream_t s)
{
    const bool trans = L.c[2] != nullptr || L.c[4] != nullptr;
    const bool mon = m.rows != nullptr;
    const void* k = select_kernel(L.scheme, dtype, trans, mon);
    if (!k) return cudaErrorInvalidValue;
    const size_t smem = mon ? 2u * (L.block / 32) * 16 * sizeof(double) : 0;
    LaunchDesc Lc = L;
    MapConsts cc = c;
    MonitorArgs mm = m;
    void* args[] = {&Lc, &cc, &mm};
    return cudaLaunchKernel(k, dim3(L.grid), dim3(L.block), args, smem, s);
}

}  // namespace phtl
