// Ramp programme kernels: an accelerating bucket whose reference momentum p0_n and RF
// voltage V_n change from turn to turn (the paper's runs change the machine parameters;
// the per-turn reading is stated in phtl.h at phtl_set_programme).
//
// The same persistent structure as the fixed-machine kernels (Sec. 2.3: turn loop inside
// the kernel, state in registers, grid-stride over particle chunks), but each turn reads
// its constants -- eta_n C, A_n, phi_s,n, sin(phi_s,n), r_n = p0_n / p0_{n+1} -- from a
// device table that the host derived in FP64 (192 bytes per turn, the same address for
// every thread, so the loads are L1 broadcasts).  The next turn's phase constants are
// loaded while the current turn computes.  After the turn's stages and the transverse
// rotation, delta and the slopes x', y' are re-expressed against the next turn's reference
// momentum (multiplied by r_n).  Stage weights are the compile-time constants of the scheme
// times the turn's eta_n C and A_n: the FP64 kernels read these products from the table
// (the host formed them, the same FP64 products), the FP32 kernels form them as
// double-float products.  The kick is the general one (phi_s,n != 0 in general).
#include <cuda_runtime.h>

#include "internal.h"
#include "ops_f32c.cuh"
#include "ops_f64.cuh"

namespace phtl {
namespace {

// ---------------------------------------------------------------------------------- FP64
namespace rf64 {

using namespace f64;

struct Turn {
    double phis, sinphis, lin, r;
};

__device__ __forceinline__ Turn load_turn(const RampTurn* __restrict__ p)
{
    Turn t;
    t.phis = __ldg(&p->phis);
    t.sinphis = __ldg(&p->sinphis);
    t.lin = __ldg(&p->lin);
    t.r = __ldg(&p->r);
    return t;
}

// The scheme's stage weights of one turn, precomputed on the host as the FP64 products of
// the scheme's constants and eta_n C, A_n (drifts first, then kicks): the same values the
// device would form, without spending FP64 operations on them every turn.
template <int S>
__device__ __forceinline__ const double* stage_weights(const RampTurn* __restrict__ e)
{
    return S == PHTL_EULER_CROMER ? e->w_ec : (S == PHTL_LEAPFROG ? e->w_lf : e->w_r4);
}

// delta += kw (sin(phi_s,n + k z) - sin(phi_s,n)), kw this stage's weight times A_n
__device__ __forceinline__ void kick(const double (&z)[P], double (&d)[P], double kw,
                                     const Turn& T, const MapConsts& c)
{
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double f = c.linear ? T.lin * z[p] : sin_f64(fma(c.k, z[p], T.phis)) - T.sinphis;
        d[p] = fma(kw, f, d[p]);
    }
}

template <int S>
__device__ __forceinline__ void turn(double (&z)[P], double (&d)[P], const Turn& T, const MapConsts& c,
                                     const double* __restrict__ w)
{
    if (S == PHTL_EULER_CROMER) {
        kick(z, d, __ldg(w + 1), T, c);
        drift(z, d, __ldg(w + 0));
    } else if (S == PHTL_LEAPFROG) {
        drift(z, d, __ldg(w + 0));
        kick(z, d, __ldg(w + 2), T, c);
        drift(z, d, __ldg(w + 1));
    } else {
        drift(z, d, __ldg(w + 0));
        kick(z, d, __ldg(w + 4), T, c);
        drift(z, d, __ldg(w + 1));
        kick(z, d, __ldg(w + 5), T, c);
        drift(z, d, __ldg(w + 2));
        kick(z, d, __ldg(w + 6), T, c);
        drift(z, d, __ldg(w + 3));
    }
}

template <int S>
__global__ void __launch_bounds__(256, 2)
    k_ramp_f64(LaunchDesc L, MapConsts c, MonitorArgs m, const RampTurn* __restrict__ prog, int64_t turn0)
{
    if (L.go && *L.go == 0) return;  // the call was cancelled before this launch
    extern __shared__ double smem[];
    double* g[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = static_cast<double*>(L.c[i]);
    const bool hx = g[2] != nullptr, hy = g[4] != nullptr;
    const bool vec = L.vec != 0;
    const int64_t chunk = static_cast<int64_t>(blockDim.x) * P;
    const int64_t nchunks = (L.n + chunk - 1) / chunk;
    int parity = 0;
    for (int64_t ci = blockIdx.x; ci < nchunks; ci += gridDim.x) {
        const int64_t base = ci * chunk + static_cast<int64_t>(threadIdx.x) * P;
        double z[P], d[P], x[P], xp[P], y[P], yp[P];
        load2(g[0], base, L.n, vec, z);
        load2(g[1], base, L.n, vec, d);
#pragma unroll
        for (int p = 0; p < P; ++p) x[p] = xp[p] = y[p] = yp[p] = 0.0;
        if (hx) {
            load2(g[2], base, L.n, vec, x);
            load2(g[3], base, L.n, vec, xp);
        }
        if (hy) {
            load2(g[4], base, L.n, vec, y);
            load2(g[5], base, L.n, vec, yp);
        }
        const int64_t left = L.n - base;
        const float cnt = left >= P ? static_cast<float>(P) : (left > 0 ? static_cast<float>(left) : 0.0f);
        if (m.rows && m.initial) {
            record<true>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, m.rows, 0);
            parity ^= 1;
        }
        int64_t until = m.until, row = m.row;
        Turn T{};
        if (L.nturns > 0) T = load_turn(prog + turn0);  // a launch reads turns [turn0, turn0 + nturns) only
        for (int t = 0; t < L.nturns; ++t) {
            // the next turn's constants, loaded while this turn computes
            const Turn Tn = load_turn(prog + turn0 + (t + 1 < L.nturns ? t + 1 : t));
            turn<S>(z, d, T, c, stage_weights<S>(prog + turn0 + t));
            if (hx) rotate(x, xp, c.mx, c.shx, c.shear_x != 0);
            if (hy) rotate(y, yp, c.my, c.shy, c.shear_y != 0);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                d[p] = T.r * d[p];
                xp[p] = T.r * xp[p];
                yp[p] = T.r * yp[p];
            }
            if (m.rows && --until == 0) {
                record<true>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, m.rows, row);
                parity ^= 1;
                ++row;
                until = m.stride;
            }
            T = Tn;
        }
        store2(g[0], base, L.n, vec, z);
        store2(g[1], base, L.n, vec, d);
        if (hx) {
            store2(g[2], base, L.n, vec, x);
            store2(g[3], base, L.n, vec, xp);
        }
        if (hy) {
            store2(g[4], base, L.n, vec, y);
            store2(g[5], base, L.n, vec, yp);
        }
    }
}

}  // namespace rf64

// ---------------------------------------------------------------------------------- FP32C
namespace rf32 {

using namespace f32c;

struct Turn {
    DF2 etaC, A, phis, sinphis, lin, r;
    double phis64;  // PHTL_F32C forms the phase in FP64
};

template <int DT>
__device__ __forceinline__ Turn load_turn(const RampTurn* __restrict__ p)
{
    Turn t;
    t.etaC = DF2{__ldg(&p->etaC_h), __ldg(&p->etaC_l)};
    t.A = DF2{__ldg(&p->A_h), __ldg(&p->A_l)};
    t.phis = DF2{__ldg(&p->phis_h), __ldg(&p->phis_l)};
    t.sinphis = DF2{__ldg(&p->sinphis_h), __ldg(&p->sinphis_l)};
    t.lin = DF2{__ldg(&p->lin_h), __ldg(&p->lin_l)};
    t.r = DF2{__ldg(&p->r_h), __ldg(&p->r_l)};
    t.phis64 = DT == PHTL_F32C ? __ldg(&p->phis) : 0.0;
    return t;
}

// kick of weight w (a compile-time constant of the scheme): delta += w A_n (sin(phi_s,n +
// k z) - sin(phi_s,n)), the phase in FP64 (PHTL_F32C), double-float (PHTL_F32CD) or
// rounded to FP32 for the SFU sine (PHTL_F32CS)
template <int DT>
__device__ __forceinline__ void kick(const DF (&z)[P], DF (&d)[P], double w, const Turn& T,
                                     const MapConsts& c)
{
    const DFC wc(w);
    const DF2 kw = df_mul(DF2{wc.h, wc.l}, T.A);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        if (DT == PHTL_F32CS) {
            float f;
            if (c.linear) {
                f = T.lin.h * (z[p].hi + z[p].c);
            } else {
                const DF2 ph = df_add(df_mul(DF2{c.k_hi, c.k_lo}, as2(z[p])), T.phis);
                f = sin_sfu(__fadd_rn(ph.h, ph.l)) - T.sinphis.h;
            }
            acc(d[p], __fmaf_rn(kw.h, f, __fmul_rn(kw.l, f)));
        } else {
            DF2 f;
            if (c.linear) {
                f = df_mul(T.lin, as2(z[p]));
            } else {
                DF2 ph;
                if (DT == PHTL_F32C) {
                    const double zd = widen_float_phase(z[p].hi) + widen_float_phase(z[p].c);
                    ph = split_phase(fma(c.k, zd, T.phis64));
                } else {
                    ph = df_add(df_mul(DF2{c.k_hi, c.k_lo}, as2(z[p])), T.phis);
                }
                f = df_add(sin_df(ph), neg2(T.sinphis));
            }
            acc2(d[p], df_mul(kw, f));
        }
    }
}

template <int DT>
__device__ __forceinline__ void drift_w(DF (&z)[P], const DF (&d)[P], double w, const Turn& T)
{
    const DFC wc(w);
    const DF2 dc = df_mul(DF2{wc.h, wc.l}, T.etaC);
    drift<DT>(z, d, dc.h, dc.l);
}

template <int S, int DT>
__device__ __forceinline__ void turn(DF (&z)[P], DF (&d)[P], const Turn& T, const MapConsts& c)
{
    if (S == PHTL_EULER_CROMER) {
        kick<DT>(z, d, kick_weight(S, 0), T, c);
        drift_w<DT>(z, d, drift_weight(S, 0), T);
    } else if (S == PHTL_LEAPFROG) {
        drift_w<DT>(z, d, drift_weight(S, 0), T);
        kick<DT>(z, d, kick_weight(S, 0), T, c);
        drift_w<DT>(z, d, drift_weight(S, 1), T);
    } else {
        drift_w<DT>(z, d, drift_weight(S, 0), T);
        kick<DT>(z, d, kick_weight(S, 0), T, c);
        drift_w<DT>(z, d, drift_weight(S, 1), T);
        kick<DT>(z, d, kick_weight(S, 1), T, c);
        drift_w<DT>(z, d, drift_weight(S, 2), T);
        kick<DT>(z, d, kick_weight(S, 2), T, c);
        drift_w<DT>(z, d, drift_weight(S, 3), T);
    }
}

// u <- r u as a double-float product, renormalised
__device__ __forceinline__ void scale(DF& u, DF2 r)
{
    const DF2 v = df_mul(r, as2(u));
    u.hi = v.h;
    u.c = v.l;
}

template <int S, int DT>
__device__ __forceinline__ void ramp_f32c_body(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                                               const RampTurn* __restrict__ prog, int64_t turn0)
{
    if (L.go && *L.go == 0) return;  // the call was cancelled before this launch
    extern __shared__ double smem[];
    float* g[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = static_cast<float*>(L.c[i]);
    const bool hx = g[2] != nullptr, hy = g[4] != nullptr;
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
        if (m.rows && m.initial) {
            record<true>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, m.rows, 0);
            parity ^= 1;
        }
        int64_t until = m.until, row = m.row;
        Turn T{};
        if (L.nturns > 0) T = load_turn<DT>(prog + turn0);  // a launch reads turns [turn0, turn0 + nturns) only
        for (int t = 0; t < L.nturns; ++t) {
            const Turn Tn = load_turn<DT>(prog + turn0 + (t + 1 < L.nturns ? t + 1 : t));
            turn<S, DT>(z, d, T, c);
            if (hx) {
#pragma unroll
                for (int p = 0; p < P; ++p) df_rotate(x[p], xp[p], c.mx_hi, c.mx_lo);
            }
            if (hy) {
#pragma unroll
                for (int p = 0; p < P; ++p) df_rotate(y[p], yp[p], c.my_hi, c.my_lo);
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                scale(d[p], T.r);
                if (hx) scale(xp[p], T.r);
                if (hy) scale(yp[p], T.r);
            }
            if (m.rows && --until == 0) {
                record<true>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, m.rows, row);
                parity ^= 1;
                ++row;
                until = m.stride;
            }
            T = Tn;
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

// FP32CD and FP32CS: the compiler's register choice; FP32C: 3 resident 256-thread blocks per SM
// (80 registers), 6.6 % faster over the three schemes (1e6 particles x 1000 turns, transverse,
// a monitor row every turn; FP32CD and FP32CS gained nothing at 2 or 3 blocks)
template <int S, int DT>
__global__ void PHTL_F32C_RAMP_BOUNDS(S, DT)
    k_ramp_f32c(LaunchDesc L, MapConsts c, MonitorArgs m, const RampTurn* __restrict__ prog, int64_t turn0)
{
    ramp_f32c_body<S, DT>(L, c, m, prog, turn0);
}

template <int S>
__global__ void PHTL_F32C_RAMP_BOUNDS_C
    k_ramp_f32c_c(LaunchDesc L, MapConsts c, MonitorArgs m, const RampTurn* __restrict__ prog, int64_t turn0)
{
    ramp_f32c_body<S, PHTL_F32C>(L, c, m, prog, turn0);
}

}  // namespace rf32

template <int S>
const void* ramp_kernel_s(int dtype)
{
    if (dtype == PHTL_F64) return reinterpret_cast<const void*>(&rf64::k_ramp_f64<S>);
    if (dtype == PHTL_F32C) return reinterpret_cast<const void*>(&rf32::k_ramp_f32c_c<S>);
    if (dtype == PHTL_F32CD) return reinterpret_cast<const void*>(&rf32::k_ramp_f32c<S, PHTL_F32CD>);
    if (dtype == PHTL_F32CS) return reinterpret_cast<const void*>(&rf32::k_ramp_f32c<S, PHTL_F32CS>);
    return nullptr;
}

const void* ramp_kernel(int scheme, int dtype)
{
    if (scheme == PHTL_EULER_CROMER) return ramp_kernel_s<PHTL_EULER_CROMER>(dtype);
    if (scheme == PHTL_LEAPFROG) return ramp_kernel_s<PHTL_LEAPFROG>(dtype);
    if (scheme == PHTL_RUTH4) return ramp_kernel_s<PHTL_RUTH4>(dtype);
    return nullptr;
}

size_t ramp_smem(int block) { return 2u * (block / 32) * 16 * sizeof(double); }

}  // namespace

int occupancy_ramp(int scheme, int dtype, int block)
{
    const void* k = ramp_kernel(scheme, dtype);
    if (!k) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, ramp_smem(block)) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_ramp(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                        const RampTurn* prog, int64_t turn0, int dtype, cudaStream_t s)
{
    const void* k = ramp_kernel(L.scheme, dtype);
    if (!k) return cudaErrorInvalidValue;
    LaunchDesc Lc = L;
    MapConsts cc = c;
    MonitorArgs mm = m;
    const RampTurn* pp = prog;
    int64_t tt = turn0;
    void* args[] = {&Lc, &cc, &mm, &pp, &tt};
    return cudaLaunchKernel(k, dim3(L.grid), dim3(L.block), args, ramp_smem(L.block), s);
}

}  // namespace phtl
