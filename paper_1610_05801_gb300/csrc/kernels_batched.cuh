// Batched persistent tracking of many independent bunches in one launch.
// (Also the device side of the serving loop, which launches it once per scheduling round
// with each job's own turn offset.)
//
// The paper's parallel axis (Sec. 2.3: independent particles, sequential turns) applied
// to a batch of bunches of very different sizes, turn counts and RF voltages: a device
// job table lists the bunches, sorted by turns (longest first), and every block tracks
// one particle tile of one job for the launch's turn chunk [t0, t0 + T).  The block
// finds its job by a binary search of the table's tile offsets.  Because the table is
// sorted by turns, the jobs still running at chunk t0 are a prefix of the table, so the
// host launches exactly their tiles, heaviest first (the hardware block scheduler then
// deals them like a longest-processing-time list).  Per-particle arithmetic is the same
// code as the single-bunch kernels (ops_f64.cuh, ops_f32c.cuh), so a bunch tracked in a
// batch gives bitwise the same particles as tracked alone.
//
// Kernel templates; instantiated by track_batched.cu for the linear map and by
// track_general_batched.cu for the widened map.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "ops_f32c.cuh"
#include "ops_f64.cuh"

namespace phtl {
namespace {

__device__ __forceinline__ int find_job(const JobDesc* __restrict__ jobs, int njobs, int64_t tile)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile_begin <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------------- FP64
template <int SCHEME, bool MON, bool ZS, bool GEN>
__device__ __forceinline__ void run_f64_zs(double (&z)[f64::P], double (&d)[f64::P],
                                        double (&x)[f64::P], double (&xp)[f64::P],
                                        double (&y)[f64::P], double (&yp)[f64::P], bool hx,
                                        bool hy, const MapConsts& c, const JobDesc& J,
                                        float cnt, int64_t t0, int nt, double* smem, int& parity)
{
    const int64_t g0 = t0 + J.turn_offset;  // turns done before this launch
    int64_t until = J.stride - (g0 % J.stride);
    int64_t row = g0 / J.stride + 1;
    double g1[4], g2[4];
    if (GEN) f64::slip_stages<SCHEME>(c, g1, g2);
    for (int t = 0; t < nt; ++t) {
        if (GEN) {
            f64::long_turn_nl<SCHEME, ZS>(z, d, c, J.dc, J.kw, J.kw2, g1, g2, c.dual_rf != 0);
            f64::transverse_gen(x, xp, y, yp, d, hx, hy, c);
        } else {
            f64::long_turn<SCHEME, ZS>(z, d, c, J.dc, J.kw);
            if (hx) f64::rotate(x, xp, c.mx, c.shx, c.shear_x != 0);
            if (hy) f64::rotate(y, yp, c.my, c.shy, c.shear_y != 0);
        }
        if (MON && J.mon) {
            if (--until == 0) {
                // a longitudinal job reduces its 6 fields only (8 lanes' worth of butterfly)
                if (hx || hy)
                    f64::record<true>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, J.mon, row);
                else
                    f64::record<false>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, J.mon, row);
                parity ^= 1;
                ++row;
                until = J.stride;
            }
        }
    }
}

template <int SCHEME, bool MON, bool GEN>
__device__ __forceinline__ void run_f64(double (&z)[f64::P], double (&d)[f64::P],
                                        double (&x)[f64::P], double (&xp)[f64::P],
                                        double (&y)[f64::P], double (&yp)[f64::P], bool hx,
                                        bool hy, const MapConsts& c, const JobDesc& J,
                                        float cnt, int64_t t0, int nt, double* smem, int& parity)
{
    if (c.phis_zero)
        run_f64_zs<SCHEME, MON, true, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
    else
        run_f64_zs<SCHEME, MON, false, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
}

// GEN: the widened map (separate kernels chosen on the host; built with MON = true, the
// per-job monitor pointer is checked at run time).
template <bool MON, bool GEN>
__global__ void __launch_bounds__(256, f64::kBatchedMinBlocks256) k_batched_f64(const JobDesc* __restrict__ jobs, int njobs,
                                                     MapConsts c, int64_t t0, int T)
{
    using namespace f64;
    extern __shared__ double smem[];
    const JobDesc J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int64_t left_turns = J.turns - t0;
    const int nt = static_cast<int>(left_turns < T ? (left_turns > 0 ? left_turns : 0) : T);
    const bool mon = MON && J.mon != nullptr;
    const bool first = t0 + J.turn_offset == 0;
    if (nt == 0 && !(mon && first)) return;  // block-uniform
    double* gz = static_cast<double*>(J.c[0]);
    double* gd = static_cast<double*>(J.c[1]);
    double* gx = static_cast<double*>(J.c[2]);
    double* gxp = static_cast<double*>(J.c[3]);
    double* gy = static_cast<double*>(J.c[4]);
    double* gyp = static_cast<double*>(J.c[5]);
    const bool hx = gx != nullptr, hy = gy != nullptr;
    const bool vec = J.vec != 0;
    const int64_t base = (blockIdx.x - J.tile_begin) * static_cast<int64_t>(blockDim.x) * P +
                         static_cast<int64_t>(threadIdx.x) * P;
    double z[P], d[P], x[P], xp[P], y[P], yp[P];
    load2(gz, base, J.n, vec, z);
    load2(gd, base, J.n, vec, d);
#pragma unroll
    for (int p = 0; p < P; ++p) x[p] = xp[p] = y[p] = yp[p] = 0.0;
    if (hx) {
        load2(gx, base, J.n, vec, x);
        load2(gxp, base, J.n, vec, xp);
    }
    if (hy) {
        load2(gy, base, J.n, vec, y);
        load2(gyp, base, J.n, vec, yp);
    }
    const int64_t left = J.n - base;
    const float cnt = left >= P ? static_cast<float>(P) : (left > 0 ? static_cast<float>(left) : 0.0f);
    int parity = 0;
    if (mon && first) {
        if (hx || hy)
            record<true>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, J.mon, 0);
        else
            record<false>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, J.mon, 0);
        parity ^= 1;
    }
    if (GEN || mon) {
        if (J.scheme == PHTL_EULER_CROMER)
            run_f64<PHTL_EULER_CROMER, true, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if (J.scheme == PHTL_LEAPFROG)
            run_f64<PHTL_LEAPFROG, true, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if (!GEN || J.scheme == PHTL_RUTH4)
            run_f64<PHTL_RUTH4, true, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if constexpr (GEN)  // RK4 lives in the widened map's kernels only
            run_f64<PHTL_RK4, true, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
    } else {
        if (J.scheme == PHTL_EULER_CROMER)
            run_f64<PHTL_EULER_CROMER, false, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if (J.scheme == PHTL_LEAPFROG)
            run_f64<PHTL_LEAPFROG, false, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if (!GEN || J.scheme == PHTL_RUTH4)
            run_f64<PHTL_RUTH4, false, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if constexpr (GEN)  // RK4 lives in the widened map's kernels only
            run_f64<PHTL_RK4, false, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
    }
    store2(gz, base, J.n, vec, z);
    store2(gd, base, J.n, vec, d);
    if (hx) {
        store2(gx, base, J.n, vec, x);
        store2(gxp, base, J.n, vec, xp);
    }
    if (hy) {
        store2(gy, base, J.n, vec, y);
        store2(gyp, base, J.n, vec, yp);
    }
}

// ---------------------------------------------------------------------------------- FP32C
template <int SCHEME, int DT, bool MON, bool ZS, bool GEN>
__device__ __forceinline__ void run_f32c_zs(f32c::DF (&z)[f32c::P], f32c::DF (&d)[f32c::P],
                                            f32c::DF (&x)[f32c::P], f32c::DF (&xp)[f32c::P],
                                            f32c::DF (&y)[f32c::P], f32c::DF (&yp)[f32c::P],
                                            bool hx, bool hy, const MapConsts& c,
                                            const JobDesc& J, float cnt, int64_t t0, int nt,
                                            double* smem, int& parity)
{
    using namespace f32c;
    const int64_t g0 = t0 + J.turn_offset;  // turns done before this launch
    int64_t until = J.stride - (g0 % J.stride);
    int64_t row = g0 / J.stride + 1;
    float g1h[4], g1l[4], g2h[4], g2l[4];
    if (GEN) slip_stages<SCHEME>(c, g1h, g1l, g2h, g2l);
    for (int t = 0; t < nt; ++t) {
        if (GEN) {
            long_turn_nl<SCHEME, DT, ZS>(z, d, c, J.dc_hi, J.dc_lo, J.kw_hi, J.kw_lo, J.kw2_hi,
                                         J.kw2_lo, g1h, g1l, g2h, g2l, c.dual_rf != 0);
            transverse_gen<DT>(x, xp, y, yp, d, hx, hy, c);
        } else {
            long_turn<SCHEME, DT, ZS>(z, d, c, J.dc_hi, J.dc_lo, J.kw_hi, J.kw_lo);
            if (hx) {
#pragma unroll
                for (int p = 0; p < P; ++p) df_rotate(x[p], xp[p], c.mx_hi, c.mx_lo);
            }
            if (hy) {
#pragma unroll
                for (int p = 0; p < P; ++p) df_rotate(y[p], yp[p], c.my_hi, c.my_lo);
            }
        }
        if (MON && J.mon) {
            if (--until == 0) {
                // a longitudinal job reduces its 6 fields only (8 lanes' worth of butterfly)
                if (hx || hy)
                    record<true>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, J.mon, row);
                else
                    record<false>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, J.mon, row);
                parity ^= 1;
                ++row;
                until = J.stride;
            }
        }
    }
}

// phi_s == 0 chosen once, outside the turn loop
template <int SCHEME, int DT, bool MON, bool GEN>
__device__ __forceinline__ void run_f32c(f32c::DF (&z)[f32c::P], f32c::DF (&d)[f32c::P],
                                         f32c::DF (&x)[f32c::P], f32c::DF (&xp)[f32c::P],
                                         f32c::DF (&y)[f32c::P], f32c::DF (&yp)[f32c::P], bool hx,
                                         bool hy, const MapConsts& c, const JobDesc& J, float cnt,
                                         int64_t t0, int nt, double* smem, int& parity)
{
    if (c.phis_zero)
        run_f32c_zs<SCHEME, DT, MON, true, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
    else
        run_f32c_zs<SCHEME, DT, MON, false, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
}

template <int DT, bool MON, bool GEN>
__global__ void PHTL_F32C_BATCHED_BOUNDS(DT, GEN) k_batched_f32c(const JobDesc* __restrict__ jobs, int njobs,
                                                      MapConsts c, int64_t t0, int T)
{
    using namespace f32c;
    extern __shared__ double smem[];
    const JobDesc J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int64_t left_turns = J.turns - t0;
    const int nt = static_cast<int>(left_turns < T ? (left_turns > 0 ? left_turns : 0) : T);
    const bool mon = MON && J.mon != nullptr;
    const bool first = t0 + J.turn_offset == 0;
    if (nt == 0 && !(mon && first)) return;
    float* g[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = static_cast<float*>(J.c[i]);
    const bool hx = g[2] != nullptr, hy = g[4] != nullptr;
    const bool vec = J.vec != 0;
    const int64_t base = (blockIdx.x - J.tile_begin) * static_cast<int64_t>(blockDim.x) * P +
                         static_cast<int64_t>(threadIdx.x) * P;
    DF z[P], d[P], x[P], xp[P], y[P], yp[P];
    load4(g[0], base, J.n, vec, z);
    load4(g[1], base, J.n, vec, d);
#pragma unroll
    for (int p = 0; p < P; ++p) x[p] = xp[p] = y[p] = yp[p] = DF{0.0f, 0.0f};
    if (hx) {
        load4(g[2], base, J.n, vec, x);
        load4(g[3], base, J.n, vec, xp);
    }
    if (hy) {
        load4(g[4], base, J.n, vec, y);
        load4(g[5], base, J.n, vec, yp);
    }
    const int64_t left = J.n - base;
    const float cnt = left >= P ? static_cast<float>(P) : (left > 0 ? static_cast<float>(left) : 0.0f);
    int parity = 0;
    if (mon && first) {
        if (hx || hy)
            record<true>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, J.mon, 0);
        else
            record<false>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, J.mon, 0);
        parity ^= 1;
    }
    if (GEN || mon) {
        if (J.scheme == PHTL_EULER_CROMER)
            run_f32c<PHTL_EULER_CROMER, DT, true, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if (J.scheme == PHTL_LEAPFROG)
            run_f32c<PHTL_LEAPFROG, DT, true, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if (!GEN || J.scheme == PHTL_RUTH4)
            run_f32c<PHTL_RUTH4, DT, true, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if constexpr (GEN)  // RK4 lives in the widened map's kernels only
            run_f32c<PHTL_RK4, DT, true, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
    } else {
        if (J.scheme == PHTL_EULER_CROMER)
            run_f32c<PHTL_EULER_CROMER, DT, false, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if (J.scheme == PHTL_LEAPFROG)
            run_f32c<PHTL_LEAPFROG, DT, false, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if (!GEN || J.scheme == PHTL_RUTH4)
            run_f32c<PHTL_RUTH4, DT, false, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
        else if constexpr (GEN)  // RK4 lives in the widened map's kernels only
            run_f32c<PHTL_RK4, DT, false, GEN>(z, d, x, xp, y, yp, hx, hy, c, J, cnt, t0, nt, smem, parity);
    }
    store4(g[0], base, J.n, vec, z);
    store4(g[1], base, J.n, vec, d);
    if (hx) {
        store4(g[2], base, J.n, vec, x);
        store4(g[3], base, J.n, vec, xp);
    }
    if (hy) {
        store4(g[4], base, J.n, vec, y);
        store4(g[5], base, J.n, vec, yp);
    }
}

}  // namespace
}  // namespace phtl
