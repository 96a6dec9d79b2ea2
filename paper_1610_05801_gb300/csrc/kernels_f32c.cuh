// FP32-compensated persistent multi-turn tracking kernel (PHTL_F32C, PHTL_F32CD,
// PHTL_F32CS); template, instantiated by track_f32c.cu for the linear map and by
// track_general.cu for the widened map.
//
// Same structure as the FP64 kernel (Sec. 2.3: turn loop inside the kernel, state in
// registers), but every coordinate is an unevaluated sum hi + comp of two floats:
//   - PHTL_F32C / PHTL_F32CD: each drift/kick increment is a double-float product of the
//     FP64 weight (split into hi + lo) and the pair, added with Knuth's TwoSum and
//     renormalised with Fast2Sum; the RF phase argument is formed from hi + comp in FP64
//     (PHTL_F32C) or in double-float arithmetic (PHTL_F32CD), and the sine is the
//     double-float polynomial sin_df (~1e-12 absolute);
//   - PHTL_F32CS: FP32 increments with split weights, the phase rounded to FP32 and the
//     SFU's __sinf;
//   - the transverse matrix (Sec. 1.1.1) is applied in double-float arithmetic (exact
//     FP32 products by fmaf, TwoSum of the two terms), so the rotation keeps ~48 bits;
//   - per-turn moment sums are FP32 per thread and across the warp (<= 128 particles),
//     then FP64 across warps and blocks.
// Each thread owns P = 4 particles (one 128-bit load of hi and one of comp per
// coordinate).  This kernel is FP32-pipe / issue bound; the FP64 variant of the phase
// argument adds a handful of FP64-pipe operations per kick.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "ops_f32c.cuh"

namespace phtl {
namespace {
namespace kf32 {

using namespace f32c;

// The turn loop of one particle chunk (state in registers throughout); ZS: phi_s == 0;
// GEN: the widened map (slippage expansion, chromaticity), chosen once per launch.
template <int SCHEME, int DT, bool TRANS, bool MON, bool ZS, bool GEN, bool DUAL>
__device__ __forceinline__ void turns(DF (&z)[P], DF (&d)[P], DF (&x)[P], DF (&xp)[P],
                                      DF (&y)[P], DF (&yp)[P], bool hx, bool hy, float cnt,
                                      const MapConsts& c, const MonitorArgs& m, int nturns,
                                      double* smem, int& parity)
{
    int64_t until = m.until, row = m.row;
    float g1h[4], g1l[4], g2h[4], g2l[4];
    if (GEN) slip_stages<SCHEME>(c, g1h, g1l, g2h, g2l);
    for (int t = 0; t < nturns; ++t) {
        if (GEN) {
            long_turn_nl<SCHEME, DT, ZS>(z, d, c, c.dc_hi, c.dc_lo, c.kw_hi, c.kw_lo, c.kw2_hi,
                                         c.kw2_lo, g1h, g1l, g2h, g2l, DUAL);
            if (TRANS) transverse_gen<DT>(x, xp, y, yp, d, hx, hy, c);
        } else {
            long_turn<SCHEME, DT, ZS>(z, d, c, c.dc_hi, c.dc_lo, c.kw_hi, c.kw_lo);
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
        }
        if (MON && m.rows) {
            if (--until == 0) {
                record<TRANS>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, m.rows, row);
                parity ^= 1;
                ++row;
                until = m.stride;
            }
        }
    }
}

// GEN: the widened map, chosen on the host (separate kernels, built with TRANS = MON =
// true; planes and monitor are checked at run time); DUAL (GEN only): with the second RF
// system.
template <int SCHEME, int DT, bool TRANS, bool MON, bool GEN, bool DUAL = false>
__global__ void PHTL_F32C_TRACK_BOUNDS(SCHEME, DT, GEN) k_track_f32c(LaunchDesc L, MapConsts c, MonitorArgs m)
{
    if (L.go && *L.go == 0) return;  // the call was cancelled before this launch
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

        if (MON && m.rows && m.initial) {
            record<TRANS>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, m.rows, 0);
            parity ^= 1;
        }
        if (c.phis_zero)
            turns<SCHEME, DT, TRANS, MON, true, GEN, DUAL>(z, d, x, xp, y, yp, hx, hy, cnt, c, m,
                                                           L.nturns, smem, parity);
        else
            turns<SCHEME, DT, TRANS, MON, false, GEN, DUAL>(z, d, x, xp, y, yp, hx, hy, cnt, c, m,
                                                            L.nturns, smem, parity);
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

}  // namespace kf32
}  // namespace
}  // namespace phtl
