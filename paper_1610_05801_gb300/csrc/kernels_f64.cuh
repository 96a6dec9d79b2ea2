// FP64 persistent multi-turn tracking kernel (template; instantiated by track_f64.cu for
// the linear map and by track_general.cu for the widened map).
//
// Sec. 2.3 of the paper: particles are independent, turns are sequential, and the
// turn loop belongs inside the kernel so that each particle's state stays in
// registers between turns.  Here every thread owns P = 2 particles (one 128-bit load
// and store per coordinate per launch), runs `nturns` turns of the chosen scheme
// (Sec. 1.1.2) and the transverse push (Sec. 1.1.1) on them, and adds the per-turn
// moment sums into the monitor rows.  Blocks walk over particle chunks in a grid-stride
// loop so the grid can be sized to the resident capacity of the GPU.  (Equal per-block
// shares were measured slower: the ragged warp at the end of every share costs more
// than the lone extra chunk some blocks run in the last round.)
//
// On GB300 the FP64 pipe retires 2 DFMA per clock per SM (1/64 of FP32), so this
// kernel is FP64-pipe bound: every FP64 operation per particle-turn counts.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "ops_f64.cuh"

namespace phtl {
namespace {
namespace kf64 {

using namespace f64;

// The turn loop of one particle chunk (state in registers throughout).  GEN: the widened
// map (slippage expansion, chromaticity, RK4), DUAL: with the second RF system; both
// chosen once per launch.
template <int SCHEME, bool TRANS, bool MON, bool ZS, bool GEN, bool DUAL>
__device__ __forceinline__ void turns(double (&z)[P], double (&d)[P], double (&x)[P],
                                      double (&xp)[P], double (&y)[P], double (&yp)[P], bool hx,
                                      bool hy, float cnt, const MapConsts& c,
                                      const MonitorArgs& m, int nturns, double* smem, int& parity)
{
    int64_t until = m.until, row = m.row;
    double g1[4], g2[4];
    if (GEN) slip_stages<SCHEME>(c, g1, g2);
    for (int t = 0; t < nturns; ++t) {
        if (GEN) {
            long_turn_nl<SCHEME, ZS>(z, d, c, c.dc, c.kw, c.kw2, g1, g2, DUAL);
            if (TRANS) transverse_gen(x, xp, y, yp, d, hx, hy, c);
        } else {
            long_turn<SCHEME, ZS>(z, d, c, c.dc, c.kw);
            if (TRANS) {
                if (hx) rotate(x, xp, c.mx, c.shx, c.shear_x != 0);
                if (hy) rotate(y, yp, c.my, c.shy, c.shear_y != 0);
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

// GEN: the widened map, chosen on the host (separate kernels, so the linear map's
// kernels keep their registers); DUAL (GEN only): with the second RF system, again a kernel
// of its own so that the rings without one keep theirs.  The GEN kernels are built with
// TRANS = MON = true and check the planes and the monitor at run time.
#ifdef PHTL_F64_RUTH4_MAXNREG
// build option: a register cap for the linear map's Ruth4 kernel instead of the blocks-per-SM
// bound (the other kernels keep the caps their bounds give: 80 for EC/LF, 128 for GEN)
#define PHTL_F64_BOUNDS(S, G) \
    __launch_bounds__(256) __maxnreg__((S) == PHTL_RUTH4 && !(G) ? PHTL_F64_RUTH4_MAXNREG : ((G) ? 128 : 80))
#else
#ifndef PHTL_F64_GEN_MIN_BLOCKS
#define PHTL_F64_GEN_MIN_BLOCKS 2
#endif
#define PHTL_F64_BOUNDS(S, G) __launch_bounds__(256, (G) ? PHTL_F64_GEN_MIN_BLOCKS : min_blocks_256<S>())
#endif
template <int SCHEME, bool TRANS, bool MON, bool GEN, bool DUAL = false>
__global__ void PHTL_F64_BOUNDS(SCHEME, GEN)
    k_track_f64(LaunchDesc L, MapConsts c, MonitorArgs m)
{
    if (L.go && *L.go == 0) return;  // the call was cancelled before this launch
    extern __shared__ double smem[];
    double* gz = static_cast<double*>(L.c[0]);
    double* gd = static_cast<double*>(L.c[1]);
    double* gx = static_cast<double*>(L.c[2]);
    double* gxp = static_cast<double*>(L.c[3]);
    double* gy = static_cast<double*>(L.c[4]);
    double* gyp = static_cast<double*>(L.c[5]);
    const bool hx = TRANS && gx != nullptr;
    const bool hy = TRANS && gy != nullptr;
    const bool vec = L.vec != 0;
    const int64_t chunk = static_cast<int64_t>(blockDim.x) * P;
    const int64_t nchunks = (L.n + chunk - 1) / chunk;
    int parity = 0;

    for (int64_t ci = blockIdx.x; ci < nchunks; ci += gridDim.x) {
        const int64_t base = ci * chunk + static_cast<int64_t>(threadIdx.x) * P;
        double z[P], d[P], x[P], xp[P], y[P], yp[P];
        load2(gz, base, L.n, vec, z);
        load2(gd, base, L.n, vec, d);
#pragma unroll
        for (int p = 0; p < P; ++p) x[p] = xp[p] = y[p] = yp[p] = 0.0;
        if (hx) {
            load2(gx, base, L.n, vec, x);
            load2(gxp, base, L.n, vec, xp);
        }
        if (hy) {
            load2(gy, base, L.n, vec, y);
            load2(gyp, base, L.n, vec, yp);
        }
        const int64_t left = L.n - base;
        const float cnt = left >= P ? static_cast<float>(P) : (left > 0 ? static_cast<float>(left) : 0.0f);

        if (MON && m.rows && m.initial) {
            record<TRANS>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, m.rows, 0);
            parity ^= 1;
        }
        if (c.phis_zero)
            turns<SCHEME, TRANS, MON, true, GEN, DUAL>(z, d, x, xp, y, yp, hx, hy, cnt, c, m,
                                                       L.nturns, smem, parity);
        else
            turns<SCHEME, TRANS, MON, false, GEN, DUAL>(z, d, x, xp, y, yp, hx, hy, cnt, c, m,
                                                        L.nturns, smem, parity);
        store2(gz, base, L.n, vec, z);
        store2(gd, base, L.n, vec, d);
        if (hx) {
            store2(gx, base, L.n, vec, x);
            store2(gxp, base, L.n, vec, xp);
        }
        if (hy) {
            store2(gy, base, L.n, vec, y);
            store2(gyp, base, L.n, vec, yp);
        }
    }
}

}  // namespace kf64
}  // namespace
}  // namespace phtl
