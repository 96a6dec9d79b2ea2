// The collective step's turn kernel for the FP32-compensated arithmetic types (PHTL_F32C,
// PHTL_F32CD, PHTL_F32CS): the same steps as k_coll_turn (track_collective.cu) on
// float-pair state, P = 4 particles per thread.
//
//   - The previous turn's kick U_k (alpha V_k + alpha_sc D_k, formed in FP64 by
//     k_wake_potential and kept as a float pair) is added with TwoSum (PHTL_F32C/CD) or
//     as one float increment (PHTL_F32CS).
//   - The slice of a particle (decided once per turn, when counting, and kept per particle
//     for the next launch's kick): PHTL_F32C takes the same FP64 decision as the FP64 kernel on
//     hi + comp (exact in FP64); PHTL_F32CD and PHTL_F32CS form u = (z - z_lo) inv_dz in
//     double-float and take floor(u_hi + u_lo) exactly from the pair (u_hi integral with a
//     negative low part lies below u_hi).  Their decisions can differ from the FP64 oracle's
//     only for particles within ~1e-14 of a slice edge; a flipped particle changes one count
//     by one and its own kick by the difference of two neighbouring slices' U.
//   - The map and the transverse rotation: the widened map's double-float code (GEN), or the
//     linear map's where the ring has no widened term (bitwise the same there, fewer
//     operations).  The two variants are built in two translation units
//     (track_collective_f32.cu, track_collective_f32_lin.cu) that include this header.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "ops_f32c.cuh"

namespace phtl {
namespace collf32 {

using namespace f32c;

template <int DT>
__device__ __forceinline__ int slice_pair(const DF& z, const CollArgs& A, int ns_hi)
{
    if (DT == PHTL_F32C) {
        const double zd = widen_bits(z.hi) + widen_bits(z.c);
        const double u = __dmul_rn(__dsub_rn(zd, A.z_lo), A.inv_dz);
        const int hi = __double2hiint(u);
        if (hi < 0) return ((hi << 1) | __double2loint(u)) == 0 ? 0 : -1;  // -0.0, or u < 0
        if (hi >= ns_hi) return -1;
        return floor_small(hi);
    }
    const DF2 t = df_add(as2(z), DF2{-A.z_lo_h, -A.z_lo_l});
    const DF2 u = df_mul(t, DF2{A.inv_dz_h, A.inv_dz_l});
    if (!(u.h >= 0.0f && u.h <= static_cast<float>(A.nslices))) return -1;  // NaN fails too
    const float fh = floorf(u.h);
    int k = static_cast<int>(fh);
    if (fh == u.h && u.l < 0.0f) --k;
    return (k >= 0 && k < A.nslices) ? k : -1;
}

// Register cap of the turn kernel.  Unlike the persistent FP32 kernels (issue-bound, state in
// registers), it loads its state every turn and waits on memory, so more resident warps pay:
// 96 registers (20 warps per SM at 128-thread blocks, a few bytes of spills in some variants)
// ran 7-18 % faster than the uncapped 115-126 (16 warps) on GB300, 104 about 2 %, and 88 or
// fewer spilled more.  Build option PHTL_COLL_F32_MAXNREG overrides it.  (Blocks are at most
// 256 threads; __maxnreg__ and __launch_bounds__ do not combine.)
#ifndef PHTL_COLL_F32_MAXNREG
#define PHTL_COLL_F32_MAXNREG 96
#endif
#define PHTL_COLL_F32_BOUNDS __maxnreg__(PHTL_COLL_F32_MAXNREG)

template <int S, int DT, bool GEN>
__global__ void PHTL_COLL_F32_BOUNDS
    k_coll_turn_f32(LaunchDesc L, MapConsts c, CollArgs A, const float2* __restrict__ U2,
                    unsigned* __restrict__ counts, uint16_t* __restrict__ slot,
                    double* __restrict__ mon_rows, int64_t rec_row, int kick, int map)
{
    extern __shared__ double smem_d[];
    unsigned* hist = reinterpret_cast<unsigned*>(smem_d);
    double* msm = smem_d + (A.nslices + 1) / 2;  // 8-byte aligned after the bins
    float* g[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = static_cast<float*>(L.c[i]);
    const bool hx = g[2] != nullptr, hy = g[4] != nullptr;
    const bool vec = L.vec != 0;
    if (counts)
        for (int k = threadIdx.x; k < A.nslices; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    griddep_wait();  // the previous turn's state, kick and cleared counts
    const int64_t chunk = static_cast<int64_t>(blockDim.x) * P;
    const int64_t nchunks = (L.n + chunk - 1) / chunk;
    int parity = 0;
    float g1h[4], g1l[4], g2h[4], g2l[4];
    if (GEN) slip_stages<S>(c, g1h, g1l, g2h, g2l);
    const int ns_hi = __double2hiint(static_cast<double>(A.nslices));
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
        if (kick) {
            int k[P];
            slots_load<P>(slot, base, L.n, k);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (k[p] != static_cast<int>(kSlotOutside)) {
                    const float2 u = __ldg(U2 + k[p]);
                    if (DT == PHTL_F32CS) acc(d[p], u.x);
                    else acc2(d[p], DF2{u.x, u.y});
                }
            }
        }
        if (mon_rows && rec_row >= 0) {
            record<true>(z, d, x, xp, y, yp, cnt, hx, hy, msm, parity, mon_rows, rec_row);
            parity ^= 1;
        }
        if (map) {
            if constexpr (GEN) {
                if (c.phis_zero)
                    long_turn_nl<S, DT, true>(z, d, c, c.dc_hi, c.dc_lo, c.kw_hi, c.kw_lo, c.kw2_hi,
                                              c.kw2_lo, g1h, g1l, g2h, g2l, c.dual_rf != 0);
                else
                    long_turn_nl<S, DT, false>(z, d, c, c.dc_hi, c.dc_lo, c.kw_hi, c.kw_lo, c.kw2_hi,
                                               c.kw2_lo, g1h, g1l, g2h, g2l, c.dual_rf != 0);
                transverse_gen<DT>(x, xp, y, yp, d, hx, hy, c);
            } else {
                if (c.phis_zero) long_turn<S, DT, true>(z, d, c, c.dc_hi, c.dc_lo, c.kw_hi, c.kw_lo);
                else long_turn<S, DT, false>(z, d, c, c.dc_hi, c.dc_lo, c.kw_hi, c.kw_lo);
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
        if (counts) {
            int k[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                k[p] = base + p < L.n ? slice_pair<DT>(z[p], A, ns_hi) : -1;
                if (k[p] >= 0) atomicAdd(hist + k[p], 1u);
            }
            slots_store<P>(slot, base, L.n, k);
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
    // the potential kernel may launch now (it waits for this grid's completion); not earlier,
    // so that its blocks do not sit on SM slots while this grid still works
    griddep_launch_dependents();
    if (counts) {
        __syncthreads();
        for (int k = threadIdx.x; k < A.nslices; k += blockDim.x) {
            const unsigned h = hist[k];
            if (h) atomicAdd(counts + k, h);
        }
    }
}

}  // namespace collf32
}  // namespace phtl
