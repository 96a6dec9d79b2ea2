// FP64 per-particle operations shared by the FP64 kernels (single bunch and batched).
//
// One thread owns P = 2 particles.  The stage order of each scheme follows the readings
// of Sec. 1.1.2 stated in phtl.h; the transverse push is the Sec. 1.1.1 matrix.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "monitor.cuh"
#include "dfloat.cuh"
#include "sin_f64.cuh"

namespace phtl {
namespace f64 {

// Particles per thread: independent FP64 dependency chains per thread (even).
#ifndef PHTL_F64_PARTICLES_PER_THREAD
#define PHTL_F64_PARTICLES_PER_THREAD 2
#endif
constexpr int P = PHTL_F64_PARTICLES_PER_THREAD;
static_assert(P % 2 == 0, "P must be even (128-bit loads of two doubles)");

// Minimum resident 256-thread blocks per SM asked of the compiler (caps registers at
// 65536 / (256 * this)): the FP64 kernels hide the FP64 pipe's latency with warps.
// Euler-Cromer and leap-frog run faster with 3 (80 registers, 24 warps per SM); Ruth4,
// with three kicks per turn in flight, with 2 (measured on GB300).
#ifndef PHTL_F64_MIN_BLOCKS_256
#define PHTL_F64_MIN_BLOCKS_256 3
#endif
#ifndef PHTL_F64_MIN_BLOCKS_256_RUTH4
#define PHTL_F64_MIN_BLOCKS_256_RUTH4 2
#endif
// The batched kernel holds all three schemes; at 3 it would spill.
constexpr int kBatchedMinBlocks256 = 2;
template <int SCHEME>
constexpr int min_blocks_256()
{
    return SCHEME == PHTL_RUTH4 ? PHTL_F64_MIN_BLOCKS_256_RUTH4 : PHTL_F64_MIN_BLOCKS_256;
}

// ZS: phi_s == 0 (stationary bucket): the force is sin(k z), with the phase product fused
// into the sine's reduction and no subtraction (the kernels choose the instantiation
// once, outside the turn loop).
template <bool ZS>
__device__ __forceinline__ double rf_force(const MapConsts& c, double z)
{
    if (c.linear) return c.lin * z;
    if (ZS) return sin_kz(c.k, c.k2opi, z);
    return sin_f64(fma(c.k, z, c.phis)) - c.sinphis;
}

__device__ __forceinline__ void drift(double (&z)[P], const double (&d)[P], double dc)
{
#pragma unroll
    for (int p = 0; p < P; ++p) z[p] = fma(-dc, d[p], z[p]);
}

template <bool ZS>
__device__ __forceinline__ void kick(const double (&z)[P], double (&d)[P], double kw,
                                     const MapConsts& c)
{
#pragma unroll
    for (int p = 0; p < P; ++p) d[p] = fma(kw, rf_force<ZS>(c, z[p]), d[p]);
}

// One turn of the scheme; stage order as in Sec. 1.1.2's readings (see phtl.h).
// dc, kw: the drift and kick weights of this bunch's scheme (w_i eta C, w_j A); the
// single-bunch kernel passes c.dc, c.kw, the batched kernel the job table's copies.
template <int SCHEME, bool ZS>
__device__ __forceinline__ void long_turn(double (&z)[P], double (&d)[P], const MapConsts& c,
                                          const double* dc, const double* kw)
{
    if (SCHEME == PHTL_EULER_CROMER) {
        kick<ZS>(z, d, kw[0], c);
        drift(z, d, dc[0]);
    } else if (SCHEME == PHTL_LEAPFROG) {
        drift(z, d, dc[0]);
        kick<ZS>(z, d, kw[0], c);
        drift(z, d, dc[1]);
    } else {
        drift(z, d, dc[0]);
        kick<ZS>(z, d, kw[0], c);
        drift(z, d, dc[1]);
        kick<ZS>(z, d, kw[1], c);
        drift(z, d, dc[2]);
        kick<ZS>(z, d, kw[2], c);
        drift(z, d, dc[3]);
    }
}

// Transverse push of one plane (Sec. 1.1.1 matrix).  With use_shear the rotation is
// applied as three shears (3 DFMA instead of 2 DMUL + 2 DFMA); the same map up to rounding.
__device__ __forceinline__ void rotate(double (&u)[P], double (&v)[P], const double (&m)[4],
                                       const double (&sh)[2], bool use_shear)
{
    if (use_shear) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
            u[p] = fma(sh[0], v[p], u[p]);
            v[p] = fma(sh[1], u[p], v[p]);
            u[p] = fma(sh[0], v[p], u[p]);
        }
        return;
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double un = fma(m[1], v[p], m[0] * u[p]);
        const double vn = fma(m[3], v[p], m[2] * u[p]);
        u[p] = un;
        v[p] = vn;
    }
}

// ---- widened map: nonlinear slippage and chromaticity -------------------------------

// Drift with the slippage expansion: z -= (dc + g1 d + g2 d^2) d for this stage's
// w eta(d) C, i.e. dc = w eta0 C, g1 = w eta1 C, g2 = w eta2 C.  With g1 = g2 = 0 it
// is bitwise the linear drift.
__device__ __forceinline__ void drift_nl(double (&z)[P], const double (&d)[P], double dc,
                                         double g1, double g2)
{
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double e = fma(fma(g2, d[p], g1), d[p], dc);
        z[p] = fma(-e, d[p], z[p]);
    }
}

// Force of the second RF system (double RF) per unit weight: sin(phi2 + k2 z) - sin(phi2),
// or cos(phi2) k2 z in rf_linear mode.
__device__ __forceinline__ double rf_force2(const MapConsts& c, double z)
{
    if (c.linear) return c.lin2 * z;
    return sin_f64(fma(c.k2, z, c.phi2)) - c.sinphi2;
}

// Kick of the widened map: the main RF system, then the second one when `dual` (a
// compile-time constant in the single-bunch kernels, which have a variant without the
// second system; the batched kernels pass the ring's flag) -- kw2: this stage's w_j A2.
template <bool ZS>
__device__ __forceinline__ void kick_gen(const double (&z)[P], double (&d)[P], double kw, double kw2,
                                         const MapConsts& c, bool dual)
{
#pragma unroll
    for (int p = 0; p < P; ++p) {
        d[p] = fma(kw, rf_force<ZS>(c, z[p]), d[p]);
        if (dual) d[p] = fma(kw2, rf_force2(c, z[p]), d[p]);
    }
}

// Right-hand side of the smooth motion per turn (classic RK4's derivative):
// dz/dn = -eta(d) C d = -(dc + g1 d + g2 d^2) d and dd/dn = kw F1(z) + kw2 F2(z), with
// dc = eta0 C, g1 = eta1 C, g2 = eta2 C, kw = A, kw2 = A2.
template <bool ZS>
__device__ __forceinline__ void rk4_rhs(double z, double d, const MapConsts& c, double dc, double g1,
                                        double g2, double kw, double kw2, bool dual, double& fz,
                                        double& fd)
{
    // the products are rounded on their own (__dmul_rn): the stage arguments and the
    // weighted sum reuse them, and an FMA contraction chosen differently where `dual` is a
    // compile-time constant than where it is not would break the bitwise agreement of the
    // single-bunch and batched kernels
    const double e = fma(fma(g2, d, g1), d, dc);
    fz = -__dmul_rn(e, d);
    fd = __dmul_rn(kw, rf_force<ZS>(c, z));
    if (dual) fd = fma(kw2, rf_force2(c, z), fd);
}

// One classic RK4 step of one turn: k1 at the start, k2 and k3 at the half step from k1
// and k2, k4 at the full step from k3, and the weighted sum (k1 + 2 k2 + 2 k3 + k4) / 6.
template <bool ZS>
__device__ __forceinline__ void rk4_turn(double (&z)[P], double (&d)[P], const MapConsts& c,
                                         double dc, double kw, double kw2, double g1, double g2,
                                         bool dual)
{
    constexpr double kSixth = 1.0 / 6.0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        double k1z, k1d, k2z, k2d, k3z, k3d, k4z, k4d;
        rk4_rhs<ZS>(z[p], d[p], c, dc, g1, g2, kw, kw2, dual, k1z, k1d);
        rk4_rhs<ZS>(fma(0.5, k1z, z[p]), fma(0.5, k1d, d[p]), c, dc, g1, g2, kw, kw2, dual, k2z, k2d);
        rk4_rhs<ZS>(fma(0.5, k2z, z[p]), fma(0.5, k2d, d[p]), c, dc, g1, g2, kw, kw2, dual, k3z, k3d);
        rk4_rhs<ZS>(__dadd_rn(z[p], k3z), __dadd_rn(d[p], k3d), c, dc, g1, g2, kw, kw2, dual, k4z, k4d);
        z[p] = fma(fma(2.0, __dadd_rn(k2z, k3z), __dadd_rn(k1z, k4z)), kSixth, z[p]);
        d[p] = fma(fma(2.0, __dadd_rn(k2d, k3d), __dadd_rn(k1d, k4d)), kSixth, d[p]);
    }
}

// One turn of the scheme with the slippage expansion (g1[i], g2[i]: stage i's w_i eta1 C,
// w_i eta2 C) and the second RF system (kw2[j]: stage j's w_j A2).
template <int SCHEME, bool ZS>
__device__ __forceinline__ void long_turn_nl(double (&z)[P], double (&d)[P], const MapConsts& c,
                                             const double* dc, const double* kw, const double* kw2,
                                             const double (&g1)[4], const double (&g2)[4], bool dual)
{
    if (SCHEME == PHTL_RK4) {
        rk4_turn<ZS>(z, d, c, dc[0], kw[0], kw2[0], g1[0], g2[0], dual);
    } else if (SCHEME == PHTL_EULER_CROMER) {
        kick_gen<ZS>(z, d, kw[0], kw2[0], c, dual);
        drift_nl(z, d, dc[0], g1[0], g2[0]);
    } else if (SCHEME == PHTL_LEAPFROG) {
        drift_nl(z, d, dc[0], g1[0], g2[0]);
        kick_gen<ZS>(z, d, kw[0], kw2[0], c, dual);
        drift_nl(z, d, dc[1], g1[1], g2[1]);
    } else {
        drift_nl(z, d, dc[0], g1[0], g2[0]);
        kick_gen<ZS>(z, d, kw[0], kw2[0], c, dual);
        drift_nl(z, d, dc[1], g1[1], g2[1]);
        kick_gen<ZS>(z, d, kw[1], kw2[1], c, dual);
        drift_nl(z, d, dc[2], g1[2], g2[2]);
        kick_gen<ZS>(z, d, kw[2], kw2[2], c, dual);
        drift_nl(z, d, dc[3], g1[3], g2[3]);
    }
}

// Stage constants g1, g2 of the slippage expansion for this scheme (loop-invariant).
template <int SCHEME>
__device__ __forceinline__ void slip_stages(const MapConsts& c, double (&g1)[4], double (&g2)[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        g1[i] = drift_weight(SCHEME, i) * c.eta1C;
        g2[i] = drift_weight(SCHEME, i) * c.eta2C;
    }
}

// Chromatic rotation of one plane: each particle turns by 2 pi (q + xi d) with its own d
// (after the turn's longitudinal step).
__device__ __forceinline__ void rotate_chroma(double (&u)[P], double (&v)[P], const double (&d)[P],
                                              double q, double xi, double b, double ib)
{
#pragma unroll
    for (int p = 0; p < P; ++p) {
        double sn, cs;
        sincos_turns(fma(xi, d[p], q), sn, cs);
        const double un = fma(b * sn, v[p], cs * u[p]);
        const double vn = fma(-(sn * ib), u[p], cs * v[p]);
        u[p] = un;
        v[p] = vn;
    }
}

// The transverse step of the general loop: chromatic where xi != 0, else the one matrix.
__device__ __forceinline__ void transverse_gen(double (&x)[P], double (&xp)[P], double (&y)[P],
                                               double (&yp)[P], const double (&d)[P], bool hx,
                                               bool hy, const MapConsts& c)
{
    if (hx) {
        if (c.chroma_x) rotate_chroma(x, xp, d, c.qx, c.xi_x, c.bx, c.ibx);
        else rotate(x, xp, c.mx, c.shx, c.shear_x != 0);
    }
    if (hy) {
        if (c.chroma_y) rotate_chroma(y, yp, d, c.qy, c.xi_y, c.by, c.iby);
        else rotate(y, yp, c.my, c.shy, c.shear_y != 0);
    }
}

// Per-thread moment contributions of one plane (a, b): sum a, sum b, sum a^2, sum b^2,
// sum ab over this thread's P particles, as double-float pairs.  The doubles are split
// into float pairs with integer operations and the products formed with the exact FP32
// product error, so the sums keep ~47 bits without using the FP64 pipe.
__device__ __forceinline__ void pair_sums_df(const double (&a)[P], const double (&b)[P], DF2* f)
{
    DF2 ap = split_bits(a[0]), bp = split_bits(b[0]);
    f[0] = ap;
    f[1] = bp;
    f[2] = df_mul(ap, ap);
    f[3] = df_mul(bp, bp);
    f[4] = df_mul(ap, bp);
#pragma unroll
    for (int p = 1; p < P; ++p) {
        ap = split_bits(a[p]);
        bp = split_bits(b[p]);
        f[0] = df_add(f[0], ap);
        f[1] = df_add(f[1], bp);
        f[2] = df_add(f[2], df_mul(ap, ap));
        f[3] = df_add(f[3], df_mul(bp, bp));
        f[4] = df_add(f[4], df_mul(ap, bp));
    }
}

// Add this block's moment sums of the current turn into monitor row `row`.
// smem: 2 * (blockDim.x / 32) * 16 DF2.
template <bool TRANS>
__device__ __forceinline__ void record(const double (&z)[P], const double (&d)[P],
                                       const double (&x)[P], const double (&xp)[P],
                                       const double (&y)[P], const double (&yp)[P],
                                       float cnt, bool hx, bool hy, double* smem, int parity,
                                       double* rows, int64_t row)
{
    constexpr int NF = TRANS ? 16 : 8;
    const DF2 zero{0.0f, 0.0f};
    DF2 f[NF];
    f[0] = DF2{cnt, 0.0f};  // 0..P: exact
    pair_sums_df(z, d, f + 1);
    if constexpr (TRANS) {
        if (hx) {
            pair_sums_df(x, xp, f + 6);
        } else {
#pragma unroll
            for (int j = 6; j < 11; ++j) f[j] = zero;
        }
        if (hy) {
            pair_sums_df(y, yp, f + 11);
        } else {
#pragma unroll
            for (int j = 11; j < 16; ++j) f[j] = zero;
        }
    } else {
        f[6] = zero;
        f[7] = zero;
    }
    block_record_df<NF>(f, reinterpret_cast<DF2*>(smem), parity, rows, row, TRANS ? 16 : 6);
}

// 128-bit accesses only where the host allowed them (vec) AND the address really is
// 16-byte aligned; anything else takes the scalar path.
__device__ __forceinline__ bool aligned16(const void* p)
{
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

__device__ __forceinline__ void load2(const double* __restrict__ g, int64_t base, int64_t n,
                                      bool vec, double (&v)[P])
{
    if (vec && base + P <= n && aligned16(g + base)) {
#pragma unroll
        for (int k = 0; k < P; k += 2) {
            const double2 t = __ldcs(reinterpret_cast<const double2*>(g + base + k));
            v[k] = t.x;
            v[k + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p) v[p] = (base + p < n) ? g[base + p] : 0.0;
    }
}

__device__ __forceinline__ void store2(double* __restrict__ g, int64_t base, int64_t n,
                                       bool vec, const double (&v)[P])
{
    if (vec && base + P <= n && aligned16(g + base)) {
#pragma unroll
        for (int k = 0; k < P; k += 2)
            __stcs(reinterpret_cast<double2*>(g + base + k), make_double2(v[k], v[k + 1]));
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (base + p < n) g[base + p] = v[p];
    }
}

}  // namespace f64
}  // namespace phtl
