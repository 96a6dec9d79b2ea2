// FP64 per-particle operations shared by the FP64 kernels (single bunch and batched).
//
// One thread owns P = 2 particles.  The stage order of each scheme follows the readings
// of Sec. 1.1.2 stated in phtl.h; the transverse push is the Sec. 1.1.1 matrix.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "monitor.cuh"
#include "sin_f64.cuh"

namespace phtl {
namespace f64 {

constexpr int P = 2;

__device__ __forceinline__ double rf_force(const MapConsts& c, double z)
{
    if (c.linear) return c.lin * z;
    return sin_f64(fma(c.k, z, c.phis)) - c.sinphis;
}

__device__ __forceinline__ void drift(double (&z)[P], const double (&d)[P], double dc)
{
#pragma unroll
    for (int p = 0; p < P; ++p) z[p] = fma(-dc, d[p], z[p]);
}

__device__ __forceinline__ void kick(const double (&z)[P], double (&d)[P], double kw,
                                     const MapConsts& c)
{
#pragma unroll
    for (int p = 0; p < P; ++p) d[p] = fma(kw, rf_force(c, z[p]), d[p]);
}

// One turn of the scheme; stage order as in Sec. 1.1.2's readings (see phtl.h).
// dc, kw: the drift and kick weights of this bunch's scheme (w_i eta C, w_j A); the
// single-bunch kernel passes c.dc, c.kw, the batched kernel the job table's copies.
template <int SCHEME>
__device__ __forceinline__ void long_turn(double (&z)[P], double (&d)[P], const MapConsts& c,
                                          const double* dc, const double* kw)
{
    if (SCHEME == PHTL_EULER_CROMER) {
        kick(z, d, kw[0], c);
        drift(z, d, dc[0]);
    } else if (SCHEME == PHTL_LEAPFROG) {
        drift(z, d, dc[0]);
        kick(z, d, kw[0], c);
        drift(z, d, dc[1]);
    } else {
        drift(z, d, dc[0]);
        kick(z, d, kw[0], c);
        drift(z, d, dc[1]);
        kick(z, d, kw[1], c);
        drift(z, d, dc[2]);
        kick(z, d, kw[2], c);
        drift(z, d, dc[3]);
    }
}

__device__ __forceinline__ void rotate(double (&u)[P], double (&v)[P], const double (&m)[4])
{
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const double un = fma(m[1], v[p], m[0] * u[p]);
        const double vn = fma(m[3], v[p], m[2] * u[p]);
        u[p] = un;
        v[p] = vn;
    }
}

__device__ __forceinline__ void pair_sums(const double (&a)[P], const double (&b)[P], double* f)
{
    f[0] = a[0];
    f[1] = b[0];
    f[2] = a[0] * a[0];
    f[3] = b[0] * b[0];
    f[4] = a[0] * b[0];
#pragma unroll
    for (int p = 1; p < P; ++p) {
        f[0] += a[p];
        f[1] += b[p];
        f[2] = fma(a[p], a[p], f[2]);
        f[3] = fma(b[p], b[p], f[3]);
        f[4] = fma(a[p], b[p], f[4]);
    }
}

template <bool TRANS>
__device__ __forceinline__ void record(const double (&z)[P], const double (&d)[P],
                                       const double (&x)[P], const double (&xp)[P],
                                       const double (&y)[P], const double (&yp)[P],
                                       double cnt, bool hx, bool hy, double* smem, int parity,
                                       double* rows, int64_t row)
{
    constexpr int NF = TRANS ? 16 : 8;
    double f[NF];
    f[0] = cnt;
    pair_sums(z, d, f + 1);
    if (TRANS) {
        if (hx) {
            pair_sums(x, xp, f + 6);
        } else {
#pragma unroll
            for (int j = 6; j < 11; ++j) f[j] = 0.0;
        }
        if (hy) {
            pair_sums(y, yp, f + 11);
        } else {
#pragma unroll
            for (int j = 11; j < 16; ++j) f[j] = 0.0;
        }
    } else {
        f[6] = 0.0;
        f[7] = 0.0;
    }
    block_record<NF>(f, smem, parity, rows, row, TRANS ? 16 : 6);
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
        const double2 t = __ldcs(reinterpret_cast<const double2*>(g + base));
        v[0] = t.x;
        v[1] = t.y;
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p) v[p] = (base + p < n) ? g[base + p] : 0.0;
    }
}

__device__ __forceinline__ void store2(double* __restrict__ g, int64_t base, int64_t n,
                                       bool vec, const double (&v)[P])
{
    if (vec && base + P <= n && aligned16(g + base)) {
        __stcs(reinterpret_cast<double2*>(g + base), make_double2(v[0], v[1]));
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (base + p < n) g[base + p] = v[p];
    }
}

}  // namespace f64
}  // namespace phtl
