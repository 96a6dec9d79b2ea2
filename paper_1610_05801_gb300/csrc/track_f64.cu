// FP64 persistent multi-turn tracking kernel.
//
// Sec. 2.3 of the paper: particles are independent, turns are sequential, and the
// turn loop belongs inside the kernel so that each particle's state stays in
// registers between turns.  Here every thread owns P = 2 particles (one 128-bit load
// and store per coordinate per launch), runs `nturns` turns of the chosen scheme
// (Sec. 1.1.2) and the transverse matrix push (Sec. 1.1.1) on them, and adds the
// per-turn moment sums into the monitor rows.  Blocks walk over particle chunks in a
// grid-stride loop so the grid can be sized to the resident capacity of the GPU.  (Equal
// per-block shares were measured slower: the ragged warp at the end of every share costs
// more than the lone extra chunk some blocks run in the last round.)
//
// On GB300 the FP64 pipe retires 2 DFMA per clock per SM (1/64 of FP32), so this
// kernel is FP64-pipe bound: every FP64 operation per particle-turn counts.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"
#include "ops_f32c.cuh"
#include "ops_f64.cuh"

namespace phtl {
namespace {

using namespace f64;

// The turn loop of one particle chunk (state in registers throughout).
template <int SCHEME, bool TRANS, bool MON, bool ZS>
__device__ __forceinline__ void turns(double (&z)[P], double (&d)[P], double (&x)[P],
                                      double (&xp)[P], double (&y)[P], double (&yp)[P], bool hx,
                                      bool hy, float cnt, const MapConsts& c,
                                      const MonitorArgs& m, int nturns, double* smem, int& parity)
{
    int64_t until = m.until, row = m.row;
    for (int t = 0; t < nturns; ++t) {
        long_turn<SCHEME, ZS>(z, d, c, c.dc, c.kw);
        if (TRANS) {
            if (hx) rotate(x, xp, c.mx, c.shx, c.shear_x != 0);
            if (hy) rotate(y, yp, c.my, c.shy, c.shear_y != 0);
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
}

template <int SCHEME, bool TRANS, bool MON>
__global__ void __launch_bounds__(256, min_blocks_256<SCHEME>()) k_track_f64(LaunchDesc L, MapConsts c, MonitorArgs m)
{
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

        if (MON && m.initial) {
            record<TRANS>(z, d, x, xp, y, yp, cnt, hx, hy, smem, parity, m.rows, 0);
            parity ^= 1;
        }
        if (c.phis_zero)
            turns<SCHEME, TRANS, MON, true>(z, d, x, xp, y, yp, hx, hy, cnt, c, m, L.nturns,
                                            smem, parity);
        else
            turns<SCHEME, TRANS, MON, false>(z, d, x, xp, y, yp, hx, hy, cnt, c, m, L.nturns,
                                             smem, parity);
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

template <int S, bool T, bool M>
const void* kernel_ptr()
{
    return reinterpret_cast<const void*>(&k_track_f64<S, T, M>);
}

const void* select_kernel(int scheme, bool trans, bool mon)
{
#define PHTL_SEL(S)                                                              \
    if (scheme == S) {                                                           \
        if (trans) return mon ? kernel_ptr<S, true, true>() : kernel_ptr<S, true, false>(); \
        return mon ? kernel_ptr<S, false, true>() : kernel_ptr<S, false, false>();         \
    }
    PHTL_SEL(PHTL_EULER_CROMER)
    PHTL_SEL(PHTL_LEAPFROG)
    PHTL_SEL(PHTL_RUTH4)
#undef PHTL_SEL
    return nullptr;
}

}  // namespace

int occupancy_f64(int scheme, bool trans, bool mon, int block)
{
    const void* k = select_kernel(scheme, trans, mon);
    if (!k) return 0;
    int nb = 0;
    const size_t smem = mon ? 2u * (block / 32) * 16 * sizeof(double) : 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_track_f64(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                             cudaStream_t s)
{
    const bool trans = L.c[2] != nullptr || L.c[4] != nullptr;
    const bool mon = m.rows != nullptr;
    const void* k = select_kernel(L.scheme, trans, mon);
    if (!k) return cudaErrorInvalidValue;
    const size_t smem = mon ? 2u * (L.block / 32) * 16 * sizeof(double) : 0;
    LaunchDesc Lc = L;
    MapConsts cc = c;
    MonitorArgs mm = m;
    void* args[] = {&Lc, &cc, &mm};
    return cudaLaunchKernel(k, dim3(L.grid), dim3(L.block), args, smem, s);
}

namespace {

__global__ void k_eval_sin(const double* __restrict__ x, double* __restrict__ y, int64_t n,
                           int which)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    {
        if (which == 2) {
            const DF2 r = f32c::sin_df(split_bits(x[i]));
            y[i] = static_cast<double>(r.h) + static_cast<double>(r.l);
        } else {
            y[i] = which == 0 ? sin_f64(x[i]) : sin(x[i]);
        }
    }
}

__global__ void k_eval_sin_kz(double k, float k2opi, const double* __restrict__ z,
                              double* __restrict__ y, int64_t n)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        y[i] = sin_kz(k, k2opi, z[i]);
}

int eval_grid(int64_t n, int block)
{
    const int64_t want = (n + block - 1) / block;
    return static_cast<int>(want < 152 * 16 ? want : 152 * 16);
}

}  // namespace

}  // namespace phtl

extern "C" int phtl_eval_sin(const double* x, double* y, int64_t n, int which, void* stream)
{
    if (n < 0 || which < 0 || which > 2) return PHTL_E_INVALID;
    if (n > 0 && (!x || !y)) return PHTL_E_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PHTL_E_NODEVICE;
    }
    if (n == 0) return PHTL_OK;
    const int block = 256;
    phtl::k_eval_sin<<<phtl::eval_grid(n, block), block, 0, static_cast<cudaStream_t>(stream)>>>(
        x, y, n, which);
    if (cudaGetLastError() != cudaSuccess) return PHTL_E_CUDA;
    return PHTL_OK;
}

extern "C" int phtl_eval_sin_kz(double k, const double* z, double* y, int64_t n, void* stream)
{
    if (n < 0 || !std::isfinite(k)) return PHTL_E_INVALID;
    if (n > 0 && (!z || !y)) return PHTL_E_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PHTL_E_NODEVICE;
    }
    if (n == 0) return PHTL_OK;
    const int block = 256;
    const float k2opi = static_cast<float>(k * (2.0 / 3.14159265358979323846));
    phtl::k_eval_sin_kz<<<phtl::eval_grid(n, block), block, 0, static_cast<cudaStream_t>(stream)>>>(
        k, k2opi, z, y, n);
    if (cudaGetLastError() != cudaSuccess) return PHTL_E_CUDA;
    return PHTL_OK;
}
