// FP64 tracking kernels of the linear map (the kernel template is in kernels_f64.cuh),
// their selection, occupancy and launch, and the sine diagnostics.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"
#include "kernels_f64.cuh"
#include "ops_f32c.cuh"
#include "ops_f64.cuh"

namespace phtl {
namespace {

using namespace f64;

template <int S, bool T, bool M>
const void* kernel_ptr()
{
    return reinterpret_cast<const void*>(&kf64::k_track_f64<S, T, M, false>);
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

int occupancy_f64(int scheme, bool trans, bool mon, int block, int gen)
{
    const void* k = gen ? general_kernel_single(scheme, PHTL_F64, gen == 2)
                        : select_kernel(scheme, trans, mon);
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
    const void* k = c.general ? general_kernel_single(L.scheme, PHTL_F64, c.dual_rf != 0)
                              : select_kernel(L.scheme, trans, mon);
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
