// FP32-compensated tracking kernels of the linear map (the kernel template is in
// kernels_f32c.cuh): selection, occupancy and launch.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_f32c.cuh"
#include "ops_f32c.cuh"

namespace phtl {
namespace {

using namespace f32c;

template <int S, int D, bool T, bool M>
const void* kptr()
{
    return reinterpret_cast<const void*>(&kf32::k_track_f32c<S, D, T, M, false>);
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
    if (dtype == PHTL_F32CS) return sel_tm<S, PHTL_F32CS>(trans, mon);
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

int occupancy_f32c(int scheme, bool trans, bool mon, int dtype, int block, int gen)
{
    const void* k = gen ? general_kernel_single(scheme, dtype, gen == 2)
                        : select_kernel(scheme, dtype, trans, mon);
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
    const void* k = c.general ? general_kernel_single(L.scheme, dtype, c.dual_rf != 0)
                              : select_kernel(L.scheme, dtype, trans, mon);
    if (!k) return cudaErrorInvalidValue;
    const size_t smem = mon ? 2u * (L.block / 32) * 16 * sizeof(double) : 0;
    LaunchDesc Lc = L;
    MapConsts cc = c;
    MonitorArgs mm = m;
    void* args[] = {&Lc, &cc, &mm};
    return cudaLaunchKernel(k, dim3(L.grid), dim3(L.block), args, smem, s);
}

}  // namespace phtl
