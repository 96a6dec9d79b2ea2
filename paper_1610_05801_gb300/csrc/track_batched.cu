// Batched launch of many independent bunches (the kernel templates and their design are
// in kernels_batched.cuh): selection, occupancy and launch.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_batched.cuh"

namespace phtl {
namespace {

const void* select_batched(int dtype, bool mon)
{
    if (dtype == PHTL_F64)
        return mon ? reinterpret_cast<const void*>(&k_batched_f64<true, false>)
                   : reinterpret_cast<const void*>(&k_batched_f64<false, false>);
    if (dtype == PHTL_F32C)
        return mon ? reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32C, true, false>)
                   : reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32C, false, false>);
    if (dtype == PHTL_F32CD)
        return mon ? reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32CD, true, false>)
                   : reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32CD, false, false>);
    if (dtype == PHTL_F32CS)
        return mon ? reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32CS, true, false>)
                   : reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32CS, false, false>);
    return nullptr;
}

}  // namespace

int particles_per_thread(int dtype) { return dtype == PHTL_F64 ? f64::P : f32c::P; }

int occupancy_batched(int dtype, bool mon, int block, bool general)
{
    const void* k = general ? general_kernel_batched(dtype) : select_batched(dtype, mon);
    if (!k) return 0;
    int nb = 0;
    const size_t smem = mon ? 2u * (block / 32) * 16 * sizeof(double) : 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_batched(const JobDesc* jobs, int32_t njobs, const MapConsts& c, int dtype,
                           bool mon, int64_t t0, int32_t T, int grid, int block, cudaStream_t s)
{
    const void* k = c.general ? general_kernel_batched(dtype) : select_batched(dtype, mon);
    if (!k) return cudaErrorInvalidValue;
    if (grid <= 0) return cudaSuccess;
    const size_t smem = mon ? 2u * (block / 32) * 16 * sizeof(double) : 0;
    const JobDesc* j = jobs;
    int nj = njobs;
    MapConsts cc = c;
    int64_t tt = t0;
    int TT = T;
    void* args[] = {&j, &nj, &cc, &tt, &TT};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, s);
}

}  // namespace phtl
