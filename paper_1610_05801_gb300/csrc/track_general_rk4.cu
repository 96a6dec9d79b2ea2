// Single-bunch kernels of the classic RK4 integrator (four force evaluations per turn),
// which only the widened map's kernel templates hold; a translation unit of its own so
// that it builds in parallel with the other widened-map kernels.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_f32c.cuh"
#include "kernels_f64.cuh"

namespace phtl {

const void* general_kernel_single_rk4(int dtype)
{
    if (dtype == PHTL_F64) return reinterpret_cast<const void*>(&kf64::k_track_f64<PHTL_RK4, true, true, true>);
    if (dtype == PHTL_F32C)
        return reinterpret_cast<const void*>(&kf32::k_track_f32c<PHTL_RK4, PHTL_F32C, true, true, true>);
    if (dtype == PHTL_F32CD)
        return reinterpret_cast<const void*>(&kf32::k_track_f32c<PHTL_RK4, PHTL_F32CD, true, true, true>);
    if (dtype == PHTL_F32CS)
        return reinterpret_cast<const void*>(&kf32::k_track_f32c<PHTL_RK4, PHTL_F32CS, true, true, true>);
    return nullptr;
}

}  // namespace phtl
