// Single-bunch kernels of the widened map with the second RF system for PHTL_F32CD and
// PHTL_F32CS (the FP64 and PHTL_F32C ones are in track_general_dual.cu).
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_f32c.cuh"

namespace phtl {
namespace {

template <int S>
const void* dual_s(int dtype)
{
    if (dtype == PHTL_F32CD)
        return reinterpret_cast<const void*>(&kf32::k_track_f32c<S, PHTL_F32CD, true, true, true, true>);
    if (dtype == PHTL_F32CS)
        return reinterpret_cast<const void*>(&kf32::k_track_f32c<S, PHTL_F32CS, true, true, true, true>);
    return nullptr;
}

}  // namespace

const void* general_kernel_single_dual_f32(int scheme, int dtype)
{
    if (scheme == PHTL_EULER_CROMER) return dual_s<PHTL_EULER_CROMER>(dtype);
    if (scheme == PHTL_LEAPFROG) return dual_s<PHTL_LEAPFROG>(dtype);
    if (scheme == PHTL_RUTH4) return dual_s<PHTL_RUTH4>(dtype);
    if (scheme == PHTL_RK4) return dual_s<PHTL_RK4>(dtype);
    return nullptr;
}

}  // namespace phtl
