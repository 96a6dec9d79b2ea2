// Single-bunch kernels of the widened map with the second RF system (double RF): the
// widened map's kernel templates with DUAL = true, kept apart so that rings without a
// second system run kernels without its code (fewer registers).  FP64 and PHTL_F32C here,
// PHTL_F32CD and PHTL_F32CS in track_general_dual_f32.cu (they build in parallel).
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_f32c.cuh"
#include "kernels_f64.cuh"

namespace phtl {
namespace {

template <int S>
const void* dual_s(int dtype)
{
    if (dtype == PHTL_F64) return reinterpret_cast<const void*>(&kf64::k_track_f64<S, true, true, true, true>);
    if (dtype == PHTL_F32C)
        return reinterpret_cast<const void*>(&kf32::k_track_f32c<S, PHTL_F32C, true, true, true, true>);
    return nullptr;
}

}  // namespace

const void* general_kernel_single_dual(int scheme, int dtype)
{
    if (dtype == PHTL_F32CD || dtype == PHTL_F32CS) return general_kernel_single_dual_f32(scheme, dtype);
    if (scheme == PHTL_EULER_CROMER) return dual_s<PHTL_EULER_CROMER>(dtype);
    if (scheme == PHTL_LEAPFROG) return dual_s<PHTL_LEAPFROG>(dtype);
    if (scheme == PHTL_RUTH4) return dual_s<PHTL_RUTH4>(dtype);
    if (scheme == PHTL_RK4) return dual_s<PHTL_RK4>(dtype);
    return nullptr;
}

}  // namespace phtl
