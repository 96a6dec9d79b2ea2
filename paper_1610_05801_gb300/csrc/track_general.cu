// Single-bunch kernels of the widened map: the slippage expansion eta(delta) in the drift,
// the chromatic transverse rotation (per-particle phase advance 2 pi (frac Q + xi
// delta)), the second RF system and the classic RK4 integrator.  The same kernel templates as the linear map (kernels_f64.cuh,
// kernels_f32c.cuh) with GEN = true, in a translation unit of their own so that neither
// the linear kernels' registers nor their build time change.  Built with TRANS = MON =
// true: the planes and the monitor are checked at run time.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_f32c.cuh"
#include "kernels_f64.cuh"

namespace phtl {

const void* general_kernel_single(int scheme, int dtype, bool dual)
{
    if (dual) return general_kernel_single_dual(scheme, dtype);
#define PHTL_GEN(S)                                                                          \
    if (scheme == S) {                                                                       \
        if (dtype == PHTL_F64) return reinterpret_cast<const void*>(&kf64::k_track_f64<S, true, true, true>); \
        if (dtype == PHTL_F32C)                                                              \
            return reinterpret_cast<const void*>(&kf32::k_track_f32c<S, PHTL_F32C, true, true, true>); \
        if (dtype == PHTL_F32CD)                                                             \
            return reinterpret_cast<const void*>(&kf32::k_track_f32c<S, PHTL_F32CD, true, true, true>); \
        if (dtype == PHTL_F32CS)                                                             \
            return reinterpret_cast<const void*>(&kf32::k_track_f32c<S, PHTL_F32CS, true, true, true>); \
        return nullptr;                                                                      \
    }
    PHTL_GEN(PHTL_EULER_CROMER)
    PHTL_GEN(PHTL_LEAPFROG)
    PHTL_GEN(PHTL_RUTH4)
#undef PHTL_GEN
    if (scheme == PHTL_RK4) return general_kernel_single_rk4(dtype);
    return nullptr;
}

}  // namespace phtl
