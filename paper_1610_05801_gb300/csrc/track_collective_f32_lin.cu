// The FP32-compensated collective turn kernel's linear-map variants (kernels_coll_f32.cuh),
// in a translation unit of their own so that the two families build in parallel.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_coll_f32.cuh"

namespace phtl {
namespace {

using collf32::k_coll_turn_f32;

template <int S>
const void* kernel_s(int dtype)
{
    if (dtype == PHTL_F32C) return reinterpret_cast<const void*>(&k_coll_turn_f32<S, PHTL_F32C, false>);
    if (dtype == PHTL_F32CD) return reinterpret_cast<const void*>(&k_coll_turn_f32<S, PHTL_F32CD, false>);
    if (dtype == PHTL_F32CS) return reinterpret_cast<const void*>(&k_coll_turn_f32<S, PHTL_F32CS, false>);
    return nullptr;
}

}  // namespace

const void* coll_kernel_f32_lin(int scheme, int dtype)
{
    if (scheme == PHTL_EULER_CROMER) return kernel_s<PHTL_EULER_CROMER>(dtype);
    if (scheme == PHTL_LEAPFROG) return kernel_s<PHTL_LEAPFROG>(dtype);
    if (scheme == PHTL_RUTH4) return kernel_s<PHTL_RUTH4>(dtype);
    return nullptr;
}

}  // namespace phtl
