// Batched kernels of the widened map for PHTL_F32CD and PHTL_F32CS (the FP64 and PHTL_F32C
// ones are in track_general_batched.cu).
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_batched.cuh"

namespace phtl {

const void* general_kernel_batched_f32(int dtype)
{
    if (dtype == PHTL_F32CD) return reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32CD, true, true>);
    if (dtype == PHTL_F32CS) return reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32CS, true, true>);
    return nullptr;
}

}  // namespace phtl
