// Batched kernels of the widened map (slippage expansion, chromaticity): the kernel
// templates of kernels_batched.cuh with GEN = true, in a translation unit of their own.
// Built with MON = true; each job's monitor pointer is checked at run time.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_batched.cuh"

namespace phtl {

const void* general_kernel_batched(int dtype)
{
    if (dtype == PHTL_F64) return reinterpret_cast<const void*>(&k_batched_f64<true, true>);
    if (dtype == PHTL_F32C) return reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32C, true, true>);
    if (dtype == PHTL_F32CD) return reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32CD, true, true>);
    if (dtype == PHTL_F32CS) return reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32CS, true, true>);
    return nullptr;
}

}  // namespace phtl
