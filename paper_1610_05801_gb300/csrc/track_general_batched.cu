// Batched kernels of the widened map (slippage expansion, chromaticity, second RF system,
// classic RK4): the kernel templates of kernels_batched.cuh with GEN = true, in
// translation units of their own (FP64 and PHTL_F32C here, PHTL_F32CD and PHTL_F32CS in
// track_general_batched_f32.cu, so that they build in parallel).  Built with MON = true;
// each job's monitor pointer is checked at run time.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_batched.cuh"

namespace phtl {

const void* general_kernel_batched(int dtype)
{
    if (dtype == PHTL_F64) return reinterpret_cast<const void*>(&k_batched_f64<true, true>);
    if (dtype == PHTL_F32C) return reinterpret_cast<const void*>(&k_batched_f32c<PHTL_F32C, true, true>);
    return general_kernel_batched_f32(dtype);
}

}  // namespace phtl
