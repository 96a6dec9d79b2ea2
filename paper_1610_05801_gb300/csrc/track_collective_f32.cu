// The FP32-compensated collective turn kernel (kernels_coll_f32.cuh): the widened map's
// variants, the dispatch between them and the linear map's (track_collective_f32_lin.cu),
// occupancy and launch.
#include <cuda_runtime.h>

#include "internal.h"
#include "kernels_coll_f32.cuh"

namespace phtl {
namespace {

using collf32::k_coll_turn_f32;

template <int S>
const void* kernel_s(int dtype)
{
    if (dtype == PHTL_F32C) return reinterpret_cast<const void*>(&k_coll_turn_f32<S, PHTL_F32C, true>);
    if (dtype == PHTL_F32CD) return reinterpret_cast<const void*>(&k_coll_turn_f32<S, PHTL_F32CD, true>);
    if (dtype == PHTL_F32CS) return reinterpret_cast<const void*>(&k_coll_turn_f32<S, PHTL_F32CS, true>);
    return nullptr;
}

const void* coll_kernel_f32(int scheme, int dtype, bool gen)
{
    if (!gen && scheme != PHTL_RK4) return coll_kernel_f32_lin(scheme, dtype);
    if (scheme == PHTL_EULER_CROMER) return kernel_s<PHTL_EULER_CROMER>(dtype);
    if (scheme == PHTL_LEAPFROG) return kernel_s<PHTL_LEAPFROG>(dtype);
    if (scheme == PHTL_RUTH4) return kernel_s<PHTL_RUTH4>(dtype);
    if (scheme == PHTL_RK4) return kernel_s<PHTL_RK4>(dtype);
    return nullptr;
}

size_t smem_bytes(int block, int ns)
{
    return static_cast<size_t>((ns + 1) / 2) * sizeof(double) + 2u * (block / 32) * 16 * sizeof(double);
}

}  // namespace

int occupancy_coll_f32(int scheme, int dtype, bool gen, int block, int nslices)
{
    const void* k = coll_kernel_f32(scheme, dtype, gen);
    if (!k) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem_bytes(block, nslices)) !=
        cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_coll_turn_f32(const LaunchDesc& L, const MapConsts& c, const CollArgs& A,
                                 const float2* U2, unsigned* counts, uint16_t* slot,
                                 double* mon_rows, int64_t rec_row, bool kick, bool map, int dtype,
                                 cudaStream_t s)
{
    const void* k = coll_kernel_f32(L.scheme, dtype, c.general != 0);
    if (!k) return cudaErrorInvalidValue;
    LaunchDesc Lc = L;
    MapConsts cc = c;
    CollArgs aa = A;
    const float2* uu = U2;
    unsigned* cn = counts;
    uint16_t* sl = slot;
    double* mr = mon_rows;
    int64_t rr = rec_row;
    int kk = kick ? 1 : 0, mm = map ? 1 : 0;
    void* args[] = {&Lc, &cc, &aa, &uu, &cn, &sl, &mr, &rr, &kk, &mm};
    return launch_pdl(k, dim3(L.grid), dim3(L.block), args, smem_bytes(L.block, A.nslices), s);
}

}  // namespace phtl
