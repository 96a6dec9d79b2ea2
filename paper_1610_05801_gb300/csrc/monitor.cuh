// Per-turn bunch-moment reduction shared by the tracking kernels.
//
// Each thread holds NF partial sums (field j of a monitor row, see phtl.h).  A warp
// reduce-scatter halves the number of fields per lane at every butterfly step, so a
// lane performs NF adds in total instead of 5*NF for NF independent butterflies; FP64
// adds are the scarce resource on this GPU (2 per clock per SM).  After the scatter,
// lane L holds the warp total of field L / (32 / NF).  The warps' totals meet in
// shared memory (double-buffered by record parity, so one __syncthreads per record
// suffices) and warp 0 adds them up and issues one FP64 atomicAdd per field.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "dfloat.cuh"
#include "phtl.h"

namespace phtl {

constexpr unsigned kFullMask = 0xffffffffu;

// Reduce-scatter NF fields (NF in {8, 16}) across the warp; returns this lane's field
// total.  Which field: NF == 16 -> lane >> 1, NF == 8 -> lane >> 2.
template <int NF>
__device__ __forceinline__ double warp_reduce_scatter(double (&f)[NF], int lane)
{
    static_assert(NF == 8 || NF == 16, "NF must be 8 or 16");
#pragma unroll
    for (int o = 16; o >= (NF == 16 ? 2 : 4); o >>= 1) {
        const int h = (NF == 16) ? (o >> 1) : (o >> 2);  // fields kept after this step
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < NF / 2; ++i) {
            if (i < h) {
                double send = upper ? f[i] : f[i + h];
                double keep = upper ? f[i + h] : f[i];
                f[i] = keep + __shfl_xor_sync(kFullMask, send, o);
            }
        }
    }
    double v = f[0];
    if (NF == 8) v += __shfl_xor_sync(kFullMask, v, 2);
    v += __shfl_xor_sync(kFullMask, v, 1);
    return v;
}

// Block-level reduction + atomics into monitor row `row`.
// smem: 2 * (blockDim.x / 32) * 16 doubles.  nvalid: number of leading fields of the
// row that may be nonzero (6 = longitudinal only, 16 = with transverse planes).
template <int NF>
__device__ __forceinline__ void block_record(double (&f)[NF], double* smem, int parity,
                                             double* __restrict__ rows, int64_t row,
                                             int nvalid)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const double v = warp_reduce_scatter<NF>(f, lane);
    double* buf = smem + parity * (nwarps * 16);
    constexpr int kShift = (NF == 16) ? 1 : 2;
    if ((lane & ((1 << kShift) - 1)) == 0) buf[warp * 16 + (lane >> kShift)] = v;
    __syncthreads();
    if (warp == 0 && lane < nvalid) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += buf[w * 16 + lane];
        atomicAdd(rows + row * PHTL_MON_FIELDS + lane, s);
    }
}

// The same reduction with double-float (FP32 pair) partial sums, for the FP64 kernel:
// the butterfly and the block sum run on the FP32 pipe; only the block total of each
// field is converted to FP64 for the atomic add.  smem: 2 * (blockDim.x / 32) * 16 DF2.
template <int NF>
__device__ __forceinline__ DF2 warp_reduce_scatter_df(DF2 (&f)[NF], int lane)
{
    static_assert(NF == 8 || NF == 16, "NF must be 8 or 16");
#pragma unroll
    for (int o = 16; o >= (NF == 16 ? 2 : 4); o >>= 1) {
        const int h = (NF == 16) ? (o >> 1) : (o >> 2);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < NF / 2; ++i) {
            if (i < h) {
                const DF2 send = upper ? f[i] : f[i + h];
                const DF2 keep = upper ? f[i + h] : f[i];
                f[i] = df_add(keep, df_shfl_xor(send, o));
            }
        }
    }
    DF2 v = f[0];
    if (NF == 8) v = df_add(v, df_shfl_xor(v, 2));
    v = df_add(v, df_shfl_xor(v, 1));
    return v;
}

template <int NF>
__device__ __forceinline__ void block_record_df(DF2 (&f)[NF], DF2* smem, int parity,
                                                double* __restrict__ rows, int64_t row,
                                                int nvalid)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const DF2 v = warp_reduce_scatter_df<NF>(f, lane);
    DF2* buf = smem + parity * (nwarps * 16);
    constexpr int kShift = (NF == 16) ? 1 : 2;
    if ((lane & ((1 << kShift) - 1)) == 0) buf[warp * 16 + (lane >> kShift)] = v;
    __syncthreads();
    if (warp == 0 && lane < nvalid) {
        DF2 s = buf[lane];
        for (int w = 1; w < nwarps; ++w) s = df_add(s, buf[w * 16 + lane]);
        atomicAdd(rows + row * PHTL_MON_FIELDS + lane, df_to_double(s));
    }
}

}  // namespace phtl
