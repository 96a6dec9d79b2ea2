// Internal declarations shared by the translation units of libphtl.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "phtl.h"

namespace phtl {

// Per-stage coefficients of one turn of the longitudinal map (Sec. 1.1.2 schemes),
// pre-multiplied on the host in FP64:
//   drift stage i:  z <- z - dc[i] * delta           dc[i] = w_i * eta * C
//   kick stage j:   delta <- delta + kw[j] * (sin(phi_s + k z) - sin(phi_s))
//                   kw[j] = w_j * A;  in rf_linear mode the bracket is lin * z.
// EC uses kw[0] then dc[0]; LF dc[0] kw[0] dc[1]; RUTH4 dc0 kw0 dc1 kw1 dc2 kw2 dc3.
struct MapConsts {
    double dc[4];
    double kw[3];
    double k;        // 2 pi h / C
    double phis;     // phi_s
    double sinphis;  // sin(phi_s)
    double lin;      // cos(phi_s) * k (rf_linear mode)
    double mx[4];    // transverse one-turn matrices, row-major
    double my[4];
    // double-float (FP32 pair) copies for the FP32 paths: value = hi + lo
    float dc_hi[4], dc_lo[4];
    float kw_hi[3], kw_lo[3];
    float k_hi, k_lo, phis_hi, phis_lo, sinphis_f, lin_f;
    float mx_hi[4], mx_lo[4], my_hi[4], my_lo[4];
    int32_t linear;  // rf_linear flag
    int32_t pad_;
};

// Where and when a launch records monitor rows.
struct MonitorArgs {
    double* rows;      // device rows (PHTL_MON_FIELDS doubles each) or nullptr
    int64_t stride;    // record every stride-th turn of the call
    int64_t until;     // turns from this launch's start until the next record (1..stride)
    int64_t row;       // row index of that next record
    int32_t initial;   // nonzero: record row 0 from the loaded state first
    int32_t pad_;
};

// One launch of a tracking kernel over a contiguous particle range.
struct LaunchDesc {
    void* c[6];        // z, dp, x, xp, y, yp (nullptr = plane off)
    int64_t n;         // particles
    int32_t nturns;    // turns in this launch
    int32_t scheme;    // PHTL_EULER_CROMER | PHTL_LEAPFROG | PHTL_RUTH4
    int32_t block;     // threads per block
    int32_t grid;      // blocks
    int32_t vec;       // nonzero: all pointers 16-byte aligned (128-bit loads)
    int32_t pad_;
};

// Launchers (one per kernel family); return cudaGetLastError() of the launch.
cudaError_t launch_track_f64(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                             cudaStream_t s);
cudaError_t launch_track_f32c(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                              int dtype, cudaStream_t s);
cudaError_t launch_perturn(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                           int dtype, cudaStream_t s);

// Resident blocks per SM of a kernel variant at a block size (0 = cannot launch).
int occupancy_f64(int scheme, bool trans, bool mon, int block);
int occupancy_f32c(int scheme, bool trans, bool mon, int dtype, int block);
int occupancy_perturn(int scheme, bool trans, bool mon, int dtype, int block);

}  // namespace phtl
