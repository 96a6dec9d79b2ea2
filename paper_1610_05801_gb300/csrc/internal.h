// Internal declarations shared by the translation units of libphtl.so.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "phtl.h"

namespace phtl {

constexpr int kNumDtypes = 4;  // PHTL_F64 .. PHTL_F32CS
constexpr double kPi = 3.14159265358979323846;

inline bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// v as an unevaluated float pair hi + lo (host): hi rounded, lo the rounded remainder.
inline void split_df(double v, float& hi, float& lo)
{
    hi = static_cast<float>(v);
    lo = static_cast<float>(v - static_cast<double>(hi));
}

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
    // the same rotations as three shears, u += p v; v += q u; u += p v with
    // p = beta tan(mu/2), q = -sin(mu)/beta (shear_* = 0: use the matrix instead)
    double shx[2], shy[2];
    int32_t shear_x, shear_y;
    int32_t phis_zero;  // phi_s == 0: the kick is sin(k z), with k z fused into the sine's reduction
    // double-float (FP32 pair) copies for the FP32 paths: value = hi + lo
    float dc_hi[4], dc_lo[4];
    float kw_hi[3], kw_lo[3];
    float k_hi, k_lo, phis_hi, phis_lo, sinphis_hi, sinphis_lo, lin_hi, lin_lo;
    float mx_hi[4], mx_lo[4], my_hi[4], my_lo[4];
    int32_t linear;  // rf_linear flag
    float k2opi;     // k * 2/pi rounded to FP32 (quadrant estimate of the fused FP64 sine)
    // widened map: nonlinear slippage eta(d) = eta0 + eta1 d + eta2 d^2 and chromaticity
    int32_t general;             // eta1, eta2 or a chromaticity nonzero: general turn loop
    int32_t chroma_x, chroma_y;  // xi != 0 in that plane
    int32_t pad2_;
    double eta1C, eta2C;         // eta1 C, eta2 C
    double qx, qy;               // frac(Q): the phase advance in turns
    double xi_x, xi_y;           // chromaticities dQ/d delta
    double bx, by, ibx, iby;     // beta and 1/beta of the chromatic rotations
    float eta1C_hi, eta1C_lo, eta2C_hi, eta2C_lo;
    float qx_hi, qx_lo, qy_hi, qy_lo, xi_x_hi, xi_x_lo, xi_y_hi, xi_y_lo;
    float bx_hi, bx_lo, by_hi, by_lo, ibx_hi, ibx_lo, iby_hi, iby_lo;
    // second RF system (double RF): stage j adds kw2[j] * (sin(phi2 + k2 z) - sin(phi2)),
    // kw2[j] = w_j * A2 (lin2 z in rf_linear mode)
    int32_t dual_rf;
    int32_t pad3_;
    double kw2[3];
    double k2, phi2, sinphi2, lin2;
    float kw2_hi[3], kw2_lo[3];
    float k2_hi, k2_lo, phi2_hi, phi2_lo, sinphi2_hi, sinphi2_lo, lin2_hi, lin2_lo;
};

// Drift stage weights w_i of each scheme (the drift of stage i is w_i eta(d) C d); the
// Ruth4 values are theta/2 and (1 - theta)/2 with theta = 1/(2 - 2^(1/3)).  RK4 has one
// "stage" of weight 1: its right-hand side uses eta(d) C itself.
__host__ __device__ constexpr double drift_weight(int scheme, int i)
{
    return scheme == PHTL_EULER_CROMER ? (i == 0 ? 1.0 : 0.0)
         : scheme == PHTL_LEAPFROG     ? (i < 2 ? 0.5 : 0.0)
         : scheme == PHTL_RK4          ? (i == 0 ? 1.0 : 0.0)
         : (i == 0 || i == 3)          ? 0.6756035959798289
                                       : -0.17560359597982889;
}

// Kick stage weights w_j of each scheme (the kick of stage j is w_j A (sin phi - sin phi_s));
// the Ruth4 values are theta, 1 - 2 theta, theta with theta = 1/(2 - 2^(1/3)).
__host__ __device__ constexpr double kick_weight(int scheme, int j)
{
    return scheme != PHTL_RUTH4 ? (j == 0 ? 1.0 : 0.0)
         : j == 1               ? -1.7024143839193155
                                : 1.3512071919596578;
}

// One turn of a ramp programme (an accelerating bucket: the reference momentum and the RF
// voltage change from turn to turn), derived in FP64 on the host by phtl_set_programme.
struct RampTurn {
    double etaC;     // eta_n C
    double A;        // q V_n / (beta_n p0_n)
    double phis;     // phi_s,n
    double sinphis;  // sin(phi_s,n)
    double lin;      // cos(phi_s,n) k (rf_linear mode)
    double r;        // p0_n / p0_{n+1}: delta and the slopes are re-expressed after the turn
    // double-float copies for the FP32 paths (value = hi + lo)
    float etaC_h, etaC_l, A_h, A_l, phis_h, phis_l, sinphis_h, sinphis_l, lin_h, lin_l, r_h, r_l;
    // each scheme's stage weights times this turn's eta_n C (drifts, first) and A_n (kicks),
    // as FP64 products: Euler-Cromer {dc0, kw0}, leap-frog {dc0, dc1, kw0}, Ruth4
    // {dc0..dc3, kw0..kw2}
    double w_ec[2];
    double w_lf[3];
    double w_r4[7];
};
static_assert(sizeof(RampTurn) == 192, "RampTurn is 192 bytes");

// Slicing grid and strength of the collective (wake) step.
struct CollArgs {
    double z_lo;     // first slice edge
    double inv_dz;   // nslices / (z_hi - z_lo)
    double alpha;    // kick per unit wake potential
    double alpha_sc; // kick per unit line-density slope (space charge)
    int32_t nslices;
    int32_t pad_;
    // double-float copies for the FP32 paths (value = hi + lo)
    float z_lo_h, z_lo_l, inv_dz_h, inv_dz_l;
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
    int32_t scheme;    // PHTL_EULER_CROMER | PHTL_LEAPFROG | PHTL_RUTH4 | PHTL_RK4
    int32_t block;     // threads per block
    int32_t grid;      // blocks
    int32_t vec;       // nonzero: all pointers 16-byte aligned (128-bit loads)
    int32_t pad_;
    const int* go;     // non-null: the launch runs only if *go != 0 (the call's cancellation
                       // gate, written by the gate kernel launched just before it)
};

// The cancellation gate in front of each persistent launch of a call (api.cu): one thread
// reads the handle's cancel epoch from host-mapped memory, writes the launch's decision to
// *go (device memory, read by every block of the launch that follows on the stream) and
// counts the turns that run into *done (host-mapped).
// True when the stream is capturing a CUDA graph (or the query fails): a captured call is
// enqueued without cancellation gates, because a replay would reuse the call's epoch.
bool stream_capturing(cudaStream_t s);
cudaError_t launch_gate(const long long* cancel_epoch, long long epoch, int* go, long long* done,
                        int nturns, bool first, cudaStream_t s);

// One bunch of a batched launch, as the batched kernels read it from the device job
// table.  Jobs are sorted by turns (descending), so the jobs still running at any turn
// chunk form a prefix of the table; tile_begin is the first block index of the job's
// particle tiles (blockDim.x * P particles each).
struct JobDesc {
    void* c[6];          // z, dp, x, xp, y, yp (x..yp pairs may be nullptr)
    double* mon;         // monitor rows or nullptr
    int64_t stride;      // monitor stride (>= 1)
    int64_t n;           // particles
    int64_t turns;       // turns per run of the batch
    int64_t tile_begin;  // first tile (block) of this job
    int64_t turn_offset; // turns this job had done before the launch sequence (monitor rows
                         // continue from there; the initial row is written when it is 0)
    double dc[4];        // drift weights w_i * eta C of the job's scheme
    double kw[3];        // kick weights w_j * A_job of the job's scheme
    float dc_hi[4];      // the same split into FP32 hi + lo (value = hi + lo)
    float dc_lo[4];
    float kw_hi[3];
    float kw_lo[3];
    double kw2[3];       // second RF system's kick weights w_j * A2 (the ring's, not per job)
    float kw2_hi[3];
    float kw2_lo[3];
    int32_t scheme;      // integrator
    int32_t vec;         // nonzero: 16-byte aligned buffers (128-bit loads)
    int32_t pad_;
};
// 6 + 1 pointers, 5 int64, 10 doubles, 20 floats, 3 int32: the no-allocation batch run's
// fixed table is PHTL_NOALLOC_MAX_JOBS of these (69,632 bytes per GPU).
static_assert(sizeof(JobDesc) == 272, "JobDesc layout changed: update the table sizes");

// Split the job's FP64 drift / kick weights into FP32 hi + lo pairs.
inline void fill_float_weights(JobDesc& J)
{
    for (int i = 0; i < 4; ++i) {
        J.dc_hi[i] = static_cast<float>(J.dc[i]);
        J.dc_lo[i] = static_cast<float>(J.dc[i] - static_cast<double>(J.dc_hi[i]));
    }
    for (int i = 0; i < 3; ++i) {
        J.kw_hi[i] = static_cast<float>(J.kw[i]);
        J.kw_lo[i] = static_cast<float>(J.kw[i] - static_cast<double>(J.kw_hi[i]));
        J.kw2_hi[i] = static_cast<float>(J.kw2[i]);
        J.kw2_lo[i] = static_cast<float>(J.kw2[i] - static_cast<double>(J.kw2_hi[i]));
    }
}

// Programmatic dependent launch (sm_90 and later): the kernel is launched while the previous
// kernel on the stream is still finishing, and must execute griddep_wait() before it touches
// memory that kernel writes (griddepcontrol.wait returns once the preceding grid has
// completed and its memory operations are visible).  griddep_launch_dependents() lets the
// next kernel's launch start early.
// Build option PHTL_NO_PDL: plain stream-ordered launches instead (for comparison).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" :::);
}

// Per-particle slice of the collective step's last slicing, kept between the turn kernel that
// counts a particle and the next one, which kicks it by that slice: 2 bytes per particle,
// kSlotOutside for a particle outside the grid.  NP consecutive particles from base (a
// multiple of NP, so the vector access is NP * 2-byte aligned).
constexpr unsigned kSlotOutside = 0xFFFFu;

template <int NP>
__device__ __forceinline__ void slots_load(const uint16_t* __restrict__ s, int64_t base, int64_t n,
                                           int (&k)[NP])
{
    static_assert(NP == 2 || NP == 4, "2 or 4 particles per thread");
    if (base + NP <= n) {
        if constexpr (NP == 2) {
            const unsigned v = *reinterpret_cast<const unsigned*>(s + base);
            k[0] = static_cast<int>(v & 0xFFFFu);
            k[1] = static_cast<int>(v >> 16);
        } else {
            const uint2 v = *reinterpret_cast<const uint2*>(s + base);
            k[0] = static_cast<int>(v.x & 0xFFFFu);
            k[1] = static_cast<int>(v.x >> 16);
            k[2] = static_cast<int>(v.y & 0xFFFFu);
            k[3] = static_cast<int>(v.y >> 16);
        }
    } else {
#pragma unroll
        for (int p = 0; p < NP; ++p) k[p] = base + p < n ? static_cast<int>(s[base + p]) : kSlotOutside;
    }
}

// k[p] < 0 is stored as kSlotOutside.
template <int NP>
__device__ __forceinline__ void slots_store(uint16_t* __restrict__ s, int64_t base, int64_t n,
                                            const int (&k)[NP])
{
    unsigned v[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) v[p] = k[p] < 0 ? kSlotOutside : static_cast<unsigned>(k[p]);
    if (base + NP <= n) {
        if constexpr (NP == 2)
            *reinterpret_cast<unsigned*>(s + base) = v[0] | (v[1] << 16);
        else
            *reinterpret_cast<uint2*>(s + base) = make_uint2(v[0] | (v[1] << 16), v[2] | (v[3] << 16));
    } else {
#pragma unroll
        for (int p = 0; p < NP; ++p)
            if (base + p < n) s[base + p] = static_cast<uint16_t>(v[p]);
    }
}

// floor(u) of a double u with 0 <= u < 4096, from its high word alone (the integer part
// has at most 12 bits, all among the 21 leading significand bits held there); no FP64
// instruction.  hi: the high word of u's bit pattern, non-negative.
__device__ __forceinline__ int floor_small(int hi)
{
    const int e = (hi >> 20) - 1023;  // unbiased exponent
    if (e < 0) return 0;              // u < 1 (zero and subnormals included)
    return ((hi & 0xFFFFF) | 0x100000) >> (20 - e);
}

inline cudaError_t launch_pdl(const void* k, dim3 grid, dim3 block, void** args, size_t smem,
                              cudaStream_t s)
{
#ifdef PHTL_NO_PDL
    return cudaLaunchKernel(k, grid, block, args, smem, s);
#endif
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, k, args);
}

// Launchers (one per kernel family); return cudaGetLastError() of the launch.
cudaError_t launch_track_f64(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                             cudaStream_t s);
cudaError_t launch_track_f32c(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                              int dtype, cudaStream_t s);
cudaError_t launch_perturn(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                           int dtype, cudaStream_t s);

// Batched launch over a job table: turns [t0, t0 + T) of every job with turns > t0
// (grid = the tiles of those jobs), or row-0 records only when T == 0.
cudaError_t launch_batched(const JobDesc* jobs, int32_t njobs, const MapConsts& c, int dtype,
                           bool mon, int64_t t0, int32_t T, int grid, int block, cudaStream_t s);
int occupancy_batched(int dtype, bool mon, int block, bool general);
int particles_per_thread(int dtype);

// Which single-bunch kernel family a map needs: 0 the linear map's, 1 the widened map's,
// 2 the widened map's with the second RF system.
inline int gen_level(const MapConsts& c) { return c.general ? (c.dual_rf ? 2 : 1) : 0; }

// Resident blocks per SM of a kernel variant at a block size (0 = cannot launch);
// gen: the kernel family (gen_level).
int occupancy_f64(int scheme, bool trans, bool mon, int block, int gen);
int occupancy_f32c(int scheme, bool trans, bool mon, int dtype, int block, int gen);
int occupancy_perturn(int scheme, bool trans, bool mon, int dtype, int block, int gen);

// Ramp programme kernels (track_ramp.cu): turns [turn0, turn0 + L.nturns) of the
// programme table prog (device memory), linear map only.
cudaError_t launch_ramp(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                        const RampTurn* prog, int64_t turn0, int dtype, cudaStream_t s);
int occupancy_ramp(int scheme, int dtype, int block);

// Collective step kernels (track_collective.cu): one turn (optionally the previous turn's
// kick U first, a monitor row, the map, the slicing of the new z), and the per-slice wake
// potential V and kick U.
// slot: the per-particle slices (written when counting, read when kicking).
cudaError_t launch_coll_turn(const LaunchDesc& L, const MapConsts& c, const CollArgs& A,
                             const double* U, unsigned* counts, uint16_t* slot, double* mon_rows,
                             int64_t rec_row, bool kick, bool map, cudaStream_t s);
cudaError_t launch_wake_potential(const unsigned* counts, const double* w, const CollArgs& A,
                                  double* V, double* U, float2* U2, unsigned* clear, cudaStream_t s);
int occupancy_coll(int scheme, bool gen, int block, int nslices);  // gen: MapConsts::general
// The FP32-compensated turn kernel (track_collective_f32.cu): the same steps on float-pair
// state, the kick read from U2 (U as hi + lo floats).
cudaError_t launch_coll_turn_f32(const LaunchDesc& L, const MapConsts& c, const CollArgs& A,
                                 const float2* U2, unsigned* counts, uint16_t* slot,
                                 double* mon_rows, int64_t rec_row, bool kick, bool map, int dtype,
                                 cudaStream_t s);
int occupancy_coll_f32(int scheme, int dtype, bool gen, int block, int nslices);
// The linear map's FP32 collective turn kernels (track_collective_f32_lin.cu; not RK4).
const void* coll_kernel_f32_lin(int scheme, int dtype);

// Kernels of the widened map (track_general.cu, track_general_batched.cu).
const void* general_kernel_single(int scheme, int dtype, bool dual);
const void* general_kernel_single_rk4(int dtype);                   // track_general_rk4.cu
const void* general_kernel_single_dual(int scheme, int dtype);      // track_general_dual.cu
const void* general_kernel_single_dual_f32(int scheme, int dtype);  // track_general_dual_f32.cu
const void* general_kernel_batched(int dtype);
const void* general_kernel_batched_f32(int dtype);  // PHTL_F32CD, PHTL_F32CS

}  // namespace phtl
