// The library-owned handle behind the opaque phtl_handle of phtl.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "phtl.h"

namespace phtl {

constexpr uint64_t kHandleMagic = 0x7068746c48414e44ull;  // "phtlHAND"

struct Server;  // continuous-batching serving loop (server.cu)

}  // namespace phtl

struct phtl_handle {
    uint64_t magic = phtl::kHandleMagic;
    phtl_params params{};
    phtl_derived derived{};
    phtl::MapConsts mc[4]{};  // per integrator
    double K2 = 0.0;          // linear strength of the second RF system, eta C A2 k2 cos(phi2)
    // monitor attached by phtl_set_monitor
    double* mon_rows = nullptr;
    int64_t mon_cap = 0;
    int64_t mon_stride = 1;
    // tuning (0 = automatic)
    int32_t block = 0;
    int64_t tpl = 0;
    int32_t max_blocks = 0;
    // device state (filled lazily by ensure_device)
    bool dev_ready = false;
    int device = -1;
    int nsm = 0;
    cudaStream_t stream = nullptr;  // library-owned stream for the host-buffer path
    phtl::Server* server = nullptr;
    // ramp programme (phtl_set_programme): per-turn table on device ramp_device
    phtl::RampTurn* ramp = nullptr;
    int64_t ramp_turns = 0;
    int ramp_device = -1;
    // collective step (phtl_set_wake): one device block holding the wake table w[ns],
    // the wake potential V[ns], the per-slice kick U[ns] (and as float pairs U2[ns]) and
    // two counts buffers [2][ns]
    void* wake_mem = nullptr;
    double* wake_w = nullptr;
    double* wake_V = nullptr;
    double* wake_U = nullptr;
    float2* wake_U2 = nullptr;   // U as float pairs for the FP32 paths
    unsigned* wake_counts = nullptr;
    phtl::CollArgs coll{};
    int wake_device = -1;
    // per-particle slice of the last slicing (2 bytes per particle, grown on demand)
    uint16_t* coll_slot = nullptr;
    int64_t coll_slot_cap = 0;
    phtl_stats stats{};
    // cancellation of persistent tracking calls (phtl_track_cancel): host-mapped words
    // [0] cancel epoch, [1] turns done by the last call's launches that ran; the device
    // gate word of the launch that follows; the epoch and turns of the last call
    long long* ctl_host = nullptr;   // host address (cudaHostAlloc, mapped)
    long long* ctl_dev = nullptr;    // its device address
    int* gate_go = nullptr;          // device word
    long long epoch = 0;
    int64_t last_turns = 0;
    bool last_gated = false;
    // phase times of the last phtl_track_host call, and its events (created on first use)
    phtl_phase_times phases{};
    cudaEvent_t phase_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace phtl {

bool handle_valid(const phtl_handle* h);
void stop_server(phtl_handle* h);
int ensure_device(phtl_handle* h);
int handle_stream(phtl_handle* h, cudaStream_t* out);
void release_handle_resources(phtl_handle* h);
void free_programme(phtl_handle* h);  // api_programme.cu
void free_wake(phtl_handle* h);       // api_collective.cu
int check_track_args(const phtl_handle* h, void* const* c, int64_t n, int64_t turns,
                     int integrator, int dtype);
int enqueue_track(phtl_handle* h, void* const* c, int64_t n, int64_t turns, int integrator,
                  int dtype, cudaStream_t s, bool perturn, double* mon_rows, int64_t mon_cap,
                  int64_t mon_stride);
int64_t auto_turns_per_launch(int dtype, int scheme, int64_t n);
void scheme_weights(int scheme, double A, double etaC, double (&dc)[4], double (&kw)[3]);
double kick_amplitude(const phtl_params& p, const phtl_derived& d, double voltage_V);
// A batched job's stage weights: its scheme's drift weights, kick weights for its own
// voltage, and the ring's second RF system (FP64 and the FP32 splits).
void job_weights(const phtl_handle* h, int scheme, double voltage_V, JobDesc& J);
// MapConsts of a batched launch: the handle's, with the widened map's kernels forced
// when a job of the group uses RK4 (only those kernels hold it).
MapConsts batch_consts(const phtl_handle* h, bool has_rk4);
// PHTL_OK if a job's own voltage gives a stable bucket with the ring's second RF system
// (the rule of phtl_create), else PHTL_E_UNSTABLE.
int voltage_check(const phtl_handle* h, double voltage_V);
// PHTL_LOG level (environment, read once; 0 = silent) and a printf-style line to stderr.
int log_level();
void log_line(const char* fmt, ...);

}  // namespace phtl
