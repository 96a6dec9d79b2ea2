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
    phtl::MapConsts mc[3]{};  // per integrator
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
    phtl_stats stats{};
};

namespace phtl {

bool handle_valid(const phtl_handle* h);
void stop_server(phtl_handle* h);
int ensure_device(phtl_handle* h);
int handle_stream(phtl_handle* h, cudaStream_t* out);
void release_handle_resources(phtl_handle* h);
int check_track_args(const phtl_handle* h, void* const* c, int64_t n, int64_t turns,
                     int integrator, int dtype);
int enqueue_track(phtl_handle* h, void* const* c, int64_t n, int64_t turns, int integrator,
                  int dtype, cudaStream_t s, bool perturn, double* mon_rows, int64_t mon_cap,
                  int64_t mon_stride);
int64_t auto_turns_per_launch(int dtype, int scheme, int64_t n);
void scheme_weights(int scheme, double A, double etaC, double (&dc)[4], double (&kw)[3]);
double kick_amplitude(const phtl_params& p, const phtl_derived& d, double voltage_V);

}  // namespace phtl
