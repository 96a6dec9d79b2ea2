// phtl_batch_run_noalloc: the batched launch without any memory allocation.
//
// Some callers cannot let this library allocate device memory: an application whose
// device memory is owned and budgeted by its own allocator or memory pool (the library
// taking memory behind its back would break that accounting), or a loop that must never
// pay for cudaMalloc / cudaFree, which can block the host and synchronise the device.
// For them this entry point runs the same batched kernels as phtl_batch_create +
// phtl_batch_run, but the job table lives in a file-scope device array of fixed size
// instead of memory allocated per batch, and no graph, autotuner probe or staging buffer
// is created.  The caller still passes the particle and monitor buffers.
//
// The array is shared by every call in the process and keeps the last call's contents;
// each call rewrites all the entries it uses, so nothing carries over from one call to
// the next.  Calls that can overlap on the GPU (for example on two streams with no
// ordering between them) race on the array and must not be issued that way.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "handle.h"
#include "internal.h"

namespace phtl {
namespace {

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) JobDesc g_noalloc_jobs[PHTL_NOALLOC_MAX_JOBS];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
JobDesc* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device (the
// array's name is only a host-side stand-in in host code).
int noalloc_table(int device, JobDesc** out)
{
    if (device < 0 || device >= kMaxDevices) return PHTL_E_NODEVICE;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_jobs);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return PHTL_E_CUDA;
        }
        g_noalloc_ptr[device] = static_cast<JobDesc*>(p);
    }
    *out = g_noalloc_ptr[device];
    return PHTL_OK;
}

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return PHTL_OK;
    cudaGetLastError();
    return PHTL_E_CUDA;
}

}  // namespace
}  // namespace phtl

using namespace phtl;

extern "C" int phtl_batch_run_noalloc(phtl_handle* h, const phtl_job* jobs, int32_t njobs,
                                      void* cuda_stream)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (njobs < 0 || (njobs > 0 && !jobs)) return PHTL_E_INVALID;
    if (njobs > PHTL_NOALLOC_MAX_JOBS) return PHTL_E_TOOBIG;
    for (int32_t i = 0; i < njobs; ++i) {
        const phtl_job& J = jobs[i];
        int rc = check_track_args(h, J.c, J.n, J.turns, J.integrator, J.dtype);
        if (rc != PHTL_OK) return rc;
        if (!std::isfinite(J.voltage_V)) return PHTL_E_INVALID;
        if (J.mon_rows) {
            if (J.mon_stride < 1 || J.turns / J.mon_stride + 1 > J.mon_capacity) return PHTL_E_INVALID;
            if (reinterpret_cast<uintptr_t>(J.mon_rows) % 8) return PHTL_E_INVALID;
        }
        if (voltage_check(h, J.voltage_V) != PHTL_OK) return PHTL_E_UNSTABLE;
        if (J.turns > (int64_t(1) << 40)) return PHTL_E_INVALID;
    }
    int rc = ensure_device(h);
    if (rc != PHTL_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // The table is copied from this call's stack frame: inside a stream capture that copy
    // would become a graph node reading a dead frame at replay, so a capturing stream is
    // refused before anything is enqueued.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return PHTL_E_CAPTURE;
    }
    if (cap != cudaStreamCaptureStatusNone) return PHTL_E_CAPTURE;
    JobDesc* table = nullptr;
    rc = noalloc_table(h->device, &table);
    if (rc != PHTL_OK) return rc;
    if (njobs == 0) return PHTL_OK;

    // Pass 1 (host only): the table of every arithmetic group and its launch shape, with
    // every check, so that a rejected call enqueues nothing.  On the stack, no allocation.
    struct Group {
        int32_t dtype, first, cnt;
        int32_t block;
        bool mon;
        MapConsts mc;
        int64_t T, tiles;
    };
    JobDesc host[PHTL_NOALLOC_MAX_JOBS];
    int32_t order[PHTL_NOALLOC_MAX_JOBS];
    Group groups[4];
    int32_t ngroups = 0, used = 0;
    for (int dt = PHTL_F64; dt <= PHTL_F32CS; ++dt) {
        int32_t cnt = 0;
        int32_t* ord = order + used;
        for (int32_t i = 0; i < njobs; ++i)
            if (jobs[i].dtype == dt) ord[cnt++] = i;
        if (cnt == 0) continue;
        std::stable_sort(ord, ord + cnt,
                         [&](int32_t a, int32_t b) { return jobs[a].turns > jobs[b].turns; });
        int64_t active = 0;
        bool mon = false, rk4 = false;
        for (int32_t k = 0; k < cnt; ++k) {
            active += jobs[ord[k]].n;
            mon = mon || jobs[ord[k]].mon_rows != nullptr;
            rk4 = rk4 || jobs[ord[k]].integrator == PHTL_RK4;
        }
        Group& g = groups[ngroups++];
        g.dtype = dt;
        g.first = used;
        g.cnt = cnt;
        g.mon = mon;
        g.mc = batch_consts(h, rk4);
        g.block = h->block > 0 ? h->block : 128;
        if (occupancy_batched(dt, mon, g.block, g.mc.general != 0) <= 0) return PHTL_E_INVALID;
        g.T = h->tpl > 0 ? h->tpl : auto_turns_per_launch(dt, jobs[ord[0]].integrator, active);
        const int64_t per_tile = static_cast<int64_t>(g.block) * particles_per_thread(dt);
        JobDesc* G = host + used;
        int64_t tiles = 0;
        for (int32_t k = 0; k < cnt; ++k) {
            const phtl_job& U = jobs[ord[k]];
            JobDesc& J = G[k];
            std::memset(&J, 0, sizeof(J));
            bool vec = true;
            for (int c = 0; c < 6; ++c) {
                J.c[c] = U.c[c];
                if (U.c[c] && reinterpret_cast<uintptr_t>(U.c[c]) % 16) vec = false;
            }
            if (dt != PHTL_F64 && (U.n * 4) % 16) vec = false;
            J.vec = vec ? 1 : 0;
            J.mon = U.mon_rows;
            J.stride = U.mon_rows ? U.mon_stride : 1;
            J.n = U.n;
            J.turns = U.turns;
            J.scheme = U.integrator;
            J.tile_begin = tiles;
            job_weights(h, U.integrator, U.voltage_V, J);
            tiles += (U.n + per_tile - 1) / per_tile;
        }
        if (tiles > (int64_t(1) << 31) - 1) return PHTL_E_INVALID;
        g.tiles = tiles;
        used += cnt;
    }

    // Pass 2: the whole table in one copy, then per group its monitor clears and its chunk
    // launches (all stream-ordered).  A CUDA error here can leave earlier groups enqueued.
    rc = cuda_rc(cudaMemcpyAsync(table, host, sizeof(JobDesc) * used, cudaMemcpyHostToDevice, s));
    if (rc != PHTL_OK) return rc;
    for (int32_t gi = 0; gi < ngroups; ++gi) {
        const Group& g = groups[gi];
        const JobDesc* G = host + g.first;
        for (int32_t k = 0; k < g.cnt; ++k) {
            if (!G[k].mon) continue;
            rc = cuda_rc(cudaMemsetAsync(G[k].mon, 0,
                                         static_cast<size_t>(G[k].turns / G[k].stride + 1) * PHTL_MON_FIELDS * 8, s));
            if (rc != PHTL_OK) return rc;
        }
        const int64_t max_turns = G[0].turns;
        int64_t t0 = 0, nl = 0;
        do {
            int32_t k = g.cnt;
            if (t0 > 0) {
                k = 0;
                while (k < g.cnt && G[k].turns > t0) ++k;
            }
            const int64_t grid = k == g.cnt ? g.tiles : G[k].tile_begin;
            const int32_t nt = static_cast<int32_t>(std::min<int64_t>(g.T, std::max<int64_t>(max_turns - t0, 0)));
            if (grid > 0) {
                rc = cuda_rc(launch_batched(table + g.first, g.cnt, g.mc, g.dtype, g.mon, t0, nt,
                                            static_cast<int>(grid), g.block, s));
                if (rc != PHTL_OK) return rc;
                ++nl;
            }
            t0 += g.T;
        } while (t0 < max_turns);
        h->stats.launches += nl;
    }
    for (int32_t i = 0; i < njobs; ++i) h->stats.particle_turns += jobs[i].n * jobs[i].turns;
    ++h->stats.calls;
    log_line("batch_run_noalloc jobs=%d groups=%d", njobs, ngroups);
    return PHTL_OK;
}
