// Host side of the batched launch (phtl_batch_*) and of the block-size / turns-per-launch
// autotuner (phtl_autotune).
//
// A batch packs many independent bunches -- different sizes, turn counts, RF voltages,
// integrators -- into one device job table per arithmetic type.  One run enqueues, per
// type, a memset of the monitors and a sequence of chunk launches (turns [t0, t0 + T)),
// each over the tiles of the jobs still running; the whole sequence is captured once into
// a CUDA graph and replayed.  Turns per launch T bound each kernel's duration (Sec. 2.3's
// hybrid loop: long enough to amortise the launch, short enough to stay responsive).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <unordered_set>
#include <vector>

#include "handle.h"
#include "internal.h"

namespace phtl {
namespace {

constexpr uint64_t kBatchMagic = 0x706874624241544bull;  // "phtbBATK"
std::mutex g_batch_mu;
std::unordered_set<const phtl_batch*> g_batches;

int check_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return PHTL_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PHTL_E_NOMEM : PHTL_E_CUDA;
}

}  // namespace

// Time `reps` launches of the batched kernel of `dtype` at block size `block` over a
// single scratch job of m particles and `turns` turns; returns particle-turns per second
// (0 on failure).  Scratch buffers are allocated and freed here.
double probe_rate(phtl_handle* h, int dtype, int scheme, int block, int64_t m, int turns,
                  cudaStream_t s)
{
    const size_t es = dtype == PHTL_F64 ? sizeof(double) : 2 * sizeof(float);
    // a multiple of 16 particles keeps z, dp and the FP32C comp halves 16-byte aligned
    m = (m + 15) / 16 * 16;
    void* zd = nullptr;
    JobDesc* dj = nullptr;
    double rate = 0.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    do {
        if (cudaMalloc(&zd, 2 * es * static_cast<size_t>(m)) != cudaSuccess) break;
        // small nonzero coordinates: the probe's cost does not depend on the values
        if (cudaMemsetAsync(zd, 0x3c, 2 * es * static_cast<size_t>(m), s) != cudaSuccess) break;
        JobDesc J;
        std::memset(&J, 0, sizeof(J));
        J.c[0] = zd;
        J.c[1] = static_cast<char*>(zd) + es * m;
        J.n = m;
        J.turns = turns;
        J.stride = 1;
        J.scheme = scheme;
        const bool aligned = reinterpret_cast<uintptr_t>(J.c[0]) % 16 == 0 &&
                             reinterpret_cast<uintptr_t>(J.c[1]) % 16 == 0 &&
                             (dtype == PHTL_F64 || (m * 4) % 16 == 0);
        J.vec = aligned ? 1 : 0;
        job_weights(h, scheme, h->params.voltage_V, J);
        if (cudaMalloc(reinterpret_cast<void**>(&dj), sizeof(JobDesc)) != cudaSuccess) break;
        if (cudaMemcpyAsync(dj, &J, sizeof(J), cudaMemcpyHostToDevice, s) != cudaSuccess) break;
        const int ppt = particles_per_thread(dtype);
        const int grid = static_cast<int>((m + static_cast<int64_t>(block) * ppt - 1) /
                                          (static_cast<int64_t>(block) * ppt));
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) break;
        // warm-up, then the best of three
        if (launch_batched(dj, 1, h->mc[scheme], dtype, false, 0, turns, grid, block, s) != cudaSuccess)
            break;
        float best = 1e30f;
        bool ok = true;
        for (int r = 0; r < 3 && ok; ++r) {
            ok = cudaEventRecord(e0, s) == cudaSuccess &&
                 launch_batched(dj, 1, h->mc[scheme], dtype, false, 0, turns, grid, block, s) ==
                     cudaSuccess &&
                 cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0.0f;
            if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best = std::min(best, ms);
        }
        if (ok && best > 0.0f && best < 1e30f)
            rate = static_cast<double>(m) * turns / (static_cast<double>(best) * 1e-3);
    } while (false);
    cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (dj) cudaFree(dj);
    if (zd) cudaFree(zd);
    cudaGetLastError();
    return rate;
}

// Autotuner: the fastest block size on a scratch probe that fills the GPU once, then the
// turns per launch that make a launch over `active` particles last about target_ms.
int autotune(phtl_handle* h, int dtype, int scheme, int64_t active, double target_ms,
             phtl_tuning* out)
{
    int rc = ensure_device(h);
    if (rc != PHTL_OK) return rc;
    cudaStream_t s = nullptr;
    rc = handle_stream(h, &s);
    if (rc != PHTL_OK) return rc;
    const int ppt = particles_per_thread(dtype);
    const int candidates[] = {64, 96, 128, 192, 256};
    int best_block = 0;
    double best_rate = 0.0;
    for (int b : candidates) {
        const int occ = occupancy_batched(dtype, false, b, h->mc[scheme].general != 0);
        if (occ <= 0) continue;
        const int64_t cap = static_cast<int64_t>(occ) * h->nsm * b * ppt;  // one full wave
        const int64_t m = std::max<int64_t>(std::min<int64_t>(std::max<int64_t>(active, 1), cap), b * ppt);
        const int probe_turns = dtype == PHTL_F64 ? 16 : 64;
        const double r = probe_rate(h, dtype, scheme, b, m, probe_turns, s);
        if (r > best_rate * 1.02) {  // prefer the smaller block unless clearly faster
            best_rate = r;
            best_block = b;
        }
    }
    if (best_block == 0) return PHTL_E_CUDA;
    const double a = static_cast<double>(std::max<int64_t>(active, 1));
    double T = best_rate * target_ms * 1e-3 / a;
    T = std::min(std::max(T, 8.0), 1048576.0);
    out->block_threads = best_block;
    out->turns_per_launch = static_cast<int64_t>(T);
    out->particle_turns_per_s = best_rate;
    return PHTL_OK;
}

}  // namespace phtl

struct phtl_batch {
    uint64_t magic = phtl::kBatchMagic;
    phtl_handle* h = nullptr;
    struct Group {
        int dtype = 0;
        bool mon = false;
        int block = 0;
        int64_t T = 0;
        std::vector<phtl::JobDesc> jobs;    // sorted by turns, descending
        std::vector<int64_t> mon_bytes;     // per sorted job
        phtl::JobDesc* d_jobs = nullptr;
        int64_t tiles = 0;
        double rate = 0.0;
        bool rk4 = false;                   // a job uses RK4: the widened map's kernels
    };
    std::vector<Group> groups;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = true;
    phtl_batch_info info{};
};

namespace phtl {
namespace {

bool batch_valid(const phtl_batch* b)
{
    if (!b) return false;
    std::lock_guard<std::mutex> g(g_batch_mu);
    return g_batches.count(b) != 0 && b->magic == kBatchMagic;
}

// Enqueue one run of the batch on stream s (monitor memsets + chunk launches).
int enqueue_batch(phtl_batch* b, cudaStream_t s, int64_t* launches)
{
    int64_t nl = 0;
    for (auto& G : b->groups) {
        for (size_t j = 0; j < G.jobs.size(); ++j)
            if (G.jobs[j].mon) {
                int rc = check_cuda(cudaMemsetAsync(G.jobs[j].mon, 0, G.mon_bytes[j], s));
                if (rc != PHTL_OK) return rc;
            }
        if (G.jobs.empty()) continue;
        const int64_t max_turns = G.jobs.front().turns;
        int64_t t0 = 0;
        do {
            // jobs still running at t0 form a prefix of the table (all jobs at t0 = 0)
            size_t k = G.jobs.size();
            if (t0 > 0) {
                k = 0;
                while (k < G.jobs.size() && G.jobs[k].turns > t0) ++k;
            }
            const int64_t grid = k == G.jobs.size() ? G.tiles : G.jobs[k].tile_begin;
            const int32_t T = static_cast<int32_t>(std::min<int64_t>(G.T, std::max<int64_t>(max_turns - t0, 0)));
            if (grid > 0) {
                int rc = check_cuda(launch_batched(G.d_jobs, static_cast<int32_t>(G.jobs.size()),
                                                   batch_consts(b->h, G.rk4), G.dtype, G.mon, t0, T,
                                                   static_cast<int>(grid), G.block, s));
                if (rc != PHTL_OK) return rc;
                ++nl;
            }
            t0 += G.T;
        } while (t0 < max_turns);
    }
    if (launches) *launches = nl;
    return PHTL_OK;
}

}  // namespace
}  // namespace phtl

using namespace phtl;

extern "C" {

int phtl_autotune(phtl_handle* h, int dtype, int integrator, int64_t active_particles,
                  double target_launch_ms, phtl_tuning* out)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (!out || dtype < PHTL_F64 || dtype > PHTL_F32CS || integrator < 0 || integrator > PHTL_RK4 ||
        active_particles < 0 || !(target_launch_ms > 0.0))
        return PHTL_E_INVALID;
    return autotune(h, dtype, integrator, active_particles, target_launch_ms, out);
}

int phtl_batch_create(phtl_handle* h, const phtl_job* jobs, int32_t njobs, int32_t use_graph,
                      phtl_batch** out)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (!out || njobs < 0 || (njobs > 0 && !jobs)) return PHTL_E_INVALID;
    *out = nullptr;
    // validate every job first
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
    phtl_batch* b = new (std::nothrow) phtl_batch();
    if (!b) return PHTL_E_NOMEM;
    b->h = h;
    b->use_graph = use_graph != 0;
    b->info.njobs = njobs;
    b->info.graph = b->use_graph ? 1 : 0;

    for (int dt = PHTL_F64; dt <= PHTL_F32CS; ++dt) {
        std::vector<int32_t> idx;
        for (int32_t i = 0; i < njobs; ++i)
            if (jobs[i].dtype == dt) idx.push_back(i);
        if (idx.empty()) continue;
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int32_t a, int32_t c) { return jobs[a].turns > jobs[c].turns; });
        phtl_batch::Group G;
        G.dtype = dt;
        int64_t active = 0, pt = 0;
        int counts[4] = {0, 0, 0, 0};
        for (int32_t i : idx) {
            active += jobs[i].n;
            pt += jobs[i].n * jobs[i].turns;
            counts[jobs[i].integrator]++;
            G.mon = G.mon || jobs[i].mon_rows != nullptr;
        }
        G.rk4 = counts[PHTL_RK4] > 0;
        const int dominant = static_cast<int>(std::max_element(counts, counts + 4) - counts);
        if (h->block > 0 && h->tpl > 0) {
            G.block = h->block;
            G.T = h->tpl;
        } else {
            phtl_tuning t;
            rc = autotune(h, dt, dominant, active, 20.0, &t);
            if (rc != PHTL_OK) {
                delete b;
                return rc;
            }
            G.block = h->block > 0 ? h->block : t.block_threads;
            G.T = h->tpl > 0 ? h->tpl : t.turns_per_launch;
            G.rate = t.particle_turns_per_s;
        }
        if (occupancy_batched(dt, G.mon, G.block, batch_consts(h, G.rk4).general != 0) <= 0) {
            delete b;
            return PHTL_E_INVALID;
        }
        const int64_t per_tile = static_cast<int64_t>(G.block) * particles_per_thread(dt);
        int64_t tiles = 0;
        for (int32_t i : idx) {
            const phtl_job& U = jobs[i];
            JobDesc J;
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
            G.jobs.push_back(J);
            G.mon_bytes.push_back(U.mon_rows ? (U.turns / U.mon_stride + 1) * PHTL_MON_FIELDS * 8 : 0);
        }
        G.tiles = tiles;
        if (tiles > (int64_t(1) << 31) - 1) {
            delete b;
            return PHTL_E_INVALID;
        }
        if (cudaMalloc(reinterpret_cast<void**>(&G.d_jobs), sizeof(JobDesc) * G.jobs.size()) != cudaSuccess ||
            cudaMemcpy(G.d_jobs, G.jobs.data(), sizeof(JobDesc) * G.jobs.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            if (G.d_jobs) cudaFree(G.d_jobs);
            for (auto& g2 : b->groups) cudaFree(g2.d_jobs);
            delete b;
            return PHTL_E_NOMEM;
        }
        const int slot = dt;
        b->info.block_threads[slot] = G.block;
        b->info.turns_per_launch[slot] = G.T;
        b->info.probe_particle_turns_per_s[slot] = G.rate;
        b->info.particle_turns_per_run += pt;
        b->info.tiles_first_launch += tiles;
        if (log_level() > 0)
            log_line("batch_create dtype=%d jobs=%zu block=%d turns_per_launch=%lld probe=%.3e "
                     "particle_turns=%.3e graph=%d", dt, G.jobs.size(), G.block,
                     static_cast<long long>(G.T), G.rate, static_cast<double>(pt), use_graph ? 1 : 0);
        b->groups.push_back(std::move(G));
    }
    {
        std::lock_guard<std::mutex> g(g_batch_mu);
        g_batches.insert(b);
    }
    *out = b;
    return PHTL_OK;
}

int phtl_batch_run(phtl_batch* b, void* cuda_stream)
{
    if (!batch_valid(b)) return PHTL_E_BADHANDLE;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (!b->use_graph) {
        int64_t nl = 0;
        int rc = enqueue_batch(b, s, &nl);
        b->info.launches_per_run = nl;
        if (rc == PHTL_OK) {
            b->h->stats.launches += nl;
            b->h->stats.particle_turns += b->info.particle_turns_per_run;
            ++b->h->stats.calls;
        }
        return rc;
    }
    if (!b->exec) {
        if (!b->cap_stream &&
            cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return check_cuda(cudaErrorUnknown);
        int rc = check_cuda(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        if (rc != PHTL_OK) return rc;
        int64_t nl = 0;
        rc = enqueue_batch(b, b->cap_stream, &nl);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (rc != PHTL_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc != PHTL_OK ? rc : PHTL_E_CUDA;
        }
        if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            b->exec = nullptr;
            return check_cuda(cudaErrorUnknown);
        }
        b->graph = g;
        b->info.launches_per_run = nl;
    }
    b->h->stats.launches += b->info.launches_per_run;
    b->h->stats.particle_turns += b->info.particle_turns_per_run;
    ++b->h->stats.calls;
    return check_cuda(cudaGraphLaunch(b->exec, s));
}

int phtl_batch_info_get(const phtl_batch* b, phtl_batch_info* out)
{
    if (!batch_valid(b)) return PHTL_E_BADHANDLE;
    if (!out) return PHTL_E_INVALID;
    *out = b->info;
    return PHTL_OK;
}

int phtl_batch_destroy(phtl_batch* b)
{
    {
        std::lock_guard<std::mutex> g(g_batch_mu);
        if (!b || !g_batches.count(b) || b->magic != kBatchMagic) return PHTL_E_BADHANDLE;
        g_batches.erase(b);
    }
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (auto& G : b->groups)
        if (G.d_jobs) cudaFree(G.d_jobs);
    cudaGetLastError();
    b->magic = 0;
    delete b;
    return PHTL_OK;
}

}  // extern "C"
