// Serving loop: the CUDA executor of the continuous-batching scheduler (server_core.h)
// and the phtl_server_* / phtl_submit / phtl_poll / phtl_wait / phtl_cancel / phtl_release
// entry points.
//
// Device work of one scheduling round: the active jobs are split by arithmetic (FP64,
// FP32C, FP32CD), each group's job table (sorted by remaining turns) is uploaded and one
// batched launch advances every job of the group by up to the round's chunk of turns.
// FP64 rounds run on one stream and FP32 rounds on another, so the two overlap on the
// device (FP64 pipe vs FP32 pipe / SFU).  The chunk of turns is re-chosen every round so
// that a round lasts about target_round_ms for the current number of active particles;
// per-particle arithmetic does not depend on the chunking, so a job's result is bitwise
// the same whatever it shared its rounds with.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "handle.h"
#include "internal.h"
#include "server_core.h"

namespace phtl {

int autotune(phtl_handle* h, int dtype, int scheme, int64_t active, double target_ms,
             phtl_tuning* out);

namespace {

struct DevJob {
    void* d[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double* mon = nullptr;
    int64_t mon_rows = 0;
    int stream = 0;  // 0: FP64 stream, 1: FP32 stream
};

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return PHTL_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PHTL_E_NOMEM : PHTL_E_CUDA;
}

int64_t coord_bytes(const phtl_request& r) { return 8 * r.n; }  // n doubles or 2n floats

int ncoords(const phtl_request& r)
{
    const void* const* p = r.resume_ticket ? const_cast<const void* const*>(r.out) : r.in;
    return 2 + (p[2] ? 2 : 0) + (p[4] ? 2 : 0);
}

}  // namespace

class CudaExec {
public:
    CudaExec(phtl_handle* h, const phtl_server_config& cfg) : h_(h), cfg_(cfg) {}

    ~CudaExec()
    {
        for (int g = 0; g < kNumDtypes; ++g) {
            if (dtab_[g]) cudaFree(dtab_[g]);
            if (htab_[g]) cudaFreeHost(htab_[g]);
        }
        for (auto& s : stream_)
            if (s) cudaStreamDestroy(s);
        cudaGetLastError();
    }

    int init()
    {
        int rc = ensure_device(h_);
        if (rc != PHTL_OK) return rc;
        cudaSetDevice(h_->device);
        for (auto& s : stream_)
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return cuda_rc(cudaErrorUnknown);
        const size_t tb = sizeof(JobDesc) * static_cast<size_t>(cfg_.max_active);
        for (int g = 0; g < kNumDtypes; ++g) {
            if (cudaMalloc(reinterpret_cast<void**>(&dtab_[g]), tb) != cudaSuccess) return cuda_rc(cudaErrorMemoryAllocation);
            if (cudaMallocHost(reinterpret_cast<void**>(&htab_[g]), tb) != cudaSuccess) return cuda_rc(cudaErrorMemoryAllocation);
            phtl_tuning t;
            rc = autotune(h_, g, PHTL_LEAPFROG, 4000000, target_ms_, &t);
            if (rc != PHTL_OK) return rc;
            block_[g] = cfg_.block_threads > 0 ? cfg_.block_threads : t.block_threads;
            rate_[g] = t.particle_turns_per_s;
            log_line("server dtype=%d block=%d probe=%.3e particle-turns/s", g, block_[g], rate_[g]);
        }
        if (cfg_.target_round_ms > 0) target_ms_ = cfg_.target_round_ms;
        return PHTL_OK;
    }

    int64_t bytes_for(const phtl_request& r) const
    {
        const int64_t mon = r.mon_rows ? (r.turns / std::max<int64_t>(r.mon_stride, 1) + 1) * PHTL_MON_FIELDS * 8 : 0;
        return ncoords(r) * coord_bytes(r) + mon;
    }

    int prepare(sched::Job& j)
    {
        cudaSetDevice(h_->device);
        const phtl_request& r = j.req;
        DevJob* dj = static_cast<DevJob*>(j.exec_state);
        const int si = r.dtype == PHTL_F64 ? 0 : 1;
        cudaStream_t s = stream_[si];
        if (!dj) {
            dj = new (std::nothrow) DevJob();
            if (!dj) return PHTL_E_NOMEM;
            j.exec_state = dj;
            dj->stream = si;
            const size_t cb = static_cast<size_t>(coord_bytes(r));
            for (int c = 0; c < 6 && r.n > 0; ++c) {
                if (!r.in[c]) continue;
                int rc = cuda_rc(cudaMallocAsync(&dj->d[c], cb, s));
                if (rc != PHTL_OK) return rc;
                rc = cuda_rc(cudaMemcpyAsync(dj->d[c], r.in[c], cb, cudaMemcpyHostToDevice, s));
                if (rc != PHTL_OK) return rc;
            }
        }
        if (dj->mon) {
            cudaFreeAsync(dj->mon, s);
            dj->mon = nullptr;
        }
        if (r.mon_rows) {
            dj->mon_rows = r.turns / r.mon_stride + 1;
            const size_t mb = static_cast<size_t>(dj->mon_rows) * PHTL_MON_FIELDS * 8;
            int rc = cuda_rc(cudaMallocAsync(reinterpret_cast<void**>(&dj->mon), mb, s));
            if (rc != PHTL_OK) return rc;
            rc = cuda_rc(cudaMemsetAsync(dj->mon, 0, mb, s));
            if (rc != PHTL_OK) return rc;
        }
        return cuda_rc(cudaStreamSynchronize(s));
    }

    // The configured number of resident waves of the batched kernel of this arithmetic, in
    // particles.  Default 8: on the 64-job trace, 2 / 4 / 8 / 16 waves gave the same throughput
    // (within 2 %) and p50 latencies of 6.8 / 6.1 / 5.6 / 5.1 s (FP64 and FP32C jobs) and
    // 1.49 / 0.75 / 0.80 / 1.17 s (every job FP32C).
    int64_t saturation(int dtype) const
    {
        const int g = dtype < 0 || dtype >= kNumDtypes ? 0 : dtype;
        const int occ = std::max(1, occupancy_batched(g, true, block_[g], h_->mc[0].general != 0));
        const int64_t waves = cfg_.waves > 0 ? cfg_.waves : 8;
        return waves * occ * h_->nsm * block_[g] * particles_per_thread(g);
    }

    void adopt(sched::Job& to, sched::Job& from)
    {
        to.exec_state = from.exec_state;
        from.exec_state = nullptr;
    }

    int run_round(std::vector<sched::Job*>& act, std::vector<int64_t>& nt, int64_t* launches)
    {
        cudaSetDevice(h_->device);
        int64_t nl = 0;
        bool used[2] = {false, false};
        for (int g = 0; g < kNumDtypes; ++g) {
            std::vector<size_t> idx;
            int64_t active = 0;
            for (size_t i = 0; i < act.size(); ++i)
                if (act[i]->req.dtype == g && act[i]->req.turns > act[i]->turns_done) {
                    idx.push_back(i);
                    active += act[i]->req.n;
                }
            if (idx.empty()) continue;
            std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
                return act[a]->req.turns - act[a]->turns_done > act[b]->req.turns - act[b]->turns_done;
            });
            const int64_t chunk_cfg = g == PHTL_F64 ? cfg_.chunk_turns_f64 : cfg_.chunk_turns_f32;
            int64_t T = chunk_cfg;
            if (T <= 0) {
                const double t = rate_[g] * target_ms_ * 1e-3 / std::max<double>(1.0, static_cast<double>(active));
                T = static_cast<int64_t>(std::min(std::max(t, 8.0), 65536.0));
            }
            const int block = block_[g];
            const int64_t per_tile = static_cast<int64_t>(block) * particles_per_thread(g);
            int64_t tiles = 0;
            bool rk4 = false;
            for (size_t k = 0; k < idx.size(); ++k) {
                const sched::Job& j = *act[idx[k]];
                const DevJob* dj = static_cast<const DevJob*>(j.exec_state);
                JobDesc& J = htab_[g][k];
                std::memset(&J, 0, sizeof(J));
                bool vec = true;
                for (int c = 0; c < 6; ++c) {
                    J.c[c] = dj->d[c];
                    if (dj->d[c] && reinterpret_cast<uintptr_t>(dj->d[c]) % 16) vec = false;
                }
                if (g != PHTL_F64 && (j.req.n * 4) % 16) vec = false;
                J.vec = vec ? 1 : 0;
                J.mon = dj->mon;
                J.stride = j.req.mon_rows ? j.req.mon_stride : 1;
                J.n = j.req.n;
                J.turns = j.req.turns - j.turns_done;
                J.turn_offset = j.turns_done;
                J.tile_begin = tiles;
                J.scheme = j.req.integrator;
                job_weights(h_, J.scheme, j.req.voltage_V, J);
                rk4 = rk4 || J.scheme == PHTL_RK4;
                tiles += (j.req.n + per_tile - 1) / per_tile;
                nt[idx[k]] = std::min<int64_t>(T, J.turns);
            }
            const int si = g == PHTL_F64 ? 0 : 1;
            cudaStream_t s = stream_[si];
            int rc = cuda_rc(cudaMemcpyAsync(dtab_[g], htab_[g], sizeof(JobDesc) * idx.size(),
                                             cudaMemcpyHostToDevice, s));
            if (rc != PHTL_OK) return rc;
            if (tiles > 0) {
                rc = cuda_rc(launch_batched(dtab_[g], static_cast<int32_t>(idx.size()), batch_consts(h_, rk4), g,
                                            true, 0, static_cast<int32_t>(T), static_cast<int>(tiles), block, s));
                if (rc != PHTL_OK) return rc;
                ++nl;
            }
            used[si] = true;
        }
        for (int si = 0; si < 2; ++si)
            if (used[si]) {
                int rc = cuda_rc(cudaStreamSynchronize(stream_[si]));
                if (rc != PHTL_OK) return rc;
            }
        // jobs that were already complete (turns == 0) advance by nothing
        *launches = nl;
        h_->stats.launches += nl;
        return PHTL_OK;
    }

    int finish(sched::Job& j)
    {
        cudaSetDevice(h_->device);
        const phtl_request& r = j.req;
        DevJob* dj = static_cast<DevJob*>(j.exec_state);
        if (!dj) return PHTL_E_CUDA;
        cudaStream_t s = stream_[dj->stream];
        const size_t cb = static_cast<size_t>(coord_bytes(r));
        for (int c = 0; c < 6 && r.n > 0; ++c)
            if (dj->d[c] && r.out[c]) {
                int rc = cuda_rc(cudaMemcpyAsync(r.out[c], dj->d[c], cb, cudaMemcpyDeviceToHost, s));
                if (rc != PHTL_OK) return rc;
            }
        if (r.mon_rows && dj->mon) {
            int rc = cuda_rc(cudaMemcpyAsync(r.mon_rows, dj->mon,
                                             static_cast<size_t>(dj->mon_rows) * PHTL_MON_FIELDS * 8,
                                             cudaMemcpyDeviceToHost, s));
            if (rc != PHTL_OK) return rc;
        }
        int rc = cuda_rc(cudaStreamSynchronize(s));
        h_->stats.particle_turns += r.n * r.turns;
        ++h_->stats.calls;
        if (!r.keep_resident) discard(j);
        return rc;
    }

    void discard(sched::Job& j)
    {
        DevJob* dj = static_cast<DevJob*>(j.exec_state);
        if (!dj) return;
        cudaSetDevice(h_->device);
        cudaStream_t s = stream_[dj->stream];
        for (auto& p : dj->d)
            if (p) cudaFreeAsync(p, s);
        if (dj->mon) cudaFreeAsync(dj->mon, s);
        cudaStreamSynchronize(s);
        cudaGetLastError();
        delete dj;
        j.exec_state = nullptr;
    }

private:
    phtl_handle* h_;
    phtl_server_config cfg_;
    cudaStream_t stream_[2] = {nullptr, nullptr};
    JobDesc* dtab_[kNumDtypes] = {};
    JobDesc* htab_[kNumDtypes] = {};
    int block_[kNumDtypes] = {128, 128, 128, 128};
    double rate_[kNumDtypes] = {1e10, 1e11, 1e11, 1e11};
    double target_ms_ = 20.0;
};

struct Server {
    CudaExec exec;
    sched::Scheduler<CudaExec> sched;
    Server(phtl_handle* h, const phtl_server_config& cfg) : exec(h, cfg), sched(exec, cfg) {}
};

void stop_server(phtl_handle* h)
{
    if (h->server) {
        h->server->sched.stop();
        delete h->server;
        h->server = nullptr;
    }
}

namespace {

int check_request(const phtl_handle* h, const phtl_request* r)
{
    if (!r) return PHTL_E_INVALID;
    if (r->integrator < PHTL_EULER_CROMER || r->integrator > PHTL_RK4) return PHTL_E_INVALID;
    if (r->dtype < PHTL_F64 || r->dtype > PHTL_F32CS) return PHTL_E_INVALID;
    if (r->n < 0 || r->turns < 0 || !std::isfinite(r->voltage_V)) return PHTL_E_INVALID;
    if (r->n > 0) {
        if (!r->out[0] || !r->out[1]) return PHTL_E_INVALID;
        if (!r->resume_ticket && (!r->in[0] || !r->in[1])) return PHTL_E_INVALID;
    }
    for (int p = 2; p < 6; p += 2) {
        const bool in_pair = r->in[p] != nullptr;
        if (in_pair != (r->in[p + 1] != nullptr)) return PHTL_E_INVALID;
        if ((r->out[p] != nullptr) != (r->out[p + 1] != nullptr)) return PHTL_E_INVALID;
        if (!r->resume_ticket && in_pair != (r->out[p] != nullptr)) return PHTL_E_INVALID;
    }
    if (r->mon_rows && r->mon_stride < 1) return PHTL_E_INVALID;
    if (voltage_check(h, r->voltage_V) != PHTL_OK) return PHTL_E_UNSTABLE;
    return PHTL_OK;
}

}  // namespace
}  // namespace phtl

using namespace phtl;

extern "C" {

int phtl_server_start(phtl_handle* h, const phtl_server_config* cfg)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (h->server) return PHTL_E_INVALID;
    phtl_server_config c{};
    if (cfg) c = *cfg;
    if (c.policy != PHTL_POLICY_SRPT && c.policy != PHTL_POLICY_SHARE) return PHTL_E_INVALID;
    if (c.memory_budget_bytes < 0 || c.max_active < 0 || c.chunk_turns_f64 < 0 || c.chunk_turns_f32 < 0 ||
        c.target_round_ms < 0 || c.waves < 0 || (c.block_threads != 0 && (c.block_threads < 32 || c.block_threads > 256 || c.block_threads % 32)))
        return PHTL_E_INVALID;
    if (c.memory_budget_bytes == 0) c.memory_budget_bytes = 150000000000ll;
    if (c.max_active == 0) c.max_active = 64;
    Server* s = new (std::nothrow) Server(h, c);
    if (!s) return PHTL_E_NOMEM;
    int rc = s->exec.init();
    if (rc != PHTL_OK) {
        delete s;
        return rc;
    }
    h->server = s;
    s->sched.start();
    return PHTL_OK;
}

int phtl_submit(phtl_handle* h, const phtl_request* r, uint64_t* ticket)
{
    if (!handle_valid(h) || !h->server) return PHTL_E_BADHANDLE;
    if (!ticket) return PHTL_E_INVALID;
    int rc = check_request(h, r);
    if (rc != PHTL_OK) return rc;
    return h->server->sched.submit(*r, ticket);
}

int phtl_poll(phtl_handle* h, uint64_t ticket, phtl_status* out)
{
    if (!handle_valid(h) || !h->server) return PHTL_E_BADHANDLE;
    if (!out) return PHTL_E_INVALID;
    return h->server->sched.poll(ticket, out);
}

int phtl_wait(phtl_handle* h, uint64_t ticket, int64_t timeout_ms, phtl_status* out)
{
    if (!handle_valid(h) || !h->server) return PHTL_E_BADHANDLE;
    if (!out) return PHTL_E_INVALID;
    return h->server->sched.wait(ticket, timeout_ms, out);
}

int phtl_cancel(phtl_handle* h, uint64_t ticket)
{
    if (!handle_valid(h) || !h->server) return PHTL_E_BADHANDLE;
    return h->server->sched.cancel(ticket);
}

int phtl_release(phtl_handle* h, uint64_t ticket)
{
    if (!handle_valid(h) || !h->server) return PHTL_E_BADHANDLE;
    return h->server->sched.release(ticket);
}

int phtl_server_get_stats(phtl_handle* h, phtl_server_stats* out)
{
    if (!handle_valid(h) || !h->server) return PHTL_E_BADHANDLE;
    if (!out) return PHTL_E_INVALID;
    return h->server->sched.stats(out);
}

int phtl_server_stop(phtl_handle* h)
{
    if (!handle_valid(h) || !h->server) return PHTL_E_BADHANDLE;
    stop_server(h);
    return PHTL_OK;
}

}  // extern "C"
