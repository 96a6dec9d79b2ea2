// Continuous-batching scheduler of the serving loop (host only, header-only).
//
// Requests (independent tracking jobs) are queued in arrival order and admitted while a
// slot is free and their device bytes fit under the memory budget.  Admitted jobs are
// tracked together in scheduling rounds: each round advances every active job by up to
// a chunk of turns in shared launches (the executor's business), after which finished
// jobs are retired -- outputs copied back, device memory returned -- and waiting jobs are
// admitted into the freed slots.  Particles are independent and turns sequential
// (Sec. 2.3 of the paper), so a job's result does not depend on which other jobs shared
// its rounds.
//
// The scheduler is templated on an executor that owns all device work:
//   int64_t bytes_for(const phtl_request&)         device bytes of one job
//   int  prepare(Job&)                             allocate + upload (a resumed job already
//                                                  holds its state: only its monitor)
//   void adopt(Job& to, Job& from)                 move a resident state to a resumed job
//   int64_t saturation(int dtype)                 particles of one arithmetic that keep the
//                                                  GPU busy (the SRPT policy's round size)
//   int  run_round(std::vector<Job*>&, std::vector<int64_t>& nt, int64_t* launches)
//   int  finish(Job&)                              download results; free unless resident
//   void discard(Job&)                             free the job's device state
// The library instantiates it with the CUDA executor (server.cu); the CPU tests with a
// host-only fake executor compiled from the tests directory.
#pragma once

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "phtl.h"

namespace phtl {
namespace sched {

inline int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Job {
    uint64_t ticket = 0;
    phtl_request req{};
    int state = PHTL_QUEUED;
    int error = PHTL_OK;
    int64_t turns_done = 0;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    int64_t bytes = 0;
    bool cancel = false;
    bool resident = false;       // device state kept after DONE (keep_resident)
    bool adopted = false;        // resumed from another job's resident state
    void* exec_state = nullptr;  // executor-owned
};

template <class Exec>
class Scheduler {
public:
    Scheduler(Exec& ex, const phtl_server_config& cfg) : ex_(ex), cfg_(cfg)
    {
        if (cfg_.memory_budget_bytes <= 0) cfg_.memory_budget_bytes = 150000000000ll;
        if (cfg_.max_active <= 0) cfg_.max_active = 64;
    }
    ~Scheduler() { stop(); }

    void start()
    {
        std::lock_guard<std::mutex> g(mu_);
        if (running_) return;
        stop_ = false;
        running_ = true;
        worker_ = std::thread([this] { loop(); });
    }

    // Queue a request (validated by the caller).  resume_ticket must name a DONE job whose
    // state is resident and compatible.
    int submit(const phtl_request& r, uint64_t* ticket)
    {
        std::lock_guard<std::mutex> g(mu_);
        if (!running_ || stop_) return PHTL_E_INVALID;
        if (r.resume_ticket) {
            auto it = jobs_.find(r.resume_ticket);
            if (it == jobs_.end()) return PHTL_E_BADHANDLE;
            const Job& o = it->second;
            // the planes a request carries: its inputs, or for a resumed job its outputs
            auto plane = [](const phtl_request& q, int p) {
                return (q.resume_ticket ? static_cast<const void*>(q.out[p]) : q.in[p]) != nullptr;
            };
            if (o.state != PHTL_DONE || !o.resident || o.req.n != r.n || o.req.dtype != r.dtype ||
                plane(o.req, 2) != plane(r, 2) || plane(o.req, 4) != plane(r, 4))
                return PHTL_E_INVALID;
            for (const auto& kv : jobs_)  // a state can be resumed once
                if (kv.second.req.resume_ticket == r.resume_ticket && kv.second.state <= PHTL_RUNNING)
                    return PHTL_E_INVALID;
        }
        Job j;
        j.ticket = next_++;
        j.req = r;
        j.t_submit = now_ns();
        j.bytes = ex_.bytes_for(r);
        if (j.bytes > cfg_.memory_budget_bytes) return PHTL_E_NOMEM;
        const uint64_t t = j.ticket;
        jobs_.emplace(t, j);
        queue_.push_back(t);
        ++submitted_;
        if (first_submit_ == 0) first_submit_ = j.t_submit;
        cv_.notify_all();
        *ticket = t;
        return PHTL_OK;
    }

    int poll(uint64_t t, phtl_status* out)
    {
        std::lock_guard<std::mutex> g(mu_);
        return fill(t, out);
    }

    int wait(uint64_t t, int64_t timeout_ms, phtl_status* out)
    {
        std::unique_lock<std::mutex> lk(mu_);
        auto it = jobs_.find(t);
        if (it == jobs_.end()) return PHTL_E_BADHANDLE;
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max<int64_t>(timeout_ms, 0));
        while (jobs_.at(t).state <= PHTL_RUNNING) {
            if (timeout_ms <= 0 || done_cv_.wait_until(lk, deadline) == std::cv_status::timeout) {
                if (jobs_.at(t).state <= PHTL_RUNNING) {
                    fill(t, out);
                    return PHTL_E_TIMEOUT;
                }
            }
        }
        return fill(t, out);
    }

    int cancel(uint64_t t)
    {
        std::lock_guard<std::mutex> g(mu_);
        auto it = jobs_.find(t);
        if (it == jobs_.end()) return PHTL_E_BADHANDLE;
        if (it->second.state > PHTL_RUNNING) return PHTL_E_INVALID;  // already final
        it->second.cancel = true;
        cv_.notify_all();
        return PHTL_OK;
    }

    int release(uint64_t t)
    {
        std::lock_guard<std::mutex> g(mu_);
        auto it = jobs_.find(t);
        if (it == jobs_.end()) return PHTL_E_BADHANDLE;
        Job& j = it->second;
        if (j.state != PHTL_DONE || !j.resident) return PHTL_E_INVALID;
        ex_.discard(j);
        j.resident = false;
        bytes_in_use_ -= j.bytes;
        cv_.notify_all();
        return PHTL_OK;
    }

    int stats(phtl_server_stats* s)
    {
        std::lock_guard<std::mutex> g(mu_);
        *s = phtl_server_stats{};
        s->submitted = submitted_;
        s->completed = completed_;
        s->failed = failed_;
        s->cancelled = cancelled_;
        s->queued = static_cast<int64_t>(queue_.size());
        s->active = static_cast<int64_t>(active_.size());
        s->bytes_in_use = bytes_in_use_;
        s->bytes_peak = bytes_peak_;
        s->rounds = rounds_;
        s->launches = launches_;
        s->particle_turns = particle_turns_;
        s->busy_s = busy_ns_ * 1e-9;
        if (!lat_.empty()) {
            std::vector<double> v = lat_;
            auto pct = [&](double p) {
                const size_t k = std::min(v.size() - 1, static_cast<size_t>(p * (v.size() - 1) + 0.5));
                std::nth_element(v.begin(), v.begin() + k, v.end());
                return v[k];
            };
            s->p50_latency_s = pct(0.50);
            s->p99_latency_s = pct(0.99);
            double sum = 0;
            for (double x : lat_) sum += x;
            s->mean_latency_s = sum / lat_.size();
        }
        if (last_done_ > first_submit_ && first_submit_ > 0)
            s->throughput_pts = particle_turns_ / ((last_done_ - first_submit_) * 1e-9);
        return PHTL_OK;
    }

    // Stop the worker: the current round completes, every job not yet DONE is cancelled,
    // resident states are freed.
    void stop()
    {
        {
            std::lock_guard<std::mutex> g(mu_);
            if (!running_) return;
            stop_ = true;
            cv_.notify_all();
        }
        if (worker_.joinable()) worker_.join();
        std::lock_guard<std::mutex> g(mu_);
        for (auto& kv : jobs_) {
            Job& j = kv.second;
            if (j.exec_state) ex_.discard(j);
            if (j.state <= PHTL_RUNNING) {
                j.state = PHTL_CANCELLED;
                j.error = PHTL_E_CANCELLED;
                j.t_done = now_ns();
                ++cancelled_;
            }
            j.resident = false;
        }
        queue_.clear();
        active_.clear();
        bytes_in_use_ = 0;
        running_ = false;
        done_cv_.notify_all();
    }

private:
    int fill(uint64_t t, phtl_status* out)
    {
        auto it = jobs_.find(t);
        if (it == jobs_.end()) return PHTL_E_BADHANDLE;
        const Job& j = it->second;
        out->state = j.state;
        out->error = j.error;
        out->turns_done = j.turns_done;
        out->t_submit_ns = j.t_submit;
        out->t_admit_ns = j.t_admit;
        out->t_done_ns = j.t_done;
        return PHTL_OK;
    }

    void finalize(Job& j, int state, int err)  // mu_ held
    {
        j.state = state;
        j.error = err;
        j.t_done = now_ns();
        if (state == PHTL_DONE) {
            ++completed_;
            lat_.push_back((j.t_done - j.t_submit) * 1e-9);
            particle_turns_ += static_cast<double>(j.req.n) * j.req.turns;
            last_done_ = j.t_done;
        } else if (state == PHTL_CANCELLED) {
            ++cancelled_;
        } else {
            ++failed_;
        }
        if (!(state == PHTL_DONE && j.resident)) bytes_in_use_ -= j.bytes;
        done_cv_.notify_all();
    }

    void loop()
    {
        std::vector<Job*> act;
        std::vector<int64_t> nt;
        for (;;) {
            std::vector<Job*> admitted;
            {
                std::unique_lock<std::mutex> lk(mu_);
                // cancelled jobs leave between rounds
                for (auto it = active_.begin(); it != active_.end();) {
                    Job& j = jobs_.at(*it);
                    if (j.cancel) {
                        ex_.discard(j);
                        finalize(j, PHTL_CANCELLED, PHTL_E_CANCELLED);
                        it = active_.erase(it);
                    } else {
                        ++it;
                    }
                }
                // admission, first come first served
                while (!queue_.empty() && static_cast<int>(active_.size() + admitted.size()) < cfg_.max_active) {
                    Job& j = jobs_.at(queue_.front());
                    if (j.cancel) {
                        queue_.pop_front();
                        bytes_in_use_ += j.bytes;  // finalize subtracts it
                        finalize(j, PHTL_CANCELLED, PHTL_E_CANCELLED);
                        continue;
                    }
                    const int64_t need = j.req.resume_ticket ? 0 : j.bytes;
                    if (bytes_in_use_ + need > cfg_.memory_budget_bytes) break;
                    queue_.pop_front();
                    if (j.req.resume_ticket) {
                        Job& o = jobs_.at(j.req.resume_ticket);
                        ex_.adopt(j, o);
                        o.resident = false;
                        j.adopted = true;
                        j.bytes = o.bytes;
                    } else {
                        bytes_in_use_ += j.bytes;
                    }
                    bytes_peak_ = std::max(bytes_peak_, bytes_in_use_);
                    j.state = PHTL_RUNNING;
                    j.t_admit = now_ns();
                    admitted.push_back(&j);
                }
                if (active_.empty() && admitted.empty()) {
                    if (stop_) break;
                    cv_.wait_for(lk, std::chrono::milliseconds(20));
                    continue;
                }
                if (stop_) {
                    for (Job* j : admitted) active_.push_back(j->ticket);
                    break;
                }
            }
            // uploads happen outside the lock
            for (Job* j : admitted) {
                const int rc = ex_.prepare(*j);  // upload, or (resumed) only a fresh monitor
                std::lock_guard<std::mutex> g(mu_);
                if (rc != PHTL_OK) {
                    ex_.discard(*j);
                    finalize(*j, PHTL_FAILED, rc);
                } else {
                    active_.push_back(j->ticket);
                }
            }
            {
                std::lock_guard<std::mutex> g(mu_);
                act.clear();
                for (uint64_t t : active_) act.push_back(&jobs_.at(t));
                if (cfg_.policy == PHTL_POLICY_SRPT) select_srpt(act);
            }
            if (act.empty()) continue;
            nt.assign(act.size(), 0);
            int64_t nl = 0;
            const int64_t r0 = now_ns();
            const int rc = ex_.run_round(act, nt, &nl);
            const int64_t r1 = now_ns();
            std::vector<Job*> fin;
            {
                std::lock_guard<std::mutex> g(mu_);
                ++rounds_;
                launches_ += nl;
                busy_ns_ += r1 - r0;
                for (size_t i = 0; i < act.size(); ++i) {
                    Job& j = *act[i];
                    if (rc != PHTL_OK) {
                        ex_.discard(j);
                        finalize(j, PHTL_FAILED, rc);
                        continue;
                    }
                    j.turns_done += nt[i];
                    if (j.turns_done >= j.req.turns) fin.push_back(&j);
                }
                if (rc != PHTL_OK) active_.clear();
            }
            for (Job* j : fin) {
                const int frc = ex_.finish(*j);
                std::lock_guard<std::mutex> g(mu_);
                active_.erase(std::remove(active_.begin(), active_.end(), j->ticket), active_.end());
                if (frc != PHTL_OK) {
                    ex_.discard(*j);
                    finalize(*j, PHTL_FAILED, frc);
                } else {
                    j->resident = j->req.keep_resident != 0;
                    finalize(*j, PHTL_DONE, PHTL_OK);
                }
                cv_.notify_all();
            }
        }
    }

    // Shortest remaining work first, per arithmetic: keep the jobs with the least
    // n * (turns left) until their particles reach the executor's saturation size, and
    // always the longest-admitted job of that arithmetic so no job starves.
    void select_srpt(std::vector<Job*>& act)  // mu_ held
    {
        std::vector<Job*> keep;
        for (int dt = PHTL_F64; dt <= PHTL_F32CS; ++dt) {
            std::vector<Job*> g;
            for (Job* j : act)
                if (j->req.dtype == dt) g.push_back(j);
            if (g.empty()) continue;
            auto work = [](const Job* j) {
                return static_cast<double>(j->req.n) * static_cast<double>(j->req.turns - j->turns_done);
            };
            std::stable_sort(g.begin(), g.end(), [&](Job* a, Job* b) { return work(a) < work(b); });
            Job* oldest = *std::min_element(g.begin(), g.end(), [](Job* a, Job* b) {
                return a->t_admit != b->t_admit ? a->t_admit < b->t_admit : a->ticket < b->ticket;
            });
            const int64_t sat = ex_.saturation(dt);
            int64_t cum = 0;
            bool has_oldest = false;
            for (Job* j : g) {
                if (cum > 0 && cum + j->req.n > sat) break;
                keep.push_back(j);
                cum += j->req.n;
                has_oldest = has_oldest || j == oldest;
            }
            if (!has_oldest) keep.push_back(oldest);
        }
        act.swap(keep);
    }

    Exec& ex_;
    phtl_server_config cfg_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::thread worker_;
    bool running_ = false, stop_ = false;
    uint64_t next_ = 1;
    std::unordered_map<uint64_t, Job> jobs_;
    std::deque<uint64_t> queue_;
    std::vector<uint64_t> active_;
    int64_t bytes_in_use_ = 0, bytes_peak_ = 0;
    int64_t submitted_ = 0, completed_ = 0, failed_ = 0, cancelled_ = 0;
    int64_t rounds_ = 0, launches_ = 0, busy_ns_ = 0;
    int64_t first_submit_ = 0, last_done_ = 0;
    double particle_turns_ = 0.0;
    std::vector<double> lat_;
};

}  // namespace sched
}  // namespace phtl
