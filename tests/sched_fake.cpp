// Test double for the serving scheduler: instantiates the library's scheduler core
// (server_core.h) with a host-only executor that does no physics.  Each round "costs"
// sum(n * turns) / rate seconds of sleep; finish() copies inputs to outputs.  Failure
// injection: a job with n == 666 fails to prepare (PHTL_E_NOMEM), a round that contains
// a job with n == 777 fails (PHTL_E_CUDA).  Used only by tests/test_scheduler_cpu.py,
// which compiles it with g++; it is not part of the library.
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "server_core.h"

using phtl::sched::Job;

struct FakeExec {
    int64_t chunk = 100;
    double rate = 1e9;  // modelled particle-turns per second
    int64_t sat = 1000000000;
    int64_t saturation(int) const { return sat; }
    int64_t bytes_for(const phtl_request& r) const
    {
        const int64_t mon = r.mon_rows ? (r.turns / (r.mon_stride > 0 ? r.mon_stride : 1) + 1) * 128 : 0;
        return 16 * r.n + mon;
    }
    int prepare(Job& j)
    {
        if (j.req.n == 666) return PHTL_E_NOMEM;
        if (!j.exec_state) j.exec_state = new int64_t(0);
        return PHTL_OK;
    }
    void adopt(Job& to, Job& from)
    {
        to.exec_state = from.exec_state;
        from.exec_state = nullptr;
    }
    int run_round(std::vector<Job*>& act, std::vector<int64_t>& nt, int64_t* launches)
    {
        double work = 0;
        for (size_t i = 0; i < act.size(); ++i) {
            if (act[i]->req.n == 777) return PHTL_E_CUDA;
            const int64_t left = act[i]->req.turns - act[i]->turns_done;
            nt[i] = left < chunk ? left : chunk;
            *static_cast<int64_t*>(act[i]->exec_state) += nt[i];
            work += static_cast<double>(act[i]->req.n) * nt[i];
        }
        std::this_thread::sleep_for(std::chrono::duration<double>(work / rate));
        *launches = 1;
        return PHTL_OK;
    }
    int finish(Job& j)
    {
        if (j.req.n > 0 && j.req.in[0] && j.req.out[0])
            std::memcpy(j.req.out[0], j.req.in[0], 8 * j.req.n);
        if (j.req.out[1]) *static_cast<double*>(j.req.out[1]) = static_cast<double>(*static_cast<int64_t*>(j.exec_state));
        if (!j.req.keep_resident) discard(j);
        return PHTL_OK;
    }
    void discard(Job& j)
    {
        delete static_cast<int64_t*>(j.exec_state);
        j.exec_state = nullptr;
    }
};

struct Fake {
    FakeExec ex;
    phtl::sched::Scheduler<FakeExec> s;
    Fake(const phtl_server_config& c) : s(ex, c) {}
};

extern "C" {

void* fake_start(int64_t budget, int32_t max_active, int64_t chunk, double rate, int32_t policy,
                 int64_t sat)
{
    phtl_server_config c{};
    c.memory_budget_bytes = budget;
    c.max_active = max_active;
    c.policy = policy;
    Fake* f = new Fake(c);
    f->ex.chunk = chunk;
    f->ex.rate = rate;
    f->ex.sat = sat;
    f->s.start();
    return f;
}

int fake_submit(void* f, const phtl_request* r, uint64_t* t) { return static_cast<Fake*>(f)->s.submit(*r, t); }
int fake_poll(void* f, uint64_t t, phtl_status* o) { return static_cast<Fake*>(f)->s.poll(t, o); }
int fake_wait(void* f, uint64_t t, int64_t ms, phtl_status* o) { return static_cast<Fake*>(f)->s.wait(t, ms, o); }
int fake_cancel(void* f, uint64_t t) { return static_cast<Fake*>(f)->s.cancel(t); }
int fake_release(void* f, uint64_t t) { return static_cast<Fake*>(f)->s.release(t); }
int fake_stats(void* f, phtl_server_stats* o) { return static_cast<Fake*>(f)->s.stats(o); }
void fake_stop(void* f)
{
    Fake* p = static_cast<Fake*>(f);
    p->s.stop();
    delete p;
}

}  // extern "C"
