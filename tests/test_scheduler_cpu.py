"""The serving scheduler's logic on the CPU, through a fake executor (tests/sched_fake.cpp)
that sleeps instead of tracking: admission order and slots, the memory budget, rounds,
cancellation, timeouts, latency percentiles, resident state and resume, and failures
injected on the host (no GPU is involved)."""
import ctypes as C
import os
import subprocess
import time

import numpy as np
import pytest

from paper_1610_05801_gb300 import phtl

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def fake(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("fake") / "libsched_fake.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-shared", "-fPIC", "-pthread",
                    f"-I{ROOT}/include", f"-I{ROOT}/paper_1610_05801_gb300/csrc",
                    os.path.join(HERE, "sched_fake.cpp"), "-o", out], check=True)
    L = C.CDLL(out)
    L.fake_start.restype = C.c_void_p
    L.fake_start.argtypes = [C.c_int64, C.c_int32, C.c_int64, C.c_double, C.c_int32, C.c_int64]
    for name, args in (("fake_submit", [C.c_void_p, C.POINTER(phtl.Request), C.POINTER(C.c_uint64)]),
                       ("fake_poll", [C.c_void_p, C.c_uint64, C.POINTER(phtl.Status)]),
                       ("fake_wait", [C.c_void_p, C.c_uint64, C.c_int64, C.POINTER(phtl.Status)]),
                       ("fake_cancel", [C.c_void_p, C.c_uint64]),
                       ("fake_release", [C.c_void_p, C.c_uint64]),
                       ("fake_stats", [C.c_void_p, C.POINTER(phtl.ServerStats)])):
        getattr(L, name).argtypes = args
        getattr(L, name).restype = C.c_int
    L.fake_stop.argtypes = [C.c_void_p]
    L.fake_stop.restype = None
    return L


class FakeServer:
    def __init__(self, L, budget=10**9, max_active=4, chunk=100, rate=1e9, policy=1, sat=10**9):
        self.L = L
        self.h = L.fake_start(budget, max_active, chunk, rate, policy, sat)
        self.keep = []

    def submit(self, n, turns, keep=False, resume=0, mon=False):
        a = np.arange(max(n, 1), dtype=np.float64)
        o = np.zeros(max(n, 1))
        r = phtl.Request()
        r.in_[0] = a.ctypes.data if not resume else None
        r.in_[1] = a.ctypes.data if not resume else None
        r.out[0] = o.ctypes.data
        r.out[1] = o.ctypes.data
        r.n, r.turns = n, turns
        r.resume_ticket = resume
        r.keep_resident = 1 if keep else 0
        if mon:
            m = np.zeros((turns + 1) * 16)
            r.mon_rows, r.mon_stride = m.ctypes.data, 1
            self.keep.append(m)
        self.keep += [a, o]
        t = C.c_uint64()
        rc = self.L.fake_submit(self.h, C.byref(r), C.byref(t))
        return rc, t.value, o

    def wait(self, t, ms=10000):
        st = phtl.Status()
        rc = self.L.fake_wait(self.h, t, ms, C.byref(st))
        return rc, st

    def poll(self, t):
        st = phtl.Status()
        assert self.L.fake_poll(self.h, t, C.byref(st)) == 0
        return st

    def stats(self):
        s = phtl.ServerStats()
        assert self.L.fake_stats(self.h, C.byref(s)) == 0
        return s

    def stop(self):
        self.L.fake_stop(self.h)


def test_fifo_admission_and_slots(fake):
    S = FakeServer(fake, max_active=2, chunk=50, rate=2e7)
    tickets = [S.submit(1000, 200)[1] for _ in range(6)]
    for t in tickets:
        rc, st = S.wait(t)
        assert rc == 0 and st.state == phtl.DONE and st.turns_done == 200
    admits = [S.poll(t).t_admit_ns for t in tickets]
    assert admits == sorted(admits)                       # first come, first served
    # at most two jobs were ever active at once: job k+2 admitted after job k finished
    for k in range(len(tickets) - 2):
        assert S.poll(tickets[k + 2]).t_admit_ns >= S.poll(tickets[k]).t_done_ns
    s = S.stats()
    assert s.completed == 6 and s.submitted == 6 and s.failed == 0
    assert 0 < s.p50_latency_s <= s.p99_latency_s and s.mean_latency_s > 0
    assert s.particle_turns == 6 * 1000 * 200 and s.throughput_pts > 0
    assert s.rounds >= 4 * 2 and s.bytes_in_use == 0
    S.stop()


def test_memory_budget_limits_concurrency(fake):
    S = FakeServer(fake, budget=16 * 1000 * 2 + 100, max_active=8, chunk=20, rate=1e7)
    ts = [S.submit(1000, 100)[1] for _ in range(5)]
    for t in ts:
        assert S.wait(t)[0] == 0
    s = S.stats()
    assert s.bytes_peak <= 16 * 1000 * 2 + 100
    assert s.bytes_peak >= 16 * 1000 * 2  # two jobs fit, three do not
    rc, _, _ = S.submit(10**6, 10)       # larger than the whole budget
    assert rc == phtl.E_NOMEM
    S.stop()


def test_cancel_queued_and_running(fake):
    S = FakeServer(fake, max_active=1, chunk=10, rate=1e6)
    _, t1, _ = S.submit(1000, 100000)     # ~100 s if left alone
    _, t2, _ = S.submit(1000, 10)
    time.sleep(0.05)
    assert S.poll(t1).state == phtl.RUNNING and S.poll(t2).state == phtl.QUEUED
    assert fake.fake_cancel(S.h, t2) == 0
    assert fake.fake_cancel(S.h, t1) == 0
    rc, st1 = S.wait(t1)
    assert rc == 0 and st1.state == phtl.CANCELLED and st1.error == phtl.E_CANCELLED
    assert st1.turns_done % 10 == 0 and st1.turns_done < 100000
    rc, st2 = S.wait(t2)
    assert st2.state == phtl.CANCELLED and st2.turns_done == 0
    assert fake.fake_cancel(S.h, t1) == phtl.E_INVALID       # already final
    assert fake.fake_cancel(S.h, 99999) == phtl.E_BADHANDLE
    assert S.stats().cancelled == 2 and S.stats().bytes_in_use == 0
    S.stop()


def test_wait_timeout(fake):
    S = FakeServer(fake, max_active=1, chunk=10, rate=1e5)
    _, t, _ = S.submit(1000, 1000)        # ~10 s
    rc, st = S.wait(t, 0)
    assert rc == phtl.E_TIMEOUT and st.state in (phtl.QUEUED, phtl.RUNNING)
    t0 = time.time()
    rc, st = S.wait(t, 100)
    assert rc == phtl.E_TIMEOUT and 0.08 < time.time() - t0 < 2.0
    fake.fake_cancel(S.h, t)
    assert S.wait(t)[0] == 0
    S.stop()


def test_resident_state_resume_and_release(fake):
    S = FakeServer(fake, budget=10**6, max_active=4, chunk=100, rate=1e9)
    rc, t1, o1 = S.submit(1000, 300, keep=True)
    assert rc == 0 and S.wait(t1)[1].state == phtl.DONE
    assert S.stats().bytes_in_use == 16000                    # still resident
    rc, t2, o2 = S.submit(1000, 200, resume=t1)
    assert rc == 0
    rc, st = S.wait(t2)
    assert st.state == phtl.DONE and st.turns_done == 200
    assert o2[0] == 300 + 200                                  # continued the same state
    assert S.stats().bytes_in_use == 0
    rc, t3, _ = S.submit(1000, 10, resume=t1)                  # state moved on: not resident
    assert rc == phtl.E_INVALID
    rc, t4, _ = S.submit(1000, 10, keep=True)
    S.wait(t4)
    assert S.stats().bytes_in_use == 16000
    assert fake.fake_release(S.h, t4) == 0
    assert S.stats().bytes_in_use == 0
    assert fake.fake_release(S.h, t4) == phtl.E_INVALID
    S.stop()


def test_injected_failures(fake):
    S = FakeServer(fake, max_active=4, chunk=10, rate=1e9)
    _, tb, _ = S.submit(666, 100)          # prepare fails
    rc, st = S.wait(tb)
    assert st.state == phtl.FAILED and st.error == phtl.E_NOMEM
    _, tr, _ = S.submit(777, 100)          # the round fails
    rc, st = S.wait(tr)
    assert st.state == phtl.FAILED and st.error == phtl.E_CUDA
    _, tok, _ = S.submit(1000, 30)         # the loop keeps serving afterwards
    assert S.wait(tok)[1].state == phtl.DONE
    s = S.stats()
    assert s.failed == 2 and s.completed == 1 and s.bytes_in_use == 0
    S.stop()


def test_stop_cancels_pending(fake):
    S = FakeServer(fake, max_active=1, chunk=10, rate=1e5)
    ts = [S.submit(1000, 10000)[1] for _ in range(3)]
    time.sleep(0.05)
    L, h = S.L, S.h
    s = phtl.ServerStats()
    L.fake_stats(h, C.byref(s))
    assert s.active == 1 and s.queued == 2
    # stop from the host while a round is in flight: everything ends CANCELLED
    st = [phtl.Status() for _ in ts]
    L.fake_stop(h)
    del st


def test_srpt_policy_finishes_short_jobs_first(fake):
    """Shortest remaining work first: with room for one job's particles per round, short jobs
    submitted after a long one still finish first, and the long (oldest) job keeps moving."""
    S = FakeServer(fake, max_active=8, chunk=50, rate=2e7, policy=0, sat=1000)
    _, tl, _ = S.submit(1000, 2000)       # long, admitted first
    shorts = [S.submit(1000, 100)[1] for _ in range(3)]
    for t in shorts + [tl]:
        assert S.wait(t)[0] == 0
    done_short = max(S.poll(t).t_done_ns for t in shorts)
    assert done_short < S.poll(tl).t_done_ns
    assert S.poll(tl).turns_done == 2000
    S.stop()
    # processor sharing: every round advances every job; the short ones still finish first,
    # but later than under SRPT relative to the long job's progress
    S2 = FakeServer(fake, max_active=8, chunk=50, rate=2e7, policy=1, sat=1000)
    _, tl2, _ = S2.submit(1000, 2000)
    sh2 = [S2.submit(1000, 100)[1] for _ in range(3)]
    for t in sh2 + [tl2]:
        assert S2.wait(t)[0] == 0
    assert S2.stats().completed == 4
    S2.stop()


def test_srpt_never_starves_the_oldest_job(fake):
    S = FakeServer(fake, max_active=8, chunk=10, rate=1e7, policy=0, sat=1000)
    _, tl, _ = S.submit(1000, 300)
    # a stream of short jobs that would always win on remaining work
    for _ in range(10):
        S.submit(1000, 20)
    time.sleep(0.05)
    assert S.poll(tl).turns_done > 0         # the oldest job advanced meanwhile
    assert S.wait(tl)[1].state == phtl.DONE
    S.stop()
