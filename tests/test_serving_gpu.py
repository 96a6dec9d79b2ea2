"""The serving loop on the GPU.

Result independence: jobs of different sizes, turn counts, voltages, integrators and
arithmetic submitted together (so they share scheduling rounds and launches) give, each,
bitwise the same particles as the same job tracked alone with phtl_track, and monitor
moments equal to FP64 rounding.  Parity: every served job of the mix also agrees with the
FP64 oracle on the same inputs, within the parity tolerances of the single-bunch path
(FP64: per particle <= 1e-10, moments <= 1e-9; FP32C / FP32CD: per particle <= 1e-8 with
median <= 1e-10, moments <= 1e-6).  Also: resume from a resident state, cancellation at a
round boundary, latency statistics.
"""
import numpy as np
import pytest

import helpers
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl, synth  # noqa: E402
from test_parity_gpu import moment_errors  # noqa: E402

DEV = "cuda:0"
MIX = [  # n, turns, voltage, integrator, dtype, monitor stride, transverse
    (20000, 3000, 2.0e6, "leapfrog", "f32c", 10, False),
    (1001, 5000, 4.5e6, "ruth4", "f64", 50, True),
    (4096, 800, 1.5e6, "euler_cromer", "f32cd", 0, True),
    (50000, 2000, 6.0e6, "leapfrog", "f32c", 1, False),
    (333, 12000, 3.0e6, "euler_cromer", "f64", 0, False),
    (7000, 1500, 5.0e6, "ruth4", "f32c", 7, True),
    (12, 100, 2.0e6, "leapfrog", "f64", 1, True),
]


def host_arrays(n, seed, dtype, transverse, voltage):
    inp = helpers.inputs(n, seed=seed, voltage=voltage, transverse=True)
    keys = ("z", "dp", "x", "xp", "y", "yp") if transverse else ("z", "dp")
    out = []
    for k in keys:
        a = inp[k]
        out.append(np.ascontiguousarray(a) if dtype == "f64" else phtl.split_f32c(a))
    while len(out) < 6:
        out.append(None)
    return out


def alone(ring, arrays, turns, V, integ, dt, stride):
    R = phtl.Ring(**dict(ring, voltage_V=V))
    tt = torch.float64 if dt == "f64" else torch.float32
    bufs = [None if a is None else torch.tensor(a, dtype=tt, device=DEV) for a in arrays]
    mon = None
    if stride:
        mon = torch.zeros((turns // stride + 1, 16), dtype=torch.float64, device=DEV)
        R.set_monitor(mon, stride=stride)
    R.track(*bufs, turns=turns, integrator=integ, dtype=dt)
    torch.cuda.synchronize()
    res = [None if b is None else b.cpu().numpy() for b in bufs]
    m = None if mon is None else mon.cpu().numpy()
    R.close()
    return res, m


def oracle_check(spec, seed, out, mon):
    """A served job's particles and monitor moments against the FP64 oracle tracking the
    same initial values (the FP32 layouts are compared through hi + comp)."""
    n, turns, V, integ, dt, stride, tr = spec
    inp = helpers.inputs(n, seed=seed, voltage=V, transverse=True)
    keys = ("z", "dp", "x", "xp", "y", "yp") if tr else ("z", "dp")
    args = [inp[k] for k in keys]
    ref = oracle.track(inp["d"], integ, *args, turns=turns, moments=bool(stride),
                       stride=stride or 1)
    got = [None if a is None else (a if dt == "f64" else phtl.join_f32c(a)) for a in out]
    refp = [ref[i] if i < len(keys) else None for i in range(6)]
    err = helpers.rel_errors(inp["d"], refp, got, inp["z"], inp["dp"])
    if dt == "f64":
        assert np.max(err) < 1e-10, (spec, np.max(err))
    else:
        assert np.max(err) < 1e-8, (spec, np.max(err))
        assert np.median(err) < 1e-10, (spec, np.median(err))
    if stride and n > 1:
        mg = phtl.moments_from_sums(mon)
        tol = 1e-9 if dt == "f64" else 1e-6
        assert moment_errors(inp["d"], mg, ref[6], with_emittance=n > 2) < tol, spec


def test_results_identical_alone_and_in_the_mix():
    ring = synth.ring(2e6, transverse=True)
    R = phtl.Ring(**ring)
    S = phtl.Server(R, max_active=4, target_round_ms=5.0)  # 7 jobs, 4 slots: admission churn
    subs = []
    for i, (n, turns, V, integ, dt, stride, tr) in enumerate(MIX):
        arrs = host_arrays(n, 300 + i, dt, tr, V)
        out = [None if a is None else np.empty_like(a) for a in arrs]
        mon = np.zeros((turns // stride + 1, 16)) if stride else None
        t = S.submit(*arrs, turns=turns, voltage_V=V, integrator=integ, dtype=dt, out=out,
                     monitor=mon, stride=stride or 1)
        subs.append((t, arrs, out, mon))
    for (t, arrs, out, mon), (n, turns, V, integ, dt, stride, tr) in zip(subs, MIX):
        rc, st = S.wait(t, 120000)
        assert rc == phtl.OK and st.state == phtl.DONE and st.turns_done == turns
        ref, mref = alone(ring, arrs, turns, V, integ, dt, stride)
        for a, b in zip(out, ref):
            if a is not None:
                assert np.array_equal(a, b), (n, turns, integ, dt)
        if stride:
            ma, mb = phtl.moments_from_sums(mon), phtl.moments_from_sums(mref)
            assert np.allclose(ma, mb, rtol=1e-11, atol=1e-300), (n, integ, dt)
    # every served job against the oracle (the chain served == alone == oracle, checked
    # directly rather than through the single-bunch parity tests)
    for i, ((t, arrs, out, mon), spec) in enumerate(zip(subs, MIX)):
        oracle_check(spec, 300 + i, out, mon)
    s = S.stats()
    assert s.completed == len(MIX) and s.failed == 0 and s.bytes_in_use == 0
    assert 0 < s.p50_latency_s <= s.p99_latency_s
    assert s.rounds > 1 and s.launches >= s.rounds
    S.stop()
    R.close()


def test_resume_from_resident_state():
    ring = synth.ring(4.5e6, transverse=True)
    R = phtl.Ring(**ring)
    S = phtl.Server(R)
    arrs = host_arrays(3000, 5, "f64", True, 4.5e6)
    out1 = [np.empty_like(a) for a in arrs]
    t1 = S.submit(*arrs, turns=700, integrator="ruth4", dtype="f64", out=out1, keep_resident=True)
    assert S.wait(t1)[1].state == phtl.DONE
    assert S.stats().bytes_in_use == 6 * 8 * 3000
    out2 = [np.empty_like(a) for a in arrs]
    t2 = S.submit(turns=500, integrator="ruth4", dtype="f64", out=out2, resume=t1)
    assert S.wait(t2)[1].state == phtl.DONE
    ref, _ = alone(ring, arrs, 1200, 4.5e6, "ruth4", "f64", 0)
    for a, b in zip(out2, ref):
        assert np.array_equal(a, b)
    assert S.stats().bytes_in_use == 0
    S.stop()
    R.close()


def test_cancel_running_job():
    ring = synth.ring(2e6)
    R = phtl.Ring(**ring)
    S = phtl.Server(R, chunk_turns_f64=100)
    arrs = host_arrays(200000, 9, "f64", False, 2e6)
    t = S.submit(*arrs, turns=10**7, integrator="ruth4", dtype="f64")  # far too long
    import time
    time.sleep(0.5)
    assert S.poll(t).state == phtl.RUNNING
    assert S.cancel(t) == phtl.OK
    rc, st = S.wait(t, 30000)
    assert rc == phtl.OK and st.state == phtl.CANCELLED and 0 < st.turns_done < 10**7
    assert st.turns_done % 100 == 0
    assert S.stats().bytes_in_use == 0
    S.stop()
    R.close()


def test_submit_validation():
    R = phtl.Ring(**synth.ring(2e6))
    S = phtl.Server(R)
    a = np.zeros(10)
    with pytest.raises(phtl.PhtlError) as e:
        S.submit(a, a, turns=10, integrator=7)
    assert e.value.code == phtl.E_INVALID
    with pytest.raises(phtl.PhtlError) as e:
        S.submit(a, a, turns=10, voltage_V=-1e6)
    assert e.value.code == phtl.E_UNSTABLE
    with pytest.raises(phtl.PhtlError) as e:
        S.submit(a, a, turns=10, resume=12345)
    assert e.value.code == phtl.E_BADHANDLE
    S.stop()
    R.close()
