"""Batched launch (job table, LPT tiles, graph capture, autotuner) on the GPU.

Result independence: a bunch tracked inside a batch gives bitwise the same particles as
the same bunch tracked alone by phtl_track; monitor moments agree to the FP64 rounding
of the (order-dependent) atomic sums.
"""
import math

import numpy as np
import pytest

import helpers
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl, synth  # noqa: E402

DEV = "cuda:0"

JOBS = [  # n, turns, voltage, integrator, dtype, monitor stride (0 = none), transverse
    (1001, 700, 2.0e6, "leapfrog", "f64", 5, True),
    (37, 1500, 4.5e6, "euler_cromer", "f64", 0, False),
    (5000, 300, 3.0e6, "ruth4", "f64", 1, True),
    (2048, 2000, 1.0e6, "leapfrog", "f32c", 10, False),
    (777, 123, 6.0e6, "ruth4", "f32cd", 3, True),
    (0, 10, 2.0e6, "euler_cromer", "f32c", 1, False),
    (10, 0, 2.0e6, "leapfrog", "f64", 1, False),
    (4099, 64, 5.0e6, "euler_cromer", "f32c", 0, True),
    (1500, 900, 3.5e6, "leapfrog", "f32cs", 2, True),
]


def _bufs(n, seed, dtype, transverse, voltage):
    inp = helpers.inputs(max(n, 1), seed=seed, voltage=voltage, transverse=True)
    keys = ("z", "dp", "x", "xp", "y", "yp") if transverse else ("z", "dp")
    out = []
    for k in keys:
        a = inp[k][:n]
        if dtype == "f64":
            out.append(torch.tensor(a, dtype=torch.float64, device=DEV))
        else:
            out.append(torch.tensor(phtl.split_f32c(a), dtype=torch.float32, device=DEV))
    while len(out) < 6:
        out.append(None)
    return out


def _mon(turns, stride):
    if not stride:
        return None
    return torch.full((turns // stride + 1, 16), float("nan"), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_bitwise_equals_single(use_graph):
    ring = synth.ring(2e6, transverse=True)
    R = phtl.Ring(**ring)
    R.set_tuning(block_threads=64, turns_per_launch=64)
    jobs, singles = [], []
    for i, (n, turns, V, integ, dt, stride, tr) in enumerate(JOBS):
        b = _bufs(n, 100 + i, dt, tr, V)
        m = _mon(turns, stride)
        jobs.append(phtl.make_job(*b, turns=turns, voltage_V=V, integrator=integ, dtype=dt,
                                  monitor=m, stride=stride or 1))
        singles.append((n, turns, V, integ, dt, stride, [None if t is None else t.clone() for t in b],
                        _mon(turns, stride)))
    B = phtl.Batch(R, jobs, use_graph=use_graph)
    B.run()
    torch.cuda.synchronize()
    info = B.info()
    assert info.njobs == len(JOBS) and info.graph == (1 if use_graph else 0)
    assert info.launches_per_run >= 2000 // 64
    for j, (n, turns, V, integ, dt, stride, b, m) in zip(jobs, singles):
        Rs = phtl.Ring(**dict(ring, voltage_V=V))
        Rs.set_tuning(block_threads=64)
        if m is not None:
            Rs.set_monitor(m, stride=stride)
        Rs.track(*b, turns=turns, integrator=integ, dtype=dt)
        torch.cuda.synchronize()
        for u, v in zip(j["c"], b):
            if u is not None:
                assert torch.equal(u, v), (n, turns, integ, dt)
        if m is not None:
            mb = phtl.moments_from_sums(j["monitor"].cpu().numpy())
            ms = phtl.moments_from_sums(m.cpu().numpy())
            assert np.allclose(mb, ms, rtol=1e-11, atol=1e-300), (n, turns, integ, dt)
        Rs.close()
    B.close()
    R.close()


def test_batch_graph_replay_continues_tracking():
    ring = synth.ring(4.5e6, transverse=True)
    R = phtl.Ring(**ring)
    R.set_tuning(block_threads=128, turns_per_launch=100)
    b1 = _bufs(3000, 7, "f64", True, 4.5e6)
    b2 = _bufs(1000, 8, "f32c", False, 4.5e6)
    ref1 = [None if t is None else t.clone() for t in b1]
    ref2 = [None if t is None else t.clone() for t in b2]
    B = phtl.Batch(R, [phtl.make_job(*b1, turns=250, integrator="ruth4", dtype="f64"),
                       phtl.make_job(*b2, turns=400, integrator="leapfrog", dtype="f32c")])
    B.run()
    B.run()
    R.track(*ref1, turns=500, integrator="ruth4", dtype="f64")
    R.track(*ref2, turns=800, integrator="leapfrog", dtype="f32c")
    torch.cuda.synchronize()
    for u, v in zip(b1 + b2, ref1 + ref2):
        if u is not None:
            assert torch.equal(u, v)
    B.close()
    R.close()


def test_batch_f64_against_oracle():
    ring = synth.ring(4.5e6, transverse=True)
    R = phtl.Ring(**ring)
    specs = [(513, 900, 2e6, "leapfrog"), (250, 1200, 5.5e6, "ruth4"), (999, 333, 1e6, "euler_cromer")]
    jobs, inputs = [], []
    for i, (n, turns, V, integ) in enumerate(specs):
        inp = helpers.inputs(n, seed=40 + i, voltage=V)
        b = [torch.tensor(inp[k], dtype=torch.float64, device=DEV) for k in ("z", "dp", "x", "xp", "y", "yp")]
        jobs.append(phtl.make_job(*b, turns=turns, voltage_V=V, integrator=integ, dtype="f64"))
        inputs.append(inp)
    B = phtl.Batch(R, jobs)
    B.run()
    torch.cuda.synchronize()
    for (n, turns, V, integ), j, inp in zip(specs, jobs, inputs):
        ref = oracle.track(inp["d"], integ, inp["z"], inp["dp"], inp["x"], inp["xp"], inp["y"],
                           inp["yp"], turns=turns)
        got = [t.cpu().numpy() for t in j["c"]]
        err = helpers.rel_errors(inp["d"], list(ref[:6]), got, inp["z"], inp["dp"])
        assert np.max(err) < 1e-10, (integ, np.max(err))
    B.close()
    R.close()


def test_autotuner_picks_a_valid_shape():
    R = phtl.Ring(**synth.ring(2e6))
    for dt, integ in (("f64", "leapfrog"), ("f32c", "leapfrog"), ("f32cd", "ruth4"),
                      ("f32cs", "euler_cromer")):
        t = R.autotune(dt, integ, active_particles=2_000_000, target_launch_ms=20.0)
        assert t.block_threads in (64, 96, 128, 192, 256)  # the autotuner's candidates
        assert 8 <= t.turns_per_launch <= 1 << 20
        assert t.particle_turns_per_s > 1e9
        # the chosen launch should last roughly the target
        est_ms = 2e6 * t.turns_per_launch / t.particle_turns_per_s * 1e3
        assert 5.0 < est_ms < 80.0 or t.turns_per_launch == 8
    R.close()


def test_autotuned_batch_with_odd_sizes():
    """Regression: the autotuner's probe must keep its scratch buffers 16-byte aligned for
    the 128-bit loads even when the batch has an odd particle count (513 here)."""
    ring = synth.ring(2e6, transverse=True)
    R = phtl.Ring(**ring)  # no tuning set: phtl_batch_create runs the autotuner per group
    specs = [(513, 250, 6.0e6, "euler_cromer", "f32cd", 0, True),
             (1001, 300, 2.0e6, "leapfrog", "f32c", 3, False),
             (7, 400, 1.0e6, "ruth4", "f64", 0, False)]
    jobs, refs = [], []
    for i, (n, turns, V, integ, dt, stride, tr) in enumerate(specs):
        b = _bufs(n, 500 + i, dt, tr, V)
        jobs.append(phtl.make_job(*b, turns=turns, voltage_V=V, integrator=integ, dtype=dt,
                                  monitor=_mon(turns, stride), stride=stride or 1))
        refs.append((V, integ, dt, turns, [None if t is None else t.clone() for t in b]))
    B = phtl.Batch(R, jobs)
    info = B.info()
    assert all(b in (0, 64, 96, 128, 192, 256) for b in info.block_threads) and len(info.block_threads) == 4
    B.run()
    torch.cuda.synchronize()
    for j, (V, integ, dt, turns, b) in zip(jobs, refs):
        Rs = phtl.Ring(**dict(ring, voltage_V=V))
        Rs.track(*b, turns=turns, integrator=integ, dtype=dt)
        torch.cuda.synchronize()
        for u, v in zip(j["c"], b):
            if u is not None:
                assert torch.equal(u, v)
        Rs.close()
    B.close()
    R.close()
