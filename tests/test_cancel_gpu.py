"""Cancellation of a long persistent tracking call (phtl_track_cancel / phtl_track_status).

A call is enqueued as many launches of a bounded number of turns; a one-thread gate kernel
in front of each launch reads the handle's cancel word from host-mapped memory, so a cancel
issued from the host while the call runs stops it at the next launch boundary.  Each launch
runs whole or not at all: the particles must equal, bitwise, the same bunch tracked for the
turns reported done, and those turns are a multiple of the turns per launch.  Nothing on
the GPU is made to fault or wait: the test only sets a host word between launches.
"""
import threading
import time

import numpy as np
import pytest

import helpers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl  # noqa: E402

DEV = "cuda:0"


def _bufs(inp, dtype):
    keys = ("z", "dp", "x", "xp", "y", "yp")
    if dtype == "f64":
        return [torch.tensor(inp[k], dtype=torch.float64, device=DEV) for k in keys]
    return [torch.tensor(phtl.split_f32c(inp[k]), dtype=torch.float32, device=DEV) for k in keys]


@pytest.mark.parametrize("dtype", ["f64", "f32cd"])
def test_cancel_stops_at_a_launch_boundary(dtype):
    n, tpl = 1_000_000, 2000
    turns = 200_000      # ~7 s uncancelled (EC, FP64): the cancel comes long before
    inp = helpers.inputs(n, seed=19, transverse=True)
    R = phtl.Ring(**inp["ring"])
    R.set_tuning(turns_per_launch=tpl)
    bufs = _bufs(inp, dtype)
    mon = torch.zeros((turns // 100 + 1, phtl.MON_FIELDS), dtype=torch.float64, device=DEV)
    R.set_monitor(mon, stride=100)
    stream = torch.cuda.Stream()
    R.track(*bufs, turns=turns, integrator="euler_cromer", dtype=dtype, stream=stream)
    t0 = time.perf_counter()
    time.sleep(0.5)
    R.cancel()
    stream.synchronize()
    waited = time.perf_counter() - t0
    rc, done = R.status()
    assert rc == phtl.E_CANCELLED, (rc, done)
    assert 0 < done < turns and done % tpl == 0, done
    assert waited < 10.0, waited
    # the rows of the turns that ran are filled, the rest stay zero
    rows = mon.cpu().numpy()
    assert np.all(rows[: done // 100 + 1, 0] == n)
    assert np.all(rows[done // 100 + 1:] == 0.0)
    got = [b.cpu() for b in bufs]
    R.close()
    # bitwise the same bunch tracked for `done` turns in the same launch shape
    R2 = phtl.Ring(**inp["ring"])
    R2.set_tuning(turns_per_launch=tpl)
    ref = _bufs(inp, dtype)
    R2.track(*ref, turns=done, integrator="euler_cromer", dtype=dtype)
    torch.cuda.synchronize()
    assert R2.status() == (phtl.OK, done)
    for a, b in zip(got, ref):
        assert torch.equal(a, b.cpu())
    R2.close()


def test_cancel_before_a_call_and_from_another_thread():
    inp = helpers.inputs(20_000, seed=23, transverse=False)
    R = phtl.Ring(**inp["ring"])
    z = torch.tensor(inp["z"], dtype=torch.float64, device=DEV)
    d = torch.tensor(inp["dp"], dtype=torch.float64, device=DEV)
    # a cancel with nothing enqueued does not touch later calls
    R.cancel()
    R.track(z, d, turns=500, integrator="leapfrog")
    torch.cuda.synchronize()
    assert R.status() == (phtl.OK, 500)
    # a cancel from another host thread while a long call runs
    R.set_tuning(turns_per_launch=10_000)
    stream = torch.cuda.Stream()
    R.track(z, d, turns=5_000_000, integrator="ruth4", stream=stream)
    th = threading.Thread(target=lambda: (time.sleep(0.3), R.cancel()))
    th.start()
    th.join()
    stream.synchronize()
    rc, done = R.status()
    assert rc == phtl.E_CANCELLED and 0 < done < 5_000_000 and done % 10_000 == 0
    # and the handle tracks normally afterwards
    R.track(z, d, turns=300, integrator="leapfrog")
    torch.cuda.synchronize()
    assert R.status() == (phtl.OK, 300)
    R.close()


def test_cancel_a_programme_call():
    import test_ramp_gpu as tr

    n, tpl, turns = 500_000, 1000, 200_000
    # a flat programme (constant momentum and voltage): long, and the bunch stays bunched
    inp = tr.ramp_inputs(n, seed=29, pb=26e9, N=turns)
    R = phtl.Ring(**inp["ring"])
    R.set_programme(inp["V"], inp["p0"])
    R.set_tuning(turns_per_launch=tpl)
    bufs = _bufs(inp, "f64")
    stream = torch.cuda.Stream()
    R.track_programme(*bufs, turn0=0, turns=turns, integrator="ruth4", stream=stream)
    time.sleep(0.5)
    R.cancel()
    stream.synchronize()
    rc, done = R.status()
    assert rc == phtl.E_CANCELLED and 0 < done < turns and done % tpl == 0, (rc, done)
    got = [b.cpu() for b in bufs]
    R.close()
    R2 = phtl.Ring(**inp["ring"])
    R2.set_programme(inp["V"], inp["p0"])
    R2.set_tuning(turns_per_launch=tpl)
    ref = _bufs(inp, "f64")
    R2.track_programme(*ref, turn0=0, turns=done, integrator="ruth4")
    torch.cuda.synchronize()
    assert R2.status() == (phtl.OK, done)
    for a, b in zip(got, ref):
        assert torch.equal(a, b.cpu())
    R2.close()


def test_a_call_captured_in_a_graph_has_no_gates():
    inp = helpers.inputs(50_000, seed=31, transverse=True)
    R = phtl.Ring(**inp["ring"])
    R.set_tuning(turns_per_launch=100)
    bufs = _bufs(inp, "f64")
    ref = _bufs(inp, "f64")
    R.track(*ref, turns=1, integrator="leapfrog")  # first device call: control words allocated
    torch.cuda.synchronize()
    R.track(*ref, turns=399, integrator="leapfrog")
    R.track(*ref, turns=400, integrator="leapfrog")
    torch.cuda.synchronize()
    R.track(*bufs, turns=1, integrator="leapfrog")
    torch.cuda.synchronize()
    gates0 = R.stats().gate_launches
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
        R.track(*bufs, turns=399, integrator="leapfrog", stream=side)
    assert R.stats().gate_launches == gates0  # captured without gates
    g.replay()
    R.cancel()  # a cancel does not reach the captured launches
    g.replay()
    torch.cuda.synchronize()
    # 1 + 399 + 399 turns against 1 + 399 + 400: compare with one more turn on the graph side
    R.track(*bufs, turns=1, integrator="leapfrog")
    torch.cuda.synchronize()
    for a, b in zip(bufs, ref):
        assert torch.equal(a, b)
    R.close()
