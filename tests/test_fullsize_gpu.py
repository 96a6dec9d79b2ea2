"""Parity at the benchmark's full size and launch configuration.

The paper-scale single bunch (1e6 particles x 1e4 turns, EC / LF / Ruth4, FP64, transverse
planes, per-turn monitors) is tracked exactly as bench.py does, then
  - sampled particles are re-tracked one by one by the oracle (the oracle cannot do all
    1e6 x 1e4 x 3 in seconds) and must agree to 1e-10 of their own amplitude (inside 90 %
    of the separatrix; 1e-8 outside it),
  - the last monitor row must equal the moments of the final particle arrays (a property
    that holds at any size).
"""
import numpy as np
import pytest

import helpers
import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import bench  # noqa: E402
from paper_1610_05801_gb300 import phtl, synth  # noqa: E402


def test_bench_workload_sampled_parity():
    wl = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    ring = synth.ring(wl["voltage"], transverse=True)
    R = phtl.Ring(**ring)
    host = bench.make_inputs(wl, R.derived(), seed=1)
    dev = torch.device("cuda:0")
    bufs = [torch.tensor(a, dtype=torch.float64, device=dev) for a in host]
    n, turns = wl["n"], wl["turns"]
    mon = torch.zeros((turns + 1, 16), dtype=torch.float64, device=dev)
    R.set_monitor(mon, stride=1)
    d = oracle.derive(ring)
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(n, 300, replace=False))
    state = [a.copy() for a in host]
    H = 0.5 * d.etaC * host[1] ** 2 + (d.A / d.k) * (1 - np.cos(d.k * host[0]))
    inside = H <= (d.A / d.k) * (1 - np.cos(0.9 * np.pi))
    for s in wl["schemes"]:
        R.track(*bufs, turns=turns, integrator=s, dtype="f64")
        torch.cuda.synchronize()
        got = [b.cpu().numpy() for b in bufs]
        ref = oracle.track(d, s, *[a[idx] for a in state], turns=turns)
        err = helpers.rel_errors(d, list(ref[:6]), [g[idx] for g in got], state[0][idx], state[1][idx])
        ins = inside[idx]
        assert np.max(err[ins]) < 1e-10, (s, np.max(err[ins]))
        if (~ins).any():
            assert np.max(err[~ins]) < 1e-8, (s, np.max(err[~ins]))
        # last monitor row = moments of the final arrays
        m_last = phtl.moments_from_sums(mon[turns].cpu().numpy())
        m_arr = oracle.moments(*got)
        for j in (2, 3, 7, 8, 12, 13):
            assert abs(m_last[j] / m_arr[j] - 1) < 1e-9, (s, j)
        for j in (4, 9, 14):
            assert abs(m_last[j] / m_arr[j] - 1) < 1e-7, (s, j)
        assert mon[turns, 0].item() == n
        state = got  # the next scheme continues from here; contours are (nearly) invariant
    R.close()
