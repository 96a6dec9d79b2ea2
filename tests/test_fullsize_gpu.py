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


def test_batched_workload_sampled_parity():
    """The 64-bunch batch of the batched workload (5.5e7 particles, turns 1e3-1e5, V 1-6 MV,
    leap-frog FP32C, per-bunch stride-1 monitors, one graph-captured autotuned batch) as
    bench.py builds it, one run: for 8 bunches spread over the table, 24 sampled particles
    re-tracked alone by the FP64 oracle at the bunch's voltage and turns (FP32C tolerance,
    grown with the turns: 3e-8 per 1e4 turns inside 90 % of the separatrix), and every
    bunch's last monitor row against the moments of its final arrays (FP32 partial sums)."""
    wl = bench.WORKLOADS["batched_64_bunches_f32c_lf"]
    specs = synth.batched_jobs(seed=3, nbunch=wl["nbunch"], total=wl["total"])
    ring = synth.ring(2e6)
    R = phtl.Ring(**ring)
    dev = torch.device("cuda:0")
    jobs, host, mons = [], [], []
    for sp in specs:
        der = phtl.Ring(**dict(ring, voltage_V=sp["voltage_V"])).derived()
        b = synth.Bucket(k=der.k, A=der.A, etaC=der.etaC, Qs=der.Qs, betagamma=der.betagamma)
        z, d, _ = synth.matched_bunch(sp["seed"], sp["n"], b)
        bz = torch.tensor(phtl.split_f32c(z), dtype=torch.float32, device=dev)
        bd = torch.tensor(phtl.split_f32c(d), dtype=torch.float32, device=dev)
        mon = torch.zeros((sp["turns"] + 1, 16), dtype=torch.float64, device=dev)
        jobs.append(phtl.make_job(bz, bd, turns=sp["turns"], voltage_V=sp["voltage_V"],
                                  integrator="leapfrog", dtype="f32c", monitor=mon, stride=1))
        host.append((z, d, bz, bd))
        mons.append(mon)
    B = phtl.Batch(R, jobs, use_graph=True)
    B.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(321)
    picks = np.linspace(0, len(specs) - 1, 8).astype(int)
    for j, sp in enumerate(specs):
        z0, d0, bz, bd = host[j]
        zf, df = phtl.join_f32c(bz.cpu().numpy()), phtl.join_f32c(bd.cpu().numpy())
        m_last = phtl.moments_from_sums(mons[j][sp["turns"]].cpu().numpy())
        m_arr = oracle.moments(zf, df)
        assert mons[j][sp["turns"], 0].item() == sp["n"]
        for k in (2, 3):
            assert abs(m_last[k] / m_arr[k] - 1) < 1e-6, (j, k)
        if j not in picks:
            continue
        od = oracle.derive(dict(ring, voltage_V=sp["voltage_V"]))
        idx = np.sort(rng.choice(sp["n"], min(24, sp["n"]), replace=False))
        ref = oracle.track(od, "leapfrog", z0[idx], d0[idx], turns=sp["turns"])
        err = helpers.rel_errors(od, list(ref[:6]), [zf[idx], df[idx], None, None, None, None],
                                 z0[idx], d0[idx])
        H = 0.5 * od.etaC * d0[idx] ** 2 + (od.A / od.k) * (1 - np.cos(od.k * z0[idx]))
        ins = H <= (od.A / od.k) * (1 - np.cos(0.9 * np.pi))
        tol = 3e-8 * max(1.0, sp["turns"] / 1e4)
        assert np.max(err[ins]) < tol, (j, sp["turns"], np.max(err[ins]), tol)
    B.close()
    R.close()
