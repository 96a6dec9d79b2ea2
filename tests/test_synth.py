"""The seeded input generator (no GPU): SplitMix64 against its published reference
outputs, determinism, and the workload recipes' properties (truncation, separatrix,
matching, halo split, batch and trace statistics)."""
import math

import numpy as np

import oracle
from paper_1610_05801_gb300 import synth


def _bucket(V=2e6):
    d = oracle.derive(synth.ring(V))
    return d, synth.Bucket(k=d.k, A=d.A, etaC=d.etaC, Qs=d.Qs, betagamma=d.betagamma)


def test_splitmix64_reference_outputs():
    # published outputs of the SplitMix64 reference generator (Steele, Lea & Flood 2014)
    assert [int(x) for x in synth.splitmix64(0, 1)] == [0xE220A8397B1DCDAF]
    assert [int(x) for x in synth.splitmix64(1234567, 3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]
    # offsets continue the same stream
    s = synth.Stream(1234567)
    assert list(s.u64(2)) + list(s.u64(1)) == list(synth.splitmix64(1234567, 3))


def test_uniform_and_normal_statistics():
    s = synth.Stream(42)
    u = s.uniform(200000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 3e-3
    g = synth.Stream(43).normal(200001)
    assert g.shape == (200001,)
    assert abs(g.mean()) < 1e-2 and abs(g.std() - 1.0) < 1e-2
    assert abs(np.mean(g ** 4) - 3.0) < 0.05  # Gaussian kurtosis


def test_matched_bunch_recipe():
    d, b = _bucket()
    z, dp, rejected = synth.matched_bunch(0, 50000, b, sigma_z=0.15)
    assert z.shape == dp.shape == (50000,)
    assert np.max(np.abs(z)) <= 0.8 * math.pi / d.k
    assert np.all(b.contour(z, dp) <= b.contour_at_amplitude(1.0))
    # linear matching: sigma_dp / sigma_z = 2 pi Qs / (eta C) (before truncation)
    ratio = dp.std() / z.std()
    assert abs(ratio / (2 * math.pi * d.Qs / d.etaC) - 1) < 0.1
    z2, dp2, _ = synth.matched_bunch(0, 50000, b, sigma_z=0.15)
    assert np.array_equal(z, z2) and np.array_equal(dp, dp2)  # deterministic
    assert b.half_length == math.pi / d.k


def test_halo_bunch_recipe():
    d, b = _bucket()
    z, dp = synth.halo_bunch(2, 40000, b)
    H = b.contour(z, dp)
    # the core is kept inside the separatrix, the uniform halo inside 98 % of it
    assert np.all(H <= b.contour_at_amplitude(1.0))
    zc, dc, _ = synth.matched_bunch(2, 40000, b)
    Hc = b.contour(zc, dc)
    lim = b.contour_at_amplitude(0.8)
    outer, outer_core = np.mean(H > lim), np.mean(Hc > lim)
    # the 40 % halo puts far more particles between 80 % and 98 % than the Gaussian core
    assert outer > 0.03 and outer > 20 * outer_core
    assert np.sum(H > b.contour_at_amplitude(0.98)) <= np.sum(Hc > b.contour_at_amplitude(0.98))
    # interleaved: the first 10 % has the same outer fraction within noise
    assert abs(np.mean(H[:4000] > lim) - outer) < 0.015


def test_batched_jobs_recipe():
    jobs = synth.batched_jobs()
    assert len(jobs) == 64
    n = np.array([j["n"] for j in jobs])
    assert n.min() >= 1000 and n.max() <= 4_000_000
    assert 4e7 < n.sum() <= 6.1e7
    assert all(1e6 <= j["voltage_V"] <= 6e6 for j in jobs)
    assert all(1000 <= j["turns"] <= 100000 for j in jobs)


def test_serving_trace_recipe():
    tr = synth.serving_trace(count=2000)
    t = np.array([j["t_arrive_s"] for j in tr])
    assert np.all(np.diff(t) > 0)
    assert abs(len(t) / t[-1] / 200.0 - 1) < 0.1           # Poisson rate 200/s
    assert {j["integrator"] for j in tr} == {0, 1, 2}
    assert abs(np.mean([j["dtype"] for j in tr]) - 0.5) < 0.05
    n = np.array([j["n"] for j in tr])
    assert n.min() >= 1e4 and n.max() <= 8e6
    # log-uniform: the median is near the geometric mean of the bounds
    assert abs(math.log(np.median(n)) - 0.5 * math.log(1e4 * 8e6)) < 0.3
