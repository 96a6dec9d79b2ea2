"""GPU parity of the ramp programme (accelerating bucket: per-turn reference momentum and
RF voltage) against the oracle.

The reading (stated in phtl.h at phtl_set_programme and in the oracle): turn n runs the
scheme's stages with eta_n C, A_n and phi_s,n from the programme, then the transverse
rotation, then delta, x' and y' are multiplied by r_n = p0[n] / p0[n+1].

Tolerances (the same derivation as the fixed machine's: per-operation rounding
differences, FMA contraction and the library's sine, grow like a tune perturbation):
  FP64        per particle <= 1e-10 of the starting bucket / transverse amplitude after
              2000 turns; moments <= 1e-9.
  FP32C/CD    per particle <= 1e-8, moments <= 1e-6 (double-float arithmetic, the stage
              weights formed per turn as double-float products).
  FP32CS      per particle <= 2e-2, moments <= 2e-3 (FP32 increments, SFU sine).
"""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl, synth  # noqa: E402
from test_parity_gpu import moment_errors  # noqa: E402

DEV = "cuda:0"
TOL = {"f64": (1e-10, 1e-9), "f32c": (1e-8, 1e-6), "f32cd": (1e-8, 1e-6), "f32cs": (2e-2, 2e-3)}
SCHEMES = ("euler_cromer", "leapfrog", "ruth4")


def programme(pa, pb, N, V0, V1=None):
    V = np.linspace(V0, V0 if V1 is None else V1, N)
    p0 = pa + (pb - pa) * np.arange(N + 1) / N
    return V, p0


def ramp_inputs(n, seed, pa=26e9, pb=None, N=2000, V0=4.5e6, V1=None, amp=0.3, **over):
    """Ring, oracle per-turn constants and a bunch well inside the starting (accelerating)
    bucket: a matched bunch of the stationary bucket scaled by `amp`.  The default ramp
    gains 2 MeV/c per turn (phi_s ~ 0.46 rad at 4.5 MV)."""
    if pb is None:
        pb = pa + 2e6 * N
    phis0 = 0.0 if 1 / 22.77 ** 2 - (938.27208816e6 / math.hypot(pa, 938.27208816e6)) ** 2 > 0 else math.pi
    ring = synth.ring(V0, transverse=True, p0_eVc=pa, phi_s_rad=phis0, **over)
    O = oracle.load()
    d = O.derive(ring)
    V, p0 = programme(pa, pb, N, V0, V1)
    tc = O.ramp_derive(ring, V, p0)
    b = synth.Bucket(k=d.k, A=d.A, etaC=d.etaC, Qs=d.Qs, betagamma=d.betagamma)
    z, dp, _ = synth.matched_bunch(seed, n, b, sigma_z=0.12, sep_frac=0.5)
    x, xp = synth.transverse_gaussian(seed + 101, n, 50.0, 2e-6, d.betagamma)
    y, yp = synth.transverse_gaussian(seed + 202, n, 50.0, 2e-6, d.betagamma)
    return dict(ring=ring, d=d, V=V, p0=p0, tc=tc, z=z * amp, dp=dp * amp, x=x, xp=xp, y=y, yp=yp)


def _dev(a, dtype):
    if dtype == "f64":
        return torch.tensor(a, dtype=torch.float64, device=DEV)
    return torch.tensor(phtl.split_f32c(a), dtype=torch.float32, device=DEV)


def _host(t, dtype):
    return t.cpu().numpy() if dtype == "f64" else phtl.join_f32c(t.cpu().numpy())


def run_gpu(inp, scheme, turn0, turns, dtype="f64", stride=None, tuning=None, splits=None):
    R = phtl.Ring(**inp["ring"])
    R.set_programme(inp["V"], inp["p0"])
    if tuning:
        R.set_tuning(**tuning)
    bufs = [_dev(inp[k], dtype) for k in ("z", "dp", "x", "xp", "y", "yp")]
    mon = None
    if stride:
        mon = torch.full((turns // stride + 1, phtl.MON_FIELDS), float("nan"),
                         dtype=torch.float64, device=DEV)
        R.set_monitor(mon, stride=stride)
    if splits:
        t = turn0
        for s in splits:
            R.track_programme(*bufs, turn0=t, turns=s, integrator=scheme, dtype=dtype)
            t += s
    else:
        R.track_programme(*bufs, turn0=turn0, turns=turns, integrator=scheme, dtype=dtype)
    torch.cuda.synchronize()
    out = [_host(b, dtype) for b in bufs]
    moms = phtl.moments_from_sums(mon.cpu().numpy()) if stride else None
    R.close()
    return out, moms


def run_ref(inp, scheme, turn0, turns, stride=None):
    r = oracle.track_ramp(inp["d"], inp["tc"], scheme, inp["z"], inp["dp"], inp["x"], inp["xp"],
                          inp["y"], inp["yp"], turn0=turn0, turns=turns, moments=bool(stride),
                          stride=stride or 1)
    return list(r[:6]), r[6]


def errors(inp, got, ref):
    d = inp["d"]
    zb = math.pi / d.k
    db = 2 * math.sqrt(abs(d.A / (d.k * d.etaC)))
    e = [np.max(np.abs(got[0] - ref[0])) / zb, np.max(np.abs(got[1] - ref[1])) / db]
    for i in (2, 4):
        amp = np.max(np.hypot(ref[i], 50.0 * ref[i + 1]))
        e += [np.max(np.abs(got[i] - ref[i])) / amp, np.max(np.abs(got[i + 1] - ref[i + 1])) * 50.0 / amp]
    return max(e)


def test_programme_table_matches_oracle_constants():
    """phi_s,n of the library's programme equals the oracle's: the synchronous particle
    (0, 0) with a test particle beside it, after the whole ramp."""
    inp = ramp_inputs(2, seed=1)
    inp["z"] = np.array([0.0, 0.02])
    inp["dp"] = np.array([0.0, 0.0])
    for k, v in (("x", 1e-3), ("xp", 2e-5), ("y", -1e-3), ("yp", 1e-5)):
        inp[k] = np.full(2, v)
    got, _ = run_gpu(inp, "leapfrog", 0, 2000)
    ref, _ = run_ref(inp, "leapfrog", 0, 2000)
    assert abs(got[0][0]) < 1e-15 and abs(got[1][0]) < 1e-18
    assert errors(inp, got, ref) < 1e-10


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("case", ["above", "below", "voltage"])
def test_ramp_f64(scheme, case):
    kw = {"above": dict(), "below": dict(pa=10e9, pb=11e9), "voltage": dict(pb=26e9, V0=2e6, V1=6e6)}[case]
    inp = ramp_inputs(4099, seed=11, **kw)
    got, mg = run_gpu(inp, scheme, 0, 2000, stride=9, tuning=dict(block_threads=64, turns_per_launch=333))
    ref, mr = run_ref(inp, scheme, 0, 2000, stride=9)
    assert errors(inp, got, ref) < TOL["f64"][0], errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < TOL["f64"][1]


@pytest.mark.parametrize("dtype", ["f32c", "f32cd", "f32cs"])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_ramp_f32(dtype, scheme):
    inp = ramp_inputs(2051, seed=13)
    got, mg = run_gpu(inp, scheme, 0, 2000, dtype=dtype, stride=10)
    ref, mr = run_ref(inp, scheme, 0, 2000, stride=10)
    assert errors(inp, got, ref) < TOL[dtype][0], errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < TOL[dtype][1]


def test_ramp_rf_linear():
    inp = ramp_inputs(257, seed=15, rf_linear=1)
    got, _ = run_gpu(inp, "ruth4", 0, 2000)
    ref, _ = run_ref(inp, "ruth4", 0, 2000)
    assert errors(inp, got, ref) < TOL["f64"][0]


@pytest.mark.parametrize("dtype", ["f64", "f32cd"])
def test_ramp_split_calls_and_launches_bitwise(dtype):
    """Turns [0, 2000) in one call, in three calls starting mid-programme, and with a
    different turns-per-launch and block size: bitwise the same particles."""
    inp = ramp_inputs(3001, seed=17)
    a, _ = run_gpu(inp, "leapfrog", 0, 2000, dtype=dtype)
    b, _ = run_gpu(inp, "leapfrog", 0, 2000, dtype=dtype, splits=[700, 1, 1299])
    c, _ = run_gpu(inp, "leapfrog", 0, 2000, dtype=dtype, tuning=dict(block_threads=32, turns_per_launch=77))
    for u, v, w in zip(a, b, c):
        assert np.array_equal(u, v) and np.array_equal(u, w)


def test_ramp_mid_programme_start():
    """Starting at turn0 = 1200 tracks the programme's turns 1200.. (not 0..)."""
    inp = ramp_inputs(1001, seed=19)
    got, mg = run_gpu(inp, "ruth4", 1200, 800, stride=50)
    ref, mr = run_ref(inp, "ruth4", 1200, 800, stride=50)
    assert errors(inp, got, ref) < TOL["f64"][0]
    assert moment_errors(inp["d"], mg, mr) < TOL["f64"][1]


@pytest.mark.parametrize("n", [1, 3, 5])
def test_ramp_ragged_small(n):
    inp = ramp_inputs(n, seed=21 + n)
    got, _ = run_gpu(inp, "euler_cromer", 0, 2000, tuning=dict(block_threads=32, turns_per_launch=500))
    ref, _ = run_ref(inp, "euler_cromer", 0, 2000)
    assert errors(inp, got, ref) < TOL["f64"][0]


def test_ramp_argument_errors():
    inp = ramp_inputs(64, seed=23, N=100)
    R = phtl.Ring(**inp["ring"])
    bufs = [_dev(inp[k], "f64") for k in ("z", "dp", "x", "xp", "y", "yp")]
    with pytest.raises(phtl.PhtlError) as e:
        R.track_programme(*bufs, turn0=0, turns=10)                 # no programme yet
    assert e.value.code == phtl.E_INVALID
    R.set_programme(inp["V"], inp["p0"])
    for kw in (dict(turn0=0, turns=101), dict(turn0=-1, turns=5), dict(turn0=95, turns=6),
               dict(turn0=0, turns=10, integrator="rk4")):
        with pytest.raises(phtl.PhtlError) as e:
            R.track_programme(*bufs, **kw)
        assert e.value.code == phtl.E_INVALID, kw
    R.track_programme(*bufs, turn0=100, turns=0)                    # empty range at the end: ok
    R.set_programme(None)
    with pytest.raises(phtl.PhtlError):
        R.track_programme(*bufs, turn0=0, turns=1)
    torch.cuda.synchronize()
    R.close()


def test_ramp_full_size_sampled():
    """1e6 particles x 300 turns in the default launch shape: a sample of 512 particles
    against the oracle; the last monitor row against the moments of the arrays."""
    n = 1_000_000
    inp = ramp_inputs(n, seed=29, N=300)
    got, mg = run_gpu(inp, "leapfrog", 0, 300, stride=100)
    idx = np.random.default_rng(7).choice(n, 512, replace=False)
    sub = dict(inp)
    for k in ("z", "dp", "x", "xp", "y", "yp"):
        sub[k] = inp[k][idx]
    ref, _ = run_ref(sub, "leapfrog", 0, 300)
    assert errors(sub, [g[idx] for g in got], ref) < TOL["f64"][0]
    full = oracle.moments(*got)
    sel = [2, 3, 7, 8, 12, 13]
    assert np.max(np.abs(mg[-1, sel] - full[sel]) / full[sel]) < 1e-9
