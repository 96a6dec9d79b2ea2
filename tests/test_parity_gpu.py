"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs.

Tolerances (from the arithmetic: per-operation rounding differences -- FMA contraction,
the library's sine within a few ulp -- act like a tune perturbation of ~1e-15):
  FP64 path  : per-particle relative error <= 1e-10 after up to 1e4 turns for particles
               inside 90 % of the separatrix (error relative to the particle's own
               amplitude, see helpers.py); monitor moments <= 1e-9 relative.
  FP32C/FP32CD (double-float): per-particle <= 1e-8 after 1e4 turns, moments <= 1e-6
               (their monitor sums are FP32 partials).
  FP32CS (SFU sine): moments <= 1e-5 after 1e4 turns, per-particle <= 1e-2.
"""
import math

import numpy as np
import pytest

import helpers
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl  # noqa: E402

SCHEMES = ("euler_cromer", "leapfrog", "ruth4")
DEV = "cuda:0"


def _dev(a, dtype="f64"):
    if a is None:
        return None
    if dtype == "f64":
        return torch.tensor(a, dtype=torch.float64, device=DEV)
    return torch.tensor(phtl.split_f32c(a), dtype=torch.float32, device=DEV)


def _host(t, dtype="f64"):
    if t is None:
        return None
    a = t.cpu().numpy()
    return a if dtype == "f64" else phtl.join_f32c(a)


def run_gpu(inp, scheme, turns, dtype="f64", transverse=True, stride=None, tuning=None,
            perturn=False, offset=0):
    """Track inp's particles on the GPU; returns (coords, moments or None)."""
    keys = ("z", "dp", "x", "xp", "y", "yp") if transverse else ("z", "dp")
    R = phtl.Ring(**inp["ring"])
    if tuning:
        R.set_tuning(**tuning)
    bufs = []
    for k in keys:
        a = inp[k]
        if offset:
            # place the data at an element offset inside a larger allocation (misaligned)
            base = _dev(np.concatenate([np.zeros(offset), a]), dtype) if dtype == "f64" else None
            if base is None:
                raise ValueError("offset only for f64")
            bufs.append(base[offset:])
        else:
            bufs.append(_dev(a, dtype))
    while len(bufs) < 6:
        bufs.append(None)
    mon = None
    if stride:
        mon = torch.full((turns // stride + 1, phtl.MON_FIELDS), float("nan"),
                         dtype=torch.float64, device=DEV)
        R.set_monitor(mon, stride=stride)
    fn = R.track_perturn if perturn else R.track
    fn(*bufs, turns=turns, integrator=scheme, dtype=dtype)
    torch.cuda.synchronize()
    out = [_host(b, dtype) for b in bufs]
    moms = phtl.moments_from_sums(mon.cpu().numpy()) if stride else None
    R.close()
    return out, moms


def run_ref(inp, scheme, turns, transverse=True, stride=None):
    args = [inp["z"], inp["dp"]]
    if transverse:
        args += [inp["x"], inp["xp"], inp["y"], inp["yp"]]
    r = oracle.track(inp["d"], scheme, *args, turns=turns, moments=bool(stride),
                     stride=stride or 1)
    return list(r[:6]), r[6]


def moment_errors(d, mg, mr, with_emittance=True):
    """Relative moment errors: means relative to the corresponding rms, rms relative to
    itself, emittance relative to rms_u * rms_u' (its natural scale).  The emittance of a
    one- or two-particle bunch is zero, where the raw-sum formula
    sqrt(<u^2><u'^2> - <uu'>^2) only resolves ~sqrt(rounding): skip it there."""
    e = []
    for off in (0, 5, 10):
        if mr[0, off + 2] == 0:
            continue
        for j, ref_scale in ((0, 2), (1, 3)):
            e.append(np.abs(mg[:, off + j] - mr[:, off + j]) / mr[:, off + ref_scale])
        for j in (2, 3):
            e.append(np.abs(mg[:, off + j] - mr[:, off + j]) / mr[:, off + j])
        if with_emittance:
            e.append(np.abs(mg[:, off + 4] - mr[:, off + 4]) / (mr[:, off + 2] * mr[:, off + 3]))
    return float(np.max(np.vstack(e)))


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("transverse", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 1001, 4099])
def test_f64_small_sizes(scheme, transverse, n):
    inp = helpers.inputs(n, seed=n, transverse=transverse)
    turns = 1000
    got, mg = run_gpu(inp, scheme, turns, transverse=transverse, stride=7,
                      tuning=dict(block_threads=32, turns_per_launch=333))
    ref, mr = run_ref(inp, scheme, turns, transverse=transverse, stride=7)
    err = helpers.rel_errors(inp["d"], ref, got, inp["z"], inp["dp"])
    assert np.max(err) < 1e-10, np.max(err)
    assert mg.shape == mr.shape
    d = inp["d"]
    zb, db = math.pi / d.k, 2 * math.sqrt(d.A / (d.k * d.etaC))
    assert np.allclose(mg[:, 0], mr[:, 0], rtol=0, atol=1e-10 * zb)
    assert np.allclose(mg[:, 1], mr[:, 1], rtol=0, atol=1e-10 * db)
    if n > 1:
        assert moment_errors(inp["d"], mg, mr, with_emittance=n > 2) < 1e-9


@pytest.mark.parametrize("scheme", SCHEMES)
def test_f64_1e4_turns_inside_90pct(scheme):
    """The stated tolerance: <= 1e-10 per particle after 1e4 turns, 90 % separatrix."""
    inp = helpers.inputs(3000, seed=11, transverse=True, sep_frac=0.9, sigma_z=0.25)
    turns = 10000
    got, mg = run_gpu(inp, scheme, turns, stride=100)
    ref, mr = run_ref(inp, scheme, turns, stride=100)
    err = helpers.rel_errors(inp["d"], ref, got, inp["z"], inp["dp"])
    assert np.max(err) < 1e-10, (np.max(err), np.argmax(err))
    assert moment_errors(inp["d"], mg, mr) < 1e-9


def test_f64_grid_stride_and_launch_chunking_are_invisible():
    """Different grids, block sizes and turns-per-launch give bitwise identical particles."""
    inp = helpers.inputs(5000, seed=3)
    a, _ = run_gpu(inp, "ruth4", 500, tuning=dict(block_threads=64, turns_per_launch=37,
                                                  max_blocks=3))
    b, _ = run_gpu(inp, "ruth4", 500, tuning=dict(block_threads=256, turns_per_launch=500))
    c, _ = run_gpu(inp, "ruth4", 500)
    for u, v, w in zip(a, b, c):
        assert np.array_equal(u, v) and np.array_equal(u, w)


def test_f64_perturn_variant_equals_persistent():
    inp = helpers.inputs(2049, seed=5)
    for scheme in SCHEMES:
        a, ma = run_gpu(inp, scheme, 200, perturn=True, stride=10)
        b, mb = run_gpu(inp, scheme, 200, stride=10)
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
        # the launches differ in shape, so the monitor sums are added in different orders:
        # the moments agree to the ordering's rounding (means relative to the rms)
        assert moment_errors(inp["d"], ma, mb) < 1e-11


def test_f64_misaligned_pointers_take_the_scalar_path():
    inp = helpers.inputs(1003, seed=9)
    got, _ = run_gpu(inp, "leapfrog", 300, offset=1)
    ref, _ = run_ref(inp, "leapfrog", 300)
    err = helpers.rel_errors(inp["d"], ref, got, inp["z"], inp["dp"])
    assert np.max(err) < 1e-10


def test_zero_turns_and_empty_bunch():
    inp = helpers.inputs(64, seed=1)
    got, mg = run_gpu(inp, "leapfrog", 0, stride=1)
    assert np.array_equal(got[0], inp["z"]) and np.array_equal(got[1], inp["dp"])
    assert mg.shape == (1, 15)
    mr = oracle.moments(inp["z"], inp["dp"], inp["x"], inp["xp"], inp["y"], inp["yp"])
    assert np.allclose(mg[0], mr, rtol=1e-12, atol=1e-18)
    R = phtl.Ring(**inp["ring"])
    mon = torch.full((11, 16), float("nan"), dtype=torch.float64, device=DEV)
    R.set_monitor(mon, stride=1)
    e = torch.zeros(0, dtype=torch.float64, device=DEV)
    R.track(e, e, turns=10)
    torch.cuda.synchronize()
    assert torch.all(mon == 0)
    R.close()


def test_linear_mode_matches_closed_form():
    """rf_linear: the GPU leap-frog map equals the closed-form matrix power."""
    import pins

    r = pins.ring(rf_linear=1.0, voltage_V=4.5e6)
    tb = pins.textbook(r)
    K, eC, a = tb["K"], tb["etaC"], tb["a"]
    M = np.array([[1 - K / 2, -eC * (1 - K / 4)], [a, 1 - K / 2]])
    mu = 2.0 * math.asin(math.sqrt(K) / 2.0)
    N = 5000
    MN = (math.sin(N * mu) * M - math.sin((N - 1) * mu) * np.eye(2)) / math.sin(mu)
    ring = dict(r, harmonic=int(r["harmonic"]), rf_linear=1)
    R = phtl.Ring(**ring)
    z = torch.tensor([0.05, -0.1], dtype=torch.float64, device=DEV)
    d = torch.tensor([2e-4, 1e-4], dtype=torch.float64, device=DEV)
    R.track(z, d, turns=N, integrator="leapfrog")
    torch.cuda.synchronize()
    for i, (z0, d0) in enumerate(((0.05, 2e-4), (-0.1, 1e-4))):
        ez, ed = MN @ np.array([z0, d0])
        assert abs(z[i].item() - ez) < 1e-11 * 0.2
        assert abs(d[i].item() - ed) < 1e-11 * 2e-3
    R.close()


@pytest.mark.parametrize("dtype", ["f32c", "f32cd", "f32cs"])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_f32c_moments_and_particles(dtype, scheme):
    inp = helpers.inputs(4096 + 7, seed=21)
    turns = 10000
    got, mg = run_gpu(inp, scheme, turns, dtype=dtype, stride=100)
    ref, mr = run_ref(inp, scheme, turns, stride=100)
    err = helpers.rel_errors(inp["d"], ref, got, inp["z"], inp["dp"])
    if dtype == "f32cs":
        # the SFU sine's absolute error (~2^-21 on [-pi, pi]) acts as a small perturbation
        # of the potential, i.e. a tune shift, so phases drift apart slowly
        assert moment_errors(inp["d"], mg, mr) < 1e-5
        assert np.max(err) < 1e-2, np.max(err)
        assert np.median(err) < 1e-4, np.median(err)
    else:
        # double-float arithmetic throughout (~48 bits); the monitor sums are FP32
        assert moment_errors(inp["d"], mg, mr) < 1e-6
        assert np.max(err) < 1e-8, np.max(err)
        assert np.median(err) < 1e-10, np.median(err)


def test_f64_transverse_special_tunes():
    """frac(Q) = 0.5 (mu = pi: the three-shear form degenerates, the matrix is used) and
    frac(Q) = 0 (identity) against the oracle."""
    from paper_1610_05801_gb300 import synth

    inp = helpers.inputs(777, seed=17)
    ring = dict(synth.ring(4.5e6, transverse=True), Qx=20.5, Qy=21.0)
    d = oracle.derive(ring)
    inp = dict(inp, ring=ring, d=d)
    for scheme in SCHEMES:
        got, _ = run_gpu(inp, scheme, 1000)
        ref, _ = run_ref(inp, scheme, 1000)
        err = helpers.rel_errors(d, ref, got, inp["z"], inp["dp"])
        assert np.max(err) < 1e-10, (scheme, np.max(err))
        assert np.allclose(got[4], inp["y"], rtol=0, atol=0) and np.allclose(got[5], inp["yp"], rtol=0, atol=0)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("case", ["accelerating_phi_s_0.3", "below_transition_phi_s_pi"])
def test_f64_nonzero_phi_s(scheme, case):
    """phi_s != 0 takes the kick's general form (phase product, sine, minus sin phi_s)
    rather than the fused sin(k z) of the phi_s = 0 bucket."""
    from paper_1610_05801_gb300 import synth
    over = dict(phi_s_rad=0.3) if case.startswith("acc") else dict(p0_eVc=10e9, phi_s_rad=math.pi)
    ring = synth.ring(4.5e6, transverse=True, **over)
    d = oracle.load().derive(ring)
    n, turns = 2001, 3000
    s = synth.Stream(31)
    zb = math.pi / d.k
    db = 2 * math.sqrt(d.A / (d.k * abs(d.etaC)))
    # a box of +-10 % of the bucket around the fixed point z = dp = 0: inside the bucket
    z = (2 * s.uniform(n) - 1) * 0.1 * zb
    dp = (2 * s.uniform(n) - 1) * 0.1 * db
    x, xp = synth.transverse_gaussian(32, n, 50.0, 2e-6, d.betagamma)
    y, yp = synth.transverse_gaussian(33, n, 50.0, 2e-6, d.betagamma)
    inp = dict(ring=ring, d=d, z=z, dp=dp, x=x, xp=xp, y=y, yp=yp)
    got, mg = run_gpu(inp, scheme, turns, stride=50)
    ref, mr = run_ref(inp, scheme, turns, stride=50)
    assert np.max(np.abs(got[0] - ref[0])) < 1e-11 * zb
    assert np.max(np.abs(got[1] - ref[1])) < 1e-11 * db
    # the motion stayed bounded near the fixed point (a real bucket, not a drift away)
    assert np.max(np.abs(ref[0])) < 0.5 * zb
    assert moment_errors(d, mg, mr) < 1e-9


@pytest.mark.parametrize("dtype", ["f64", "f32cd"])
def test_grids_and_blocks_are_invisible(dtype):
    """Capped grids, odd block sizes and turns-per-launch give the same particles bitwise
    and the same moments up to the order of the FP64 block sums (the per-thread and
    per-warp partials group the same particles whatever the grid)."""
    inp = helpers.inputs(4099, seed=17)
    a, ma = run_gpu(inp, "leapfrog", 300, dtype=dtype, stride=3,
                    tuning=dict(block_threads=256, max_blocks=5))
    b, mb = run_gpu(inp, "leapfrog", 300, dtype=dtype, stride=3,
                    tuning=dict(block_threads=96, max_blocks=13, turns_per_launch=41))
    c, mc = run_gpu(inp, "leapfrog", 300, dtype=dtype, stride=3)
    for u, v, w in zip(a, b, c):
        assert np.array_equal(u, v) and np.array_equal(u, w)
    for m in (mb, mc):
        assert moment_errors(inp["d"], m, ma) < 1e-11
