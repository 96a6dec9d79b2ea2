"""GPU parity of the collective step (uniform slicing, wake potential, wake kick) against
the oracle: one step on identical inputs, and turns of map + collective step.

The reading (phtl.h at phtl_set_wake, and the oracle): after each turn's map the particles
are counted on nslices uniform slices of [z_lo, z_hi), V_k = sum_{j >= k} c_j w[j - k],
D_k the central difference of the counts (space charge), and delta += alpha V_k +
alpha_sc D_k of the particle's own slice.

Tolerances:
  counts      bit-exact on identical z (the slice index is the same two FP64 operations on
              both sides, so the integer decision is taken in the same precision);
  V           <= 1e-13 of max |V| (the GPU sums each slice's terms in 32 lane-strided
              partial sums, the oracle in order: rounding only);
  one step    delta within 1e-15 absolute plus |alpha| times the V tolerance;
  many turns  per particle <= 1e-10 of the bucket / transverse amplitude after 1000 turns,
              moments <= 1e-9 (the map's tolerances; the kick adds a deterministic force
              computed from identical counts on both sides as long as no particle sits
              within rounding of a slice edge, a ~1e-4 chance at these sizes).
"""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl  # noqa: E402
from test_parity_gpu import moment_errors  # noqa: E402
from test_widened_gpu import widened_inputs  # noqa: E402

DEV = "cuda:0"
SCHEMES4 = ("euler_cromer", "leapfrog", "ruth4", "rk4")


def wake_table(ns, seed=3):
    """A decaying oscillating wake (resonator-like), seeded amplitude jitter."""
    m = np.arange(ns)
    rng = np.random.default_rng(seed)
    return np.exp(-m / (0.1 * ns + 1.0)) * np.cos(m / (0.05 * ns + 1.0)) * (1 + 0.1 * rng.normal(size=ns))


def grid(ns, lo=-0.75, hi=0.75):
    return dict(z_lo=lo, z_hi=hi, inv_dz=ns / (hi - lo))


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device=DEV)


@pytest.mark.parametrize("ns,alpha_sc", [(1, 0.0), (7, 0.0), (256, 0.0), (4096, 0.0), (2, 3e-9),
                                         (256, 3e-9), (4096, -1e-8)])
def test_one_step_matches_oracle(ns, alpha_sc):
    inp = widened_inputs(100_003, seed=31)
    z, dp = inp["z"], inp["dp"]
    g = grid(ns)
    w = wake_table(ns)
    alpha = -2e-9
    R = phtl.Ring(**inp["ring"])
    R.set_wake(w, g["z_lo"], g["z_hi"], alpha, alpha_sc)
    zt, dt = _t(z), _t(dp)
    cnt = torch.zeros(ns, dtype=torch.int32, device=DEV)
    V = torch.zeros(ns, dtype=torch.float64, device=DEV)
    R.collective_kick(zt, dt, counts_out=cnt, V_out=V)
    torch.cuda.synchronize()
    z1, d1, c_ref, V_ref = oracle.collective_kick(z, dp, g["z_lo"], g["inv_dz"], w, alpha, alpha_sc)
    assert np.array_equal(cnt.cpu().numpy().astype(np.int64), c_ref)
    assert np.array_equal(zt.cpu().numpy(), z)
    vs = np.max(np.abs(V_ref))
    assert np.max(np.abs(V.cpu().numpy() - V_ref)) <= 1e-13 * vs
    # the kick: wake part to the V tolerance; the space-charge part (half-integer slopes
    # times alpha_sc) and the sum to rounding
    sc = abs(alpha_sc) * max(1, int(np.max(c_ref)))
    assert np.max(np.abs(dt.cpu().numpy() - d1)) <= 1e-15 + abs(alpha) * 1e-13 * vs + 4e-16 * sc
    R.close()


def test_range_edges_and_outside_particles():
    """z_lo is in the first slice; z_hi, beyond, below and NaN-free outliers are neither
    counted nor kicked."""
    ns = 64
    g = grid(ns)
    dz = 1.5 / ns
    z = np.array([g["z_lo"], g["z_hi"], 5.0, -5.0, g["z_lo"] + 0.5 * dz, g["z_hi"] - 1e-9])
    dp = np.zeros(z.size)
    R = phtl.Ring(**widened_inputs(1, seed=1)["ring"])
    R.set_wake(np.ones(ns), g["z_lo"], g["z_hi"], 1.0)
    zt, dt = _t(z), _t(dp)
    cnt = torch.zeros(ns, dtype=torch.int32, device=DEV)
    R.collective_kick(zt, dt, counts_out=cnt)
    torch.cuda.synchronize()
    _, d1, c_ref, _ = oracle.collective_kick(z, dp, g["z_lo"], g["inv_dz"], np.ones(ns), 1.0)
    assert np.array_equal(cnt.cpu().numpy().astype(np.int64), c_ref)
    assert np.array_equal(dt.cpu().numpy(), d1)
    assert d1[1] == 0.0 and d1[2] == 0.0 and d1[3] == 0.0
    R.close()


def _edge_positions(ns):
    """Positions on [0, 1) whose slice decision sits on a bit-pattern edge: signed zeros,
    subnormals, the slice edges k / ns and their neighbours, the top edge and just below it,
    non-finite values."""
    tiny = 5e-324
    zs = [-0.0, 0.0, tiny, -tiny, 2.2250738585072014e-308, -1e-300, 1.0, 1.0 - 2.0 ** -53,
          np.nextafter(1.0, 2.0), float("nan"), -float("nan"), float("inf"), -float("inf"), 0.5]
    for k in range(0, ns + 1, max(1, ns // 37)):
        e = k / ns
        zs += [e, np.nextafter(e, -1.0), np.nextafter(e, 2.0)]
    return np.array(zs, dtype=np.float64)


@pytest.mark.parametrize("dtype", ["f64", "f32c"])
@pytest.mark.parametrize("ns", [1, 3, 7, 4096])
def test_slice_decision_at_bit_pattern_edges(ns, dtype):
    """The slice decision (two FP64 operations, then integer range test and floor on u's bit
    pattern) counts exactly the particles the oracle's floor((z - z_lo) inv_dz) counts, on
    signed zeros, subnormals, every slice edge and its neighbours, the top edge and
    non-finite positions; the kick then moves exactly those particles.  FP32C decides on
    hi + comp in FP64, so it takes positions that a float pair holds exactly."""
    z = _edge_positions(ns)
    if dtype == "f32c":
        z = np.array([v for v in z if not np.isfinite(v) or float(np.float32(v)) == v
                      or v == 0.0], dtype=np.float64)
    dp = np.linspace(-1e-3, 1e-3, z.size)
    if dtype == "f32c":
        dp = phtl.join_f32c(phtl.split_f32c(dp))  # values a float pair holds exactly
    w = wake_table(ns)
    alpha = -1e-7
    R = phtl.Ring(**widened_inputs(1, seed=1)["ring"])
    R.set_wake(w, 0.0, 1.0, alpha)
    with np.errstate(invalid="ignore"):  # the pair of an infinity has a NaN low part
        zt = _t(z) if dtype == "f64" else _pair(z)
    dt = _t(dp) if dtype == "f64" else _pair(dp)
    cnt = torch.zeros(ns, dtype=torch.int32, device=DEV)
    R.collective_kick(zt, dt, counts_out=cnt, dtype=dtype)
    torch.cuda.synchronize()
    _, d1, c_ref, V_ref = oracle.collective_kick(z, dp, 0.0, float(ns), w, alpha)
    assert np.array_equal(cnt.cpu().numpy().astype(np.int64), c_ref)
    got = dt.cpu().numpy() if dtype == "f64" else phtl.join_f32c(dt.cpu().numpy())
    moved_ref = d1 != dp
    moved = got != dp
    assert np.array_equal(moved, moved_ref)
    vs = max(np.max(np.abs(V_ref)), 1.0)
    assert np.max(np.abs(got - d1)) <= 1e-15 + abs(alpha) * 1e-13 * vs
    R.close()


def run_gpu(inp, scheme, turns, w, g, alpha, stride=None, tuning=None, alpha_sc=0.0):
    R = phtl.Ring(**inp["ring"])
    if tuning:
        R.set_tuning(**tuning)
    R.set_wake(w, g["z_lo"], g["z_hi"], alpha, alpha_sc)
    bufs = [_t(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
    mon = None
    if stride:
        mon = torch.full((turns // stride + 1, phtl.MON_FIELDS), float("nan"), dtype=torch.float64,
                         device=DEV)
        R.set_monitor(mon, stride=stride)
    R.track_collective(*bufs, turns=turns, integrator=scheme)
    torch.cuda.synchronize()
    out = [b.cpu().numpy() for b in bufs]
    moms = phtl.moments_from_sums(mon.cpu().numpy()) if stride else None
    R.close()
    return out, moms


def run_ref(inp, scheme, turns, w, g, alpha, stride=None, alpha_sc=0.0):
    r = oracle.track_collective(inp["d"], scheme, inp["z"], inp["dp"], inp["x"], inp["xp"],
                                inp["y"], inp["yp"], turns=turns, z_lo=g["z_lo"],
                                inv_dz=g["inv_dz"], w=w, alpha=alpha, alpha_sc=alpha_sc,
                                moments=bool(stride), stride=stride or 1)
    return list(r[:6]), r[6]


def errors(inp, got, ref):
    d = inp["d"]
    zb, db = math.pi / d.k, 2 * math.sqrt(d.A / (d.k * d.etaC))
    e = [np.max(np.abs(got[0] - ref[0])) / zb, np.max(np.abs(got[1] - ref[1])) / db]
    for i in (2, 4):
        amp = np.max(np.hypot(ref[i], 50.0 * ref[i + 1]))
        e += [np.max(np.abs(got[i] - ref[i])) / amp, np.max(np.abs(got[i + 1] - ref[i + 1])) * 50.0 / amp]
    return max(e)


@pytest.mark.parametrize("scheme", SCHEMES4)
def test_turns_match_oracle(scheme):
    inp = widened_inputs(4099, seed=33)
    ns = 128
    g, w = grid(ns), wake_table(ns)
    alpha = -5e-9       # the wake's kick ~1e-3 of the RF kick at the bunch centre
    got, mg = run_gpu(inp, scheme, 1000, w, g, alpha, stride=7,
                      tuning=dict(block_threads=64))
    ref, mr = run_ref(inp, scheme, 1000, w, g, alpha, stride=7)
    assert errors(inp, got, ref) < 1e-10, errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < 1e-9
    # the wake does act: without it the bunch ends elsewhere
    plain, _ = run_ref(inp, scheme, 1000, w, g, 0.0)
    assert np.max(np.abs(plain[1] - ref[1])) > 1e3 * np.max(np.abs(got[1] - ref[1]))


@pytest.mark.parametrize("scheme", ["leapfrog", "ruth4"])
def test_turns_with_space_charge(scheme):
    """Wake and space charge together over 1000 turns."""
    inp = widened_inputs(4099, seed=34)
    ns = 128
    g, w = grid(ns), wake_table(ns, seed=5)
    got, mg = run_gpu(inp, scheme, 1000, w, g, -3e-9, stride=11, alpha_sc=2e-8)
    ref, mr = run_ref(inp, scheme, 1000, w, g, -3e-9, stride=11, alpha_sc=2e-8)
    assert errors(inp, got, ref) < 1e-10, errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < 1e-9
    nosc, _ = run_ref(inp, scheme, 1000, w, g, -3e-9)
    assert np.max(np.abs(nosc[1] - ref[1])) > 1e3 * np.max(np.abs(got[1] - ref[1]))


def test_turns_widened_double_rf():
    inp = widened_inputs(2049, seed=35, eta1=0.05, eta2=2.0, xi_x=5.0, xi_y=-3.0,
                         harmonic2=2 * 4620, voltage2_V=1.35e6, phi2_rad=0.0)
    ns = 200
    g, w = grid(ns), wake_table(ns, seed=4)
    got, mg = run_gpu(inp, "ruth4", 500, w, g, 3e-9, stride=50)
    ref, mr = run_ref(inp, "ruth4", 500, w, g, 3e-9, stride=50)
    assert errors(inp, got, ref) < 1e-10
    assert moment_errors(inp["d"], mg, mr) < 1e-9


@pytest.mark.parametrize("dtype", ["f32c", "f32cd", "f32cs"])
def test_turns_widened_double_rf_f32(dtype):
    """The FP32 types on the widened, double-RF ring (the widened map's double-float code)."""
    inp = widened_inputs(2049, seed=35, eta1=0.05, eta2=2.0, xi_x=5.0, xi_y=-3.0,
                         harmonic2=2 * 4620, voltage2_V=1.35e6, phi2_rad=0.0)
    ns = 200
    g, w = grid(ns), wake_table(ns, seed=4)
    R = phtl.Ring(**inp["ring"])
    R.set_wake(w, g["z_lo"], g["z_hi"], 3e-9)
    bufs = [_pair(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
    mon = torch.zeros((500 // 50 + 1, phtl.MON_FIELDS), dtype=torch.float64, device=DEV)
    R.set_monitor(mon, stride=50)
    R.track_collective(*bufs, turns=500, integrator="ruth4", dtype=dtype)
    torch.cuda.synchronize()
    got = [phtl.join_f32c(b.cpu().numpy()) for b in bufs]
    mg = phtl.moments_from_sums(mon.cpu().numpy())
    R.close()
    ref, mr = run_ref(inp, "ruth4", 500, w, g, 3e-9, stride=50)
    tol = {"f32c": (1e-8, 1e-6), "f32cd": (1e-8, 1e-6), "f32cs": (2e-2, 2e-3)}[dtype]
    assert errors(inp, got, ref) < tol[0], errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < tol[1]


@pytest.mark.parametrize("dtype", ["f32cd", "f32cs"])
@pytest.mark.parametrize("scheme", ["leapfrog", "ruth4"])
def test_zero_strength_equals_plain_tracking_f32(dtype, scheme):
    """alpha = 0 in the FP32 types: bitwise the pairs of phtl_track (the linear map's
    double-float code on both sides)."""
    inp = widened_inputs(3001, seed=38)
    g, w = grid(64), wake_table(64)
    R = phtl.Ring(**inp["ring"])
    R.set_wake(w, g["z_lo"], g["z_hi"], 0.0)
    a = [_pair(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
    b = [_pair(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
    R.track_collective(*a, turns=300, integrator=scheme, dtype=dtype)
    R.track(*b, turns=300, integrator=scheme, dtype=dtype)
    torch.cuda.synchronize()
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    R.close()


@pytest.mark.parametrize("scheme", ["euler_cromer", "ruth4"])
def test_zero_strength_equals_plain_tracking(scheme):
    """alpha = 0: bitwise the particles of phtl_track (the turn's map is the same code; the
    state's HBM round trip per turn is exact)."""
    inp = widened_inputs(3001, seed=37)
    g, w = grid(64), wake_table(64)
    a, _ = run_gpu(inp, scheme, 300, w, g, 0.0)
    R = phtl.Ring(**inp["ring"])
    bufs = [_t(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
    R.track(*bufs, turns=300, integrator=scheme)
    torch.cuda.synchronize()
    for u, b in zip(a, bufs):
        assert np.array_equal(u, b.cpu().numpy())
    R.close()


@pytest.mark.parametrize("n", [1, 3, 5])
def test_ragged_small(n):
    inp = widened_inputs(n, seed=39 + n)
    g, w = grid(16), wake_table(16)
    got, mg = run_gpu(inp, "leapfrog", 300, w, g, -1e-6, stride=100, tuning=dict(block_threads=32))
    ref, mr = run_ref(inp, "leapfrog", 300, w, g, -1e-6, stride=100)
    assert errors(inp, got, ref) < 1e-10
    assert np.allclose(mg[:, :4], mr[:, :4], rtol=1e-9, atol=1e-18)


@pytest.mark.parametrize("dtype", ["f64", "f32cd"])
def test_one_ring_growing_and_shrinking_bunches(dtype):
    """The slice of each particle is kept between launches in a buffer of the ring's that
    grows with the bunch: calls with 1001, 5003, 3 and 4099 particles on one ring, a one-step
    kick in between, each against the oracle (no slice of an earlier call leaks in)."""
    g, w = grid(64), wake_table(64)
    alpha = -2e-9
    R = phtl.Ring(**widened_inputs(1, seed=1)["ring"])
    R.set_wake(w, g["z_lo"], g["z_hi"], alpha)
    tol = 1e-10 if dtype == "f64" else 1e-8
    for i, n in enumerate((1001, 5003, 3, 4099)):
        inp = widened_inputs(n, seed=60 + i)
        if dtype == "f64":
            bufs = [_t(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
        else:
            bufs = [_pair(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
        R.track_collective(*bufs, turns=200, integrator="leapfrog", dtype=dtype)
        torch.cuda.synchronize()
        got = [b.cpu().numpy() if dtype == "f64" else phtl.join_f32c(b.cpu().numpy()) for b in bufs]
        ref, _ = run_ref(inp, "leapfrog", 200, w, g, alpha)
        assert errors(inp, got, ref) < tol, (n, errors(inp, got, ref))
        if n == 5003:
            # a one-step kick on the first 1000 particles of the tracked bunch
            z0 = got[0][:1000].copy()
            d0 = got[1][:1000].copy()
            zt, dt = (_t(z0), _t(d0)) if dtype == "f64" else (_pair(z0), _pair(d0))
            R.collective_kick(zt, dt, dtype=dtype)
            torch.cuda.synchronize()
            d1 = dt.cpu().numpy() if dtype == "f64" else phtl.join_f32c(dt.cpu().numpy())
            _, dref, _, _ = oracle.collective_kick(z0, d0, g["z_lo"], g["inv_dz"], w, alpha)
            # V to rounding (1000 counts at most); the pair's precision on delta itself
            scale = abs(alpha) * np.max(np.abs(w)) * 1000
            assert np.max(np.abs(d1 - dref)) <= 1e-12 * scale + 1e-14 * np.max(np.abs(d0))
    R.close()


@pytest.mark.parametrize("dtype", ["f32c", "f32cd"])
@pytest.mark.parametrize("n", [1, 3, 5, 4097])
def test_ragged_small_f32(dtype, n):
    """FP32 types on sizes that leave a partial thread (4 particles per thread) and an
    unaligned comp half: the kept slices take the scalar path there."""
    inp = widened_inputs(n, seed=80 + n)
    g, w = grid(16), wake_table(16)
    alpha = -1e-6 if n < 10 else -2e-9
    R = phtl.Ring(**inp["ring"])
    R.set_tuning(block_threads=32)
    R.set_wake(w, g["z_lo"], g["z_hi"], alpha)
    bufs = [_pair(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
    R.track_collective(*bufs, turns=300, integrator="leapfrog", dtype=dtype)
    torch.cuda.synchronize()
    got = [phtl.join_f32c(b.cpu().numpy()) for b in bufs]
    R.close()
    ref, _ = run_ref(inp, "leapfrog", 300, w, g, alpha)
    assert errors(inp, got, ref) < 1e-8, errors(inp, got, ref)


def test_zero_turns_records_row_zero_only():
    inp = widened_inputs(1001, seed=41)
    g, w = grid(32), wake_table(32)
    got, mg = run_gpu(inp, "leapfrog", 0, w, g, 1e-6, stride=1)
    for k, u in zip(("z", "dp", "x", "xp", "y", "yp"), got):
        assert np.array_equal(u, inp[k])
    ref = oracle.moments(*[inp[k] for k in ("z", "dp", "x", "xp", "y", "yp")])
    assert mg.shape[0] == 1 and np.allclose(mg[0], ref, rtol=1e-9, atol=1e-18)


def test_argument_errors():
    inp = widened_inputs(64, seed=43)
    R = phtl.Ring(**inp["ring"])
    bufs = [_t(inp[k]) for k in ("z", "dp")]
    with pytest.raises(phtl.PhtlError) as e:
        R.track_collective(*bufs, turns=1)              # no wake attached
    assert e.value.code == phtl.E_INVALID
    R.set_wake(np.ones(8), -0.5, 0.5, 1e-6)
    rc = phtl.load().phtl_track_collective(R.handle, bufs[0].data_ptr(), bufs[1].data_ptr(), None,
                                           None, None, None, 64, 1, 9, 0, None)
    assert rc == phtl.E_INVALID                          # no such integrator
    R.set_wake(None)
    with pytest.raises(phtl.PhtlError):
        R.collective_kick(*bufs)
    R.close()


def _pair(a):
    return torch.tensor(phtl.split_f32c(np.asarray(a, dtype=np.float64)), dtype=torch.float32,
                        device=DEV)


@pytest.mark.parametrize("dtype", ["f32c", "f32cd", "f32cs"])
def test_one_step_f32(dtype):
    """FP32 types: the same counts (slice decisions in FP64 from hi + comp, or exactly from
    the double-float u: the inputs lie nowhere near an edge to 1e-12), the kick to the
    pair's precision (FP32CS: one float, the pair's truncated high part)."""
    inp = widened_inputs(50_001, seed=51)
    z, dp = inp["z"], inp["dp"]
    ns = 300
    g, w = grid(ns), wake_table(ns)
    alpha, alpha_sc = -2e-9, 5e-9
    R = phtl.Ring(**inp["ring"])
    R.set_wake(w, g["z_lo"], g["z_hi"], alpha, alpha_sc)
    zt, dt = _pair(z), _pair(dp)
    cnt = torch.zeros(ns, dtype=torch.int32, device=DEV)
    R.collective_kick(zt, dt, counts_out=cnt, dtype=dtype)
    torch.cuda.synchronize()
    _, d1, c_ref, V_ref = oracle.collective_kick(z, dp, g["z_lo"], g["inv_dz"], w, alpha, alpha_sc)
    assert np.array_equal(cnt.cpu().numpy().astype(np.int64), c_ref)
    got = phtl.join_f32c(dt.cpu().numpy())
    kick = np.max(np.abs(d1 - dp))
    # FP32CS adds the high float of the kick's pair: the FP64 value's top 24 bits,
    # truncated (relative error below 2^-23)
    tol = 1e-12 * np.max(np.abs(dp)) + (2.5e-7 * kick if dtype == "f32cs" else 1e-12 * kick)
    assert np.max(np.abs(got - d1)) <= tol, (np.max(np.abs(got - d1)), tol)
    R.close()


@pytest.mark.parametrize("dtype", ["f32c", "f32cd", "f32cs"])
@pytest.mark.parametrize("scheme", ["leapfrog", "ruth4"])
def test_turns_f32(dtype, scheme):
    """FP32 types over 1000 turns against the FP64 oracle, with the tolerances of the FP32
    paths (per particle 1e-8 / 2e-2, moments 1e-6 / 2e-3)."""
    inp = widened_inputs(2051, seed=53)
    ns = 128
    g, w = grid(ns), wake_table(ns)
    R = phtl.Ring(**inp["ring"])
    R.set_wake(w, g["z_lo"], g["z_hi"], -5e-9, 1e-8)
    bufs = [_pair(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
    mon = torch.zeros((1000 // 10 + 1, phtl.MON_FIELDS), dtype=torch.float64, device=DEV)
    R.set_monitor(mon, stride=10)
    R.track_collective(*bufs, turns=1000, integrator=scheme, dtype=dtype)
    torch.cuda.synchronize()
    got = [phtl.join_f32c(b.cpu().numpy()) for b in bufs]
    mg = phtl.moments_from_sums(mon.cpu().numpy())
    R.close()
    ref, mr = run_ref(inp, scheme, 1000, w, g, -5e-9, stride=10, alpha_sc=1e-8)
    tol = {"f32c": (1e-8, 1e-6), "f32cd": (1e-8, 1e-6), "f32cs": (2e-2, 2e-3)}[dtype]
    assert errors(inp, got, ref) < tol[0], errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < tol[1]


def test_full_size_sampled():
    """1e6 particles x 100 turns in the default launch shape against the oracle run on the
    whole bunch (the step couples every particle): a 512-particle sample and the moments."""
    n = 1_000_000
    inp = widened_inputs(n, seed=45)
    ns = 512
    g, w = grid(ns), wake_table(ns)
    got, mg = run_gpu(inp, "leapfrog", 100, w, g, -5e-11, stride=50)
    ref, mr = run_ref(inp, "leapfrog", 100, w, g, -5e-11, stride=50)
    idx = np.random.default_rng(9).choice(n, 512, replace=False)
    sub = dict(inp)
    assert errors(sub, [u[idx] for u in got], [v[idx] for v in ref]) < 1e-10
    assert moment_errors(inp["d"], mg, mr) < 1e-9
