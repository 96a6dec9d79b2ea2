"""GPU parity of the classic RK4 integrator and of the second RF system (double RF)
against the oracle, through the single-bunch, per-turn, batched, no-allocation and
serving paths.

RK4 is Sec. 1.1.2's "Runge-Kutta" read literally: one classic RK4 step per turn on
dz/dn = -eta(delta) C delta, d delta/dn = A F1(z) + A2 F2(z).  The second RF system adds
w A2 (sin(phi2 + k2 z) - sin phi2) to every kick (and to RK4's force).

Tolerances (the same derivation as the linear map's; RK4 is not symplectic, but over
1000 turns its map is as smooth as the others, so the per-operation rounding
differences -- FMA contraction, the library's sine -- grow the same way):
  FP64        per particle <= 1e-10 of the bucket / transverse amplitude; moments <= 1e-9.
  FP32C/CD    per particle <= 1e-8, moments <= 1e-6 (double-float stages and sine).
  FP32CS      per particle <= 2e-2, moments <= 2e-3 (FP32 stages, SFU sine).
"""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl  # noqa: E402
from test_parity_gpu import moment_errors, run_gpu, run_ref  # noqa: E402
from test_widened_gpu import TOL, errors, widened_inputs  # noqa: E402

H = 4620
# second system at twice the harmonic, 30 % of the main voltage (bunch-lengthening mode
# when in phase); the oracle's pins use the same shape
DUAL = dict(harmonic2=2 * H, voltage2_V=0.3 * 4.5e6, phi2_rad=0.0)
DUAL_PHASED = dict(harmonic2=2 * H, voltage2_V=0.3 * 4.5e6, phi2_rad=-0.4)
FLAT = dict(harmonic2=2 * H, voltage2_V=-0.5 * 4.5e6, phi2_rad=0.0)   # K = 0
WIDE = dict(eta1=0.05, eta2=2.0, xi_x=5.0, xi_y=-3.0)
SCHEMES4 = ("euler_cromer", "leapfrog", "ruth4", "rk4")


@pytest.mark.parametrize("case", ["plain", "dual", "wide_dual"])
def test_rk4_f64(case):
    over = {"plain": {}, "dual": DUAL, "wide_dual": dict(WIDE, **DUAL)}[case]
    inp = widened_inputs(4099, seed=61, **over)
    got, mg = run_gpu(inp, "rk4", 1000, stride=7, tuning=dict(block_threads=64,
                                                             turns_per_launch=333))
    ref, mr = run_ref(inp, "rk4", 1000, stride=7)
    assert errors(inp, got, ref) < TOL["f64"][0], errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < TOL["f64"][1]


@pytest.mark.parametrize("scheme", SCHEMES4)
@pytest.mark.parametrize("dual", ["dual", "phased"])
def test_double_rf_f64(scheme, dual):
    inp = widened_inputs(2053, seed=63, **(DUAL if dual == "dual" else DUAL_PHASED))
    got, mg = run_gpu(inp, scheme, 1000, stride=10)
    ref, mr = run_ref(inp, scheme, 1000, stride=10)
    assert errors(inp, got, ref) < TOL["f64"][0], errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < TOL["f64"][1]


@pytest.mark.parametrize("scheme", SCHEMES4)
def test_double_rf_nonzero_phi_s(scheme):
    """phi_s != 0 and phi2 != 0: both general kicks, small amplitudes."""
    inp = widened_inputs(1001, seed=65, phi_s=0.3, **DUAL_PHASED)
    inp["z"] = inp["z"] * 0.3
    inp["dp"] = inp["dp"] * 0.3
    got, mg = run_gpu(inp, scheme, 1000, stride=25)
    ref, mr = run_ref(inp, scheme, 1000, stride=25)
    assert errors(inp, got, ref) < TOL["f64"][0]
    assert moment_errors(inp["d"], mg, mr) < TOL["f64"][1]


@pytest.mark.parametrize("scheme", ["leapfrog", "rk4"])
def test_flat_bottom_bucket(scheme):
    """V2 = -V/2 at h2 = 2h cancels the linear slope (K = 0): accepted, and tracked as
    the oracle tracks it."""
    # a bunch matched to the double-RF bucket (the flat bottom has no linear tune to
    # match to), tracked in the flat-bottomed one
    inp = widened_inputs(1023, seed=67, **DUAL)
    inp["ring"] = dict(inp["ring"], **FLAT)
    inp["d"] = oracle.load().derive(inp["ring"])
    assert abs(inp["d"].K) < 1e-15 and np.std(inp["dp"]) > 0
    got, mg = run_gpu(inp, scheme, 1000, stride=50)
    ref, mr = run_ref(inp, scheme, 1000, stride=50)
    assert errors(inp, got, ref) < TOL["f64"][0]
    assert moment_errors(inp["d"], mg, mr) < TOL["f64"][1]


@pytest.mark.parametrize("dtype", ["f32c", "f32cd", "f32cs"])
@pytest.mark.parametrize("scheme", ["leapfrog", "rk4"])
def test_rk4_and_double_rf_f32(dtype, scheme):
    inp = widened_inputs(2051, seed=69, **dict(WIDE, **DUAL))
    got, mg = run_gpu(inp, scheme, 1000, dtype=dtype, stride=10)
    ref, mr = run_ref(inp, scheme, 1000, stride=10)
    assert errors(inp, got, ref) < TOL[dtype][0], errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < TOL[dtype][1]


@pytest.mark.parametrize("dtype", ["f32c", "f32cd", "f32cs"])
def test_rk4_f32_plain(dtype):
    """RK4 on the linear-map ring (no widened term): the FP32 RK4 stages alone."""
    inp = widened_inputs(1025, seed=71)
    got, mg = run_gpu(inp, "rk4", 1000, dtype=dtype, stride=20)
    ref, mr = run_ref(inp, "rk4", 1000, stride=20)
    assert errors(inp, got, ref) < TOL[dtype][0], errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < TOL[dtype][1]


@pytest.mark.parametrize("n", [1, 3, 5])
def test_rk4_ragged_small(n):
    inp = widened_inputs(n, seed=73 + n, **DUAL)
    got, _ = run_gpu(inp, "rk4", 500, tuning=dict(block_threads=32, turns_per_launch=77))
    ref, _ = run_ref(inp, "rk4", 500)
    assert errors(inp, got, ref) < TOL["f64"][0]


def test_rk4_rf_linear_matches_oracle():
    """rf_linear: RK4's one-turn matrix is the 4th-order Taylor polynomial of the linear
    flow (pinned in the oracle); the GPU follows the oracle to rounding."""
    inp = widened_inputs(257, seed=79, rf_linear=1, **DUAL)
    got, _ = run_gpu(inp, "rk4", 1000)
    ref, _ = run_ref(inp, "rk4", 1000)
    assert errors(inp, got, ref) < TOL["f64"][0]


@pytest.mark.parametrize("dtype", ["f64", "f32cd"])
def test_rk4_perturn_equals_persistent(dtype):
    inp = widened_inputs(2049, seed=81, **DUAL)
    a, ma = run_gpu(inp, "rk4", 150, dtype=dtype, stride=10)
    b, mb = run_gpu(inp, "rk4", 150, dtype=dtype, stride=10, perturn=True)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    # monitor sums added in another order: the moments agree to its rounding
    assert moment_errors(inp["d"], ma, mb) < 1e-11


def _bufs(inp, dtype):
    out = []
    for k in ("z", "dp", "x", "xp", "y", "yp"):
        a = inp[k]
        out.append(torch.tensor(a if dtype == "f64" else phtl.split_f32c(a),
                                dtype=torch.float64 if dtype == "f64" else torch.float32,
                                device="cuda:0"))
    return out


@pytest.mark.parametrize("ring_case", ["plain", "dual"])
@pytest.mark.parametrize("dtype", ["f64", "f32cd", "f32cs"])
def test_rk4_batch_and_noalloc_equal_alone(ring_case, dtype):
    """An RK4 job batched with a leap-frog job (RK4 forces the widened map's batched
    kernel for its group) tracks bitwise as alone, through phtl_batch_run and
    phtl_batch_run_noalloc; the batch's other job too."""
    inp = widened_inputs(3001, seed=83, **({} if ring_case == "plain" else DUAL))
    R = phtl.Ring(**inp["ring"])
    alone_rk4, alone_lf = _bufs(inp, dtype), _bufs(inp, dtype)
    R.track(*alone_rk4, turns=120, integrator="rk4", dtype=dtype)
    R.track(*alone_lf, turns=300, integrator="leapfrog", dtype=dtype)
    torch.cuda.synchronize()
    for use_noalloc in (False, True):
        jb = [_bufs(inp, dtype), _bufs(inp, dtype)]
        jobs = [phtl.make_job(*jb[0], turns=120, integrator="rk4", dtype=dtype),
                phtl.make_job(*jb[1], turns=300, integrator="leapfrog", dtype=dtype)]
        if use_noalloc:
            phtl.batch_run_noalloc(R, jobs)
        else:
            B = phtl.Batch(R, jobs)
            B.run()
        torch.cuda.synchronize()
        for u, v in zip(alone_rk4, jb[0]):
            assert torch.equal(u, v), use_noalloc
        for u, v in zip(alone_lf, jb[1]):
            assert torch.equal(u, v), use_noalloc
        if not use_noalloc:
            B.close()
    R.close()


def test_rk4_serving_equals_alone():
    """A served RK4 job (chunked into scheduling rounds, sharing them with a Ruth4 job on
    a double-RF ring) comes out bitwise as tracked alone."""
    inp = widened_inputs(2001, seed=87, **DUAL)
    R = phtl.Ring(**inp["ring"])
    host_a = [np.array(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
    host_b = [np.array(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
    alone_a = [torch.tensor(a, device="cuda:0") for a in host_a]
    alone_b = [torch.tensor(a, device="cuda:0") for a in host_b]
    R.track(*alone_a, turns=400, integrator="rk4", dtype="f64")
    R.track(*alone_b, turns=250, integrator="ruth4", dtype="f64")
    torch.cuda.synchronize()
    S = phtl.Server(R, memory_budget_bytes=1e9, max_active=4, chunk_turns_f64=64)
    try:
        ta = S.submit(*host_a, turns=400, integrator="rk4", dtype="f64")
        tb = S.submit(*host_b, turns=250, integrator="ruth4", dtype="f64")
        for t in (ta, tb):
            rc, st = S.wait(t)
            assert rc == 0 and st.state == phtl.DONE
    finally:
        S.stop()
    for u, v in zip(alone_a, host_a):
        assert np.array_equal(u.cpu().numpy(), v)
    for u, v in zip(alone_b, host_b):
        assert np.array_equal(u.cpu().numpy(), v)
    # and both served jobs against the oracle directly
    ref_a, _ = run_ref(inp, "rk4", 400)
    ref_b, _ = run_ref(inp, "ruth4", 250)
    assert errors(inp, host_a, ref_a) < TOL["f64"][0], errors(inp, host_a, ref_a)
    assert errors(inp, host_b, ref_b) < TOL["f64"][0], errors(inp, host_b, ref_b)
    R.close()


def test_rk4_full_size_sampled():
    """1e6 particles x 100 turns in the bench's launch shape: a sample of 512 particles
    against the oracle, and the monitor's last row against the moments of the arrays."""
    n = 1_000_000
    inp = widened_inputs(n, seed=89, **DUAL)
    got, mg = run_gpu(inp, "rk4", 100, stride=50)
    idx = np.random.default_rng(5).choice(n, 512, replace=False)
    sub = dict(inp)
    for k in ("z", "dp", "x", "xp", "y", "yp"):
        sub[k] = inp[k][idx]
    ref, _ = run_ref(sub, "rk4", 100)
    gs = [g[idx] for g in got]
    assert errors(sub, gs, ref) < TOL["f64"][0]
    full = oracle.moments(*got)
    assert np.max(np.abs(mg[-1, [2, 3, 7, 8]] - full[[2, 3, 7, 8]]) / full[[2, 3, 7, 8]]) < 1e-9
    assert math.isfinite(mg[-1, 4])
