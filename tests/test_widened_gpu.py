"""GPU parity of the widened map against the oracle: the slippage expansion
eta(delta) = eta0 + eta1 delta + eta2 delta^2 in the drift and the chromatic transverse
rotation 2 pi (frac Q + xi delta), alone and together, for every scheme and arithmetic,
through the single-bunch, per-turn, batched and serving paths.

Tolerances (the same derivation as the linear map's):
  FP64        per particle <= 1e-10 of the bucket / transverse amplitude after 1000 turns;
              moments <= 1e-9.  The chromatic angle is rounded once per turn on both
              sides (~1e-16), the drift polynomial likewise.
  FP32C/CD    per particle <= 1e-8, moments <= 1e-6 (double-float sine and cosine,
              ~4e-12 absolute per turn).
  FP32CS      per particle <= 2e-2, moments <= 2e-3 (FP32 angle and SFU sine/cosine).
"""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl, synth  # noqa: E402
from test_parity_gpu import moment_errors, run_gpu, run_ref  # noqa: E402

SCHEMES = ("euler_cromer", "leapfrog", "ruth4")
# bounded motion inside the 4.5 MV bucket (the oracle's pins use the same coefficients)
ETA1, ETA2 = 0.05, 2.0
XI_X, XI_Y = 5.0, -3.0
CASES = {
    "slippage": dict(eta1=ETA1, eta2=ETA2),
    "chromaticity": dict(xi_x=XI_X, xi_y=XI_Y),
    "both": dict(eta1=ETA1, eta2=ETA2, xi_x=XI_X, xi_y=XI_Y),
}


def widened_inputs(n, seed, phi_s=0.0, **over):
    ring = synth.ring(4.5e6, transverse=True, phi_s_rad=phi_s, **over)
    d = oracle.load().derive(ring)
    b = synth.Bucket(k=d.k, A=d.A, etaC=d.etaC, Qs=d.Qs, betagamma=d.betagamma)
    z, dp, _ = synth.matched_bunch(seed, n, b, sigma_z=0.12, sep_frac=0.5)
    x, xp = synth.transverse_gaussian(seed + 101, n, 50.0, 2e-6, d.betagamma)
    y, yp = synth.transverse_gaussian(seed + 202, n, 50.0, 2e-6, d.betagamma)
    return dict(ring=ring, d=d, z=z, dp=dp, x=x, xp=xp, y=y, yp=yp)


def errors(inp, got, ref):
    d = inp["d"]
    zb, db = math.pi / d.k, 2 * math.sqrt(d.A / (d.k * d.etaC))
    ez = np.max(np.abs(got[0] - ref[0])) / zb
    ed = np.max(np.abs(got[1] - ref[1])) / db
    et = 0.0
    for i in (2, 4):
        amp = np.max(np.hypot(ref[i], 50.0 * ref[i + 1]))
        et = max(et, np.max(np.abs(got[i] - ref[i])) / amp,
                 np.max(np.abs(got[i + 1] - ref[i + 1])) * 50.0 / amp)
    return max(ez, ed, et)


TOL = {"f64": (1e-10, 1e-9), "f32c": (1e-8, 1e-6), "f32cd": (1e-8, 1e-6), "f32cs": (2e-2, 2e-3)}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("scheme", SCHEMES)
def test_widened_f64(case, scheme):
    inp = widened_inputs(4099, seed=41, **CASES[case])
    got, mg = run_gpu(inp, scheme, 1000, stride=7, tuning=dict(block_threads=64,
                                                              turns_per_launch=333))
    ref, mr = run_ref(inp, scheme, 1000, stride=7)
    assert errors(inp, got, ref) < TOL["f64"][0]
    assert moment_errors(inp["d"], mg, mr) < TOL["f64"][1]


@pytest.mark.parametrize("dtype", ["f32c", "f32cd", "f32cs"])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_widened_f32(dtype, scheme):
    inp = widened_inputs(2051, seed=43, **CASES["both"])
    got, mg = run_gpu(inp, scheme, 1000, dtype=dtype, stride=10)
    ref, mr = run_ref(inp, scheme, 1000, stride=10)
    assert errors(inp, got, ref) < TOL[dtype][0], errors(inp, got, ref)
    assert moment_errors(inp["d"], mg, mr) < TOL[dtype][1]


@pytest.mark.parametrize("scheme", SCHEMES)
def test_widened_nonzero_phi_s(scheme):
    """phi_s != 0 (general kick) together with the widened map."""
    inp = widened_inputs(1001, seed=47, phi_s=0.3, **CASES["both"])
    d = inp["d"]
    zb = math.pi / d.k
    inp["z"] = inp["z"] * 0.3            # stay well inside the smaller accelerating bucket
    inp["dp"] = inp["dp"] * 0.3
    got, mg = run_gpu(inp, scheme, 1000, stride=25)
    ref, mr = run_ref(inp, scheme, 1000, stride=25)
    assert np.max(np.abs(got[0] - ref[0])) < 1e-11 * zb
    assert errors(inp, got, ref) < 1e-10
    assert moment_errors(d, mg, mr) < 1e-9


def test_widened_zero_coefficients_equal_linear_map():
    """eta1 = eta2 = xi = 0 selects the linear kernels: the general path is not taken, and
    the general path itself, fed coefficients that vanish in one plane, matches."""
    inp = widened_inputs(2049, seed=49)
    a, _ = run_gpu(inp, "leapfrog", 300)
    inp2 = widened_inputs(2049, seed=49, xi_y=1e-300)   # general path; x plane achromatic
    b, _ = run_gpu(inp2, "leapfrog", 300)
    # longitudinal and x: the same operations in both kernels -> bitwise
    for i in (0, 1, 2, 3):
        assert np.array_equal(a[i], b[i]), i


def test_widened_perturn_equals_persistent():
    inp = widened_inputs(2049, seed=51, **CASES["both"])
    a, ma = run_gpu(inp, "ruth4", 200, stride=10)
    b, mb = run_gpu(inp, "ruth4", 200, stride=10, perturn=True)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    # monitor sums added in another order: the moments agree to its rounding
    assert moment_errors(inp["d"], ma, mb) < 1e-11


@pytest.mark.parametrize("dtype", ["f64", "f32cd"])
def test_widened_batch_equals_alone(dtype):
    """Batched jobs on a ring with the widened map track bitwise as alone."""
    inp = widened_inputs(3001, seed=53, **CASES["both"])
    R = phtl.Ring(**inp["ring"])
    dev = "cuda:0"

    def bufs():
        out = []
        for k in ("z", "dp", "x", "xp", "y", "yp"):
            a = inp[k]
            out.append(torch.tensor(a if dtype == "f64" else phtl.split_f32c(a),
                                    dtype=torch.float64 if dtype == "f64" else torch.float32,
                                    device=dev))
        return out

    alone = bufs()
    R.track(*alone, turns=250, integrator="leapfrog", dtype=dtype)
    jb = [bufs(), bufs()]
    jobs = [phtl.make_job(*jb[0], turns=250, integrator="leapfrog", dtype=dtype),
            phtl.make_job(*jb[1], turns=100, integrator="ruth4", dtype=dtype)]
    B = phtl.Batch(R, jobs)
    B.run()
    torch.cuda.synchronize()
    for u, v in zip(alone, jb[0]):
        assert torch.equal(u, v)
    ref = bufs()
    R.track(*ref, turns=100, integrator="ruth4", dtype=dtype)
    torch.cuda.synchronize()
    for u, v in zip(ref, jb[1]):
        assert torch.equal(u, v)
    B.close()
    R.close()


def test_widened_serving_equals_alone():
    inp = widened_inputs(2001, seed=57, **CASES["both"])
    R = phtl.Ring(**inp["ring"])
    host = [np.array(inp[k]) for k in ("z", "dp", "x", "xp", "y", "yp")]
    alone = [torch.tensor(a, device="cuda:0") for a in host]
    R.track(*alone, turns=400, integrator="ruth4", dtype="f64")
    torch.cuda.synchronize()
    S = phtl.Server(R, memory_budget_bytes=1e9, max_active=4)
    try:
        t = S.submit(*host, turns=400, integrator="ruth4", dtype="f64")
        rc, st = S.wait(t)
        assert rc == 0 and st.state == phtl.DONE
    finally:
        S.stop()
    for u, v in zip(alone, host):
        assert np.array_equal(u.cpu().numpy(), v)
    ref, _ = run_ref(inp, "ruth4", 400)  # the served job against the oracle directly
    assert errors(inp, host, ref) < TOL["f64"][0], errors(inp, host, ref)
    R.close()
