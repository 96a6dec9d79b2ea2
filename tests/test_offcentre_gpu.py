"""Monitor moments of an off-centre bunch against the oracle's two-pass moments.

A short bunch (sigma_z = 5 mm, matched) displaced by 20 sigma in z and delta and by 20 sigma
in x and x' performs dipole (centroid) oscillations about the bucket's fixed point: its raw
second moments sum u^2 are up to ~400 times its spread, and var = <u^2> - <u>^2 loses
(mean / rms)^2 times the sums' rounding to cancellation.  The monitor sums are taken about
the fixed point (0, 0) -- the synchronous particle and closed orbit, about which every
centroid of this map oscillates -- so the bound follows from the partials' precision:
  - the FP64 kernels keep double-float (~47-bit) partials: (20)^2 * 2^-47 ~ 3e-12, far inside
    the FP64 parity tolerance of 1e-9;
  - the FP32 kernels keep FP32 partials per thread and warp (128 particles): the warp's sum of
    squares carries ~2^-24 per butterfly level relative to (mean^2 + rms^2), i.e. about
    1e-6 (1 + (mean/rms)^2) of the variance, averaging down over the W warps as 1/sqrt(W):
    measured 1.1e-4 at 20 sigma for 5000 particles (40 warps); tolerance 5e-4 (a centred
    bunch's is 1e-6).
FP32CS gets 5e-3: its SFU sine (~4e-7 absolute) shifts the synchrotron tune by ~5e-7
relative, i.e. ~6e-5 rad of centroid phase after 2000 turns, which a 20-sigma dipole
amplitude turns into ~1e-3 of the rms in the mean.  Means are compared relative to the
matching rms.  The ramp programme (accelerating bucket) is checked the same way.
"""
import numpy as np
import pytest

import helpers
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl, synth  # noqa: E402
from test_parity_gpu import moment_errors, run_gpu, run_ref  # noqa: E402

TOL = {"f64": 1e-9, "f32c": 5e-4, "f32cd": 5e-4, "f32cs": 5e-3}
OFFSET_SIGMAS = 20.0


def offcentre_inputs(n, seed, voltage=4.5e6):
    ring = synth.ring(voltage, transverse=True)
    d = oracle.derive(ring)
    z, dp, _ = synth.matched_bunch(seed, n, helpers.bucket_of(d), sigma_z=0.005)
    x, xp = synth.transverse_gaussian(seed + 101, n, 50.0, 2e-6, d.betagamma)
    y, yp = synth.transverse_gaussian(seed + 202, n, 50.0, 2e-6, d.betagamma)
    z = z + OFFSET_SIGMAS * np.std(z)
    dp = dp + OFFSET_SIGMAS * np.std(dp)
    x = x + OFFSET_SIGMAS * np.std(x)
    xp = xp + OFFSET_SIGMAS * np.std(xp)
    return dict(ring=ring, d=d, z=z, dp=dp, x=x, xp=xp, y=y, yp=yp)


@pytest.mark.parametrize("dtype", ["f64", "f32c", "f32cd", "f32cs"])
@pytest.mark.parametrize("scheme", ["leapfrog", "ruth4"])
def test_offcentre_bunch_moments(dtype, scheme):
    inp = offcentre_inputs(5003, seed=41)
    # the centroid really is far out, relative to the spread, at the start
    assert abs(np.mean(inp["z"])) > 15 * np.std(inp["z"])
    got, mg = run_gpu(inp, scheme, 2000, dtype=dtype, stride=10)
    ref, mr = run_ref(inp, scheme, 2000, stride=10)
    # and it oscillates: somewhere along the track it sits far from the origin
    assert np.max(np.abs(mr[:, 0]) / mr[:, 2]) > 15
    err = moment_errors(inp["d"], mg, mr)
    assert err < TOL[dtype], (dtype, scheme, err)


@pytest.mark.parametrize("dtype", ["f64", "f32c"])
def test_offcentre_bunch_through_a_ramp(dtype):
    import test_ramp_gpu as tr

    inp = tr.ramp_inputs(4099, seed=43, amp=0.05)
    for k in ("z", "dp", "x", "xp"):
        inp[k] = inp[k] + OFFSET_SIGMAS * np.std(inp[k])
    got, mg = tr.run_gpu(inp, "leapfrog", 0, 2000, dtype=dtype, stride=10)
    ref, mr = tr.run_ref(inp, "leapfrog", 0, 2000, stride=10)
    assert np.max(np.abs(mr[:, 0]) / mr[:, 2]) > 15
    assert moment_errors(inp["d"], mg, mr) < TOL[dtype]
