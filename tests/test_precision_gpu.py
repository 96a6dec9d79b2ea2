"""The stated accuracy of the FP32-compensated path, on the GPU, against the FP64 oracle.

The bar: bunch moments (mean z and delta relative to the matching rms, rms z, rms delta,
emittance relative to rms_z * rms_delta) within 1e-4 of FP64 after 1e6 leap-frog turns, with
the Hamiltonian drift reported.  The workload is the precision sweep's bunch (2 MV ring, 60 %
matched core and 40 % uniform halo out to 98 % of the separatrix, core and halo interleaved
by a seeded permutation); its first N_SUB particles are a fair subsample (a prefix of the
bench's 1e4-particle comparison subsample) and are tracked alone: particles are independent,
so they come out bitwise as they would inside the full 4e6-particle run.

Hamiltonian drift: per particle (H_end - H_start) / H_start of the smooth Hamiltonian
H = eta C delta^2 / 2 + (A / k)(1 - cos k z).  For leap-frog it is dominated by the map's own
O(K) difference between its conserved quantity and H, which the FP64 oracle shows equally;
what the FP32 arithmetic adds on top is the difference of the two drifts, bounded here.

PHTL_F32CS (FP32 increments, SFU sine) does not reach the 1e-4 bar over 1e6 turns: its
moments are held to the bound it does meet, so that a change in it shows.
"""
import math

import numpy as np
import pytest

import helpers
import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_1610_05801_gb300 import phtl, synth  # noqa: E402
from test_parity_gpu import moment_errors  # noqa: E402

DEV = "cuda:0"
N_FULL = 4_000_000
N_SUB = 1500
TURNS = 1_000_000
STRIDE = 10_000
BAR = {"f32c": 1e-4, "f32cd": 1e-4, "f32cs": 1e-2}


def hamiltonian(d, z, dp):
    return 0.5 * d.etaC * dp * dp + (d.A / d.k) * (1.0 - np.cos(d.k * z))


@pytest.fixture(scope="module")
def sweep():
    ring = synth.ring(2e6)
    d = oracle.derive(ring)
    z, dp = synth.halo_bunch(2, N_FULL, helpers.bucket_of(d))
    z, dp = np.ascontiguousarray(z[:N_SUB]), np.ascontiguousarray(dp[:N_SUB])
    ref = oracle.track(d, "leapfrog", z, dp, turns=TURNS, moments=True, stride=STRIDE)
    return dict(ring=ring, d=d, z=z, dp=dp, ref=ref)


@pytest.mark.parametrize("dtype", ["f32c", "f32cd", "f32cs"])
def test_fp32_moments_after_1e6_turns(sweep, dtype, record_property):
    d, ref = sweep["d"], sweep["ref"]
    R = phtl.Ring(**sweep["ring"])
    bz = torch.tensor(phtl.split_f32c(sweep["z"]), dtype=torch.float32, device=DEV)
    bd = torch.tensor(phtl.split_f32c(sweep["dp"]), dtype=torch.float32, device=DEV)
    mon = torch.full((TURNS // STRIDE + 1, phtl.MON_FIELDS), float("nan"), dtype=torch.float64,
                     device=DEV)
    R.set_monitor(mon, stride=STRIDE)
    R.track(bz, bd, turns=TURNS, integrator="leapfrog", dtype=dtype)
    torch.cuda.synchronize()
    mg = phtl.moments_from_sums(mon.cpu().numpy())
    z32 = phtl.join_f32c(bz.cpu().numpy())
    d32 = phtl.join_f32c(bd.cpu().numpy())
    R.close()

    err = moment_errors(d, mg, ref[6])
    h0 = hamiltonian(d, sweep["z"], sweep["dp"])
    drift32 = (hamiltonian(d, z32, d32) - h0) / h0
    drift64 = (hamiltonian(d, ref[0], ref[1]) - h0) / h0
    report = dict(dtype=dtype, max_rel_moment_err=err,
                  h_drift_median=float(np.median(drift32)),
                  h_drift_abs_max=float(np.max(np.abs(drift32))),
                  oracle_h_drift_median=float(np.median(drift64)),
                  oracle_h_drift_abs_max=float(np.max(np.abs(drift64))),
                  h_drift_diff_abs_max=float(np.max(np.abs(drift32 - drift64))))
    for k, v in report.items():
        record_property(k, v)
    print(report)
    assert mg.shape == ref[6].shape and np.all(np.isfinite(mg))
    assert err < BAR[dtype], report
    # the drift is the scheme's bounded O(K) oscillation, not a growth
    assert report["h_drift_abs_max"] < 2e-3, report
    assert math.isfinite(report["h_drift_median"])
    if dtype != "f32cs":
        # double-float state, increments and sine: per particle the drift follows the oracle's
        assert abs(report["h_drift_median"] - report["oracle_h_drift_median"]) < 1e-9, report
        assert report["h_drift_diff_abs_max"] < 1e-5, report
