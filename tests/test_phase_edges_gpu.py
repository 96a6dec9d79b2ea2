"""Edge values of the RF phase argument in the FP32-compensated kernels against the oracle.

PHTL_F32C forms the phase k z in FP64 from the coordinate's two floats and splits it back
into a float pair; for magnitudes outside [2^-74, 2^128) the split takes its general form,
and beyond |k z| = 1e4 the double-float sine takes the FP64 one.  Particles placed on
those edges -- the synchronous particle (z = 0 exactly, which must stay there), phases of
1e-30 and below 2^-74, a coordinate whose high float is subnormal, and a particle outside
the bucket whose phase runs past 1e4 -- must follow the FP64 oracle like the rest of the
bunch (per-particle tolerance of the double-float arithmetic, 1e-8 of the particle's
amplitude; the escaped particle 1e-8 of its own |z|).
"""
import math

import numpy as np
import pytest

import helpers
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl  # noqa: E402

DEV = "cuda:0"


def edge_bunch(n=4000, seed=61):
    inp = helpers.inputs(n, seed=seed, transverse=False)
    d = inp["d"]
    zb = math.pi / d.k
    db = 2 * math.sqrt(abs(d.A / (d.k * d.etaC)))
    z, dp = inp["z"].copy(), inp["dp"].copy()
    edges = [(0.0, 0.0), (1e-30, 0.0), (-1e-30, 0.0), (2.0 ** -76 / d.k, 0.0),
             (-(2.0 ** -80) / d.k, 0.0), (1e-40, 0.0), (-1e-41, 0.0), (0.0, 1e-38),
             (2.0 ** -60, -(2.0 ** -61)), (0.3 * zb, 0.0), (-0.8 * zb, 0.0), (0.0, 0.7 * db)]
    for i, (ze, de) in enumerate(edges):
        z[i], dp[i] = ze, de
    escaped = len(edges)
    # outside the bucket (65 bucket heights): runs away, |k z| passes 1e4 after ~1400 turns
    z[escaped], dp[escaped] = 0.0, 0.4
    return inp, z, dp, len(edges), escaped


@pytest.mark.parametrize("dtype", ["f32c", "f32cd"])
@pytest.mark.parametrize("scheme", ["leapfrog", "ruth4"])
def test_phase_edges_follow_the_oracle(dtype, scheme):
    inp, z, dp, nedge, esc = edge_bunch()
    d = inp["d"]
    turns = 3000
    R = phtl.Ring(**inp["ring"])
    bz = torch.tensor(phtl.split_f32c(z), dtype=torch.float32, device=DEV)
    bd = torch.tensor(phtl.split_f32c(dp), dtype=torch.float32, device=DEV)
    R.track(bz, bd, turns=turns, integrator=scheme, dtype=dtype)
    torch.cuda.synchronize()
    gz = phtl.join_f32c(bz.cpu().numpy())
    gd = phtl.join_f32c(bd.cpu().numpy())
    R.close()
    ref = oracle.track(d, scheme, z, dp, turns=turns)
    rz, rd = ref[0], ref[1]
    assert np.all(np.isfinite(gz)) and np.all(np.isfinite(gd))
    # the synchronous particle stays exactly at the fixed point
    assert gz[0] == 0.0 and gd[0] == 0.0
    # the escaped particle's phase ran past the double-float sine's range
    assert abs(d.k * rz[esc]) > 1e4
    assert abs(gz[esc] - rz[esc]) <= 1e-8 * abs(rz[esc])
    assert abs(gd[esc] - rd[esc]) <= 1e-8 * abs(rd[esc])
    inside = np.ones(len(z), bool)
    inside[esc] = False
    err = helpers.rel_errors(d, [rz[inside], rd[inside], None, None, None, None],
                             [gz[inside], gd[inside], None, None, None, None],
                             z[inside], dp[inside])
    assert np.max(err[:nedge]) < 1e-8, err[:nedge]
    assert np.max(err) < 1e-8
