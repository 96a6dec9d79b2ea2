"""Regression fixtures under tests/golden/ (written by tests/golden/make_golden.py from the
oracle alone; the paper prints no physics values).  On the CPU the oracle must reproduce
them to 1e-13 of the bucket size (its arithmetic is uncontracted FP64; the slack only
covers another C library's sine on another host, so a difference means the oracle's
arithmetic changed); on the GPU the library must match them within the FP64 parity
tolerance (per particle 1e-10 of the bucket size after 1000 turns, moments 1e-9)."""
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "oracle_small_workload_1000turns.txt")


def load_fixture():
    parts, moms = {}, {}
    with open(FIXTURE) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            if tok[0] == "particle":
                parts.setdefault(tok[1], []).append((int(tok[2]), float(tok[3]), float(tok[4])))
            elif tok[0] == "moments":
                moms[tok[1]] = np.array([float(v) for v in tok[2:]])
    return parts, moms


def _inputs():
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_golden

    return make_golden.inputs(), make_golden.TURNS


def test_oracle_reproduces_fixture():
    parts, moms = load_fixture()
    (ring, d, z, dp), turns = _inputs()
    assert set(parts) == {"euler_cromer", "leapfrog", "ruth4", "rk4"}
    zb, db = math.pi / d.k, 2 * math.sqrt(d.A / (d.k * d.etaC))
    for s, rows in parts.items():
        zf, df, *_, mom = oracle.track(d, s, z, dp, turns=turns, moments=True, stride=turns)
        for i, zi, di in rows:
            assert abs(zf[i] - zi) / zb < 1e-13 and abs(df[i] - di) / db < 1e-13, (s, i)
        scale = np.array([mom[-1, 2], mom[-1, 3], mom[-1, 2], mom[-1, 3], mom[-1, 4]])
        assert np.all(np.abs(mom[-1, :5] - moms[s]) <= 1e-13 * np.abs(scale)), s


@pytest.mark.gpu
def test_library_matches_fixture():
    torch = pytest.importorskip("torch")
    from paper_1610_05801_gb300 import phtl

    parts, moms = load_fixture()
    (ring, d, z, dp), turns = _inputs()
    zb, db = math.pi / d.k, 2 * math.sqrt(d.A / (d.k * d.etaC))
    R = phtl.Ring(**ring)
    for s, rows in parts.items():
        Z = torch.tensor(z, dtype=torch.float64, device="cuda:0")
        D = torch.tensor(dp, dtype=torch.float64, device="cuda:0")
        mon = torch.zeros((2, phtl.MON_FIELDS), dtype=torch.float64, device="cuda:0")
        R.set_monitor(mon, stride=turns)
        R.track(Z, D, turns=turns, integrator=s, dtype="f64")
        torch.cuda.synchronize()
        zg, dg = Z.cpu().numpy(), D.cpu().numpy()
        for i, zi, di in rows:
            assert abs(zg[i] - zi) / zb < 1e-10 and abs(dg[i] - di) / db < 1e-10, (s, i)
        m = phtl.moments_from_sums(mon.cpu().numpy())[-1, :5]
        ref = moms[s]
        assert np.all(np.abs(m[[2, 3]] - ref[[2, 3]]) / ref[[2, 3]] < 1e-9), s
        assert abs(m[0] - ref[0]) / ref[2] < 1e-9 and abs(m[1] - ref[1]) / ref[3] < 1e-9, s
    R.set_monitor(None)
    R.close()
