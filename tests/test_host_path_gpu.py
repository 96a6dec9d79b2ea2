"""The host-buffer path on the GPU: phtl_track_host gives the oracle's particles, times the
phases of the paper's CUDA profile (allocate, copy in, kernel, copy out, free) with CUDA
events, and PHTL_LOG prints one line per tracking call."""
import os
import subprocess
import sys

import numpy as np
import pytest

import helpers
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("dtype", ["f64", "f32c"])
def test_track_host_phases_and_parity(dtype):
    n, turns = 200_003, 2000
    inp = helpers.inputs(n, seed=7, transverse=True)
    keys = ("z", "dp", "x", "xp", "y", "yp")
    host = [np.array(inp[k], dtype=np.float64, copy=True) if dtype == "f64" else phtl.split_f32c(inp[k])
            for k in keys]
    mon = np.zeros((turns // 10 + 1, phtl.MON_FIELDS))
    R = phtl.Ring(**inp["ring"])
    assert R.phase_times()["total_ms"] == 0.0  # nothing measured before the first call
    R.track_host(*host, turns=turns, integrator="leapfrog", dtype=dtype, mon_rows=mon,
                 mon_stride=10)
    p = R.phase_times()
    R.close()
    for k in ("alloc_ms", "h2d_ms", "kernel_ms", "d2h_ms", "free_ms", "total_ms", "wall_ms"):
        assert p[k] >= 0.0, (k, p)
    parts = p["alloc_ms"] + p["h2d_ms"] + p["kernel_ms"] + p["d2h_ms"] + p["free_ms"]
    assert abs(parts - p["total_ms"]) <= 1e-3 * p["total_ms"] + 0.05, p
    # 4e8 particle-turns: the kernels dominate, the copies are tens of MB
    assert p["kernel_ms"] > p["h2d_ms"] and p["kernel_ms"] > p["d2h_ms"], p
    assert p["wall_ms"] >= p["total_ms"] * 0.99, p
    assert p["h2d_bytes"] == 6 * 8 * n
    assert p["d2h_bytes"] == 6 * 8 * n + mon.nbytes
    assert p["launches"] >= 1
    # and the result is the oracle's
    got = [a if dtype == "f64" else phtl.join_f32c(a) for a in host]
    ref = oracle.track(inp["d"], "leapfrog", *[inp[k] for k in keys], turns=turns)
    err = helpers.rel_errors(inp["d"], list(ref[:6]), got, inp["z"], inp["dp"])
    assert np.max(err) < (1e-10 if dtype == "f64" else 1e-8)


def test_log_lines_on_stderr():
    code = (
        "import sys; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
        "import numpy as np, helpers\n"
        "from paper_1610_05801_gb300 import phtl\n"
        "inp = helpers.inputs(1000, seed=3, transverse=False)\n"
        "R = phtl.Ring(**inp['ring'])\n"
        "z, d = np.ascontiguousarray(inp['z']), np.ascontiguousarray(inp['dp'])\n"
        "R.track_host(z, d, turns=50, integrator='ruth4', dtype='f64')\n"
        "R.close()\n" % (ROOT, os.path.join(ROOT, "tests")))
    env = dict(os.environ, PHTL_LOG="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stderr.splitlines() if ln.startswith("phtl: ")]
    assert any(ln.startswith("phtl: track n=1000 turns=50 integrator=2 dtype=0") for ln in lines), lines
    assert any(ln.startswith("phtl: track_host alloc=") for ln in lines), lines
    env.pop("PHTL_LOG")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and "phtl: " not in r.stderr
