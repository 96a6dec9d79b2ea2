"""The library's own FP64 sine (Cody-Waite reduction + fitted polynomial) against CUDA's
sin() and against 30-digit mpmath values: a few ulp on the kick's argument range."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1610_05801_gb300 import phtl  # noqa: E402


def _args():
    rng = np.random.default_rng(0)
    parts = [np.linspace(-4 * math.pi, 4 * math.pi, 400001),
             rng.uniform(-1e5, 1e5, 200000),
             rng.uniform(-1e-3, 1e-3, 50000),
             np.array([0.0, -0.0, 1e-300, -1e-300, math.pi, -math.pi, math.pi / 2, 1e5 - 1,
                       1e5, 1e6, -3e7, 1e300, np.inf, -np.inf, np.nan])]
    return np.concatenate(parts)


def test_own_sine_vs_cuda_sine():
    x = _args()
    t = torch.tensor(x, dtype=torch.float64, device="cuda:0")
    own = phtl.eval_sin(t, 0).cpu().numpy()
    ref = phtl.eval_sin(t, 1).cpu().numpy()
    fin = np.isfinite(x)
    assert np.all(np.isnan(own[~fin]))
    assert np.all(own[x == 0.0] == 0.0)  # the sign of a zero result is not preserved
    small = fin & (np.abs(x) < 1e5)
    absdiff = np.abs(own[small] - ref[small])
    assert np.max(absdiff) <= 4 * 2.0 ** -53, np.max(absdiff)   # <= 4 ulp of 1
    big = np.abs(ref[small]) > 1e-3
    rel = np.abs(own[small][big] / ref[small][big] - 1)
    assert np.max(rel) < 4e-15, np.max(rel)
    tiny = fin & (np.abs(x) < 1e-3) & (x != 0)
    assert np.max(np.abs(own[tiny] / ref[tiny] - 1)) < 3e-16
    # beyond 1e5 the library falls back to CUDA's sine: identical
    far = fin & (np.abs(x) >= 1e5)
    assert np.array_equal(own[far], ref[far])


def test_own_sine_vs_mpmath():
    mp = pytest.importorskip("mpmath")
    x = np.random.default_rng(1).uniform(-math.pi, math.pi, 3000)
    own = phtl.eval_sin(torch.tensor(x, dtype=torch.float64, device="cuda:0"), 0).cpu().numpy()
    with mp.workdps(30):
        exact = np.array([float(mp.sin(mp.mpf(v))) for v in x])
    ulp = np.spacing(np.abs(exact))
    assert np.max(np.abs(own - exact) / ulp) <= 4
