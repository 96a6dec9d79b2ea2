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


def _sin_kz_reference(k, z):
    """sin(k z) of the exact product k z: Dekker's two-product (Veltkamp split, exact in
    FP64 without FMA) gives k z = p + e, then sin(p + e) ~ sin p + e cos p."""
    def split(a):
        c = 134217729.0 * a
        hi = c - (c - a)
        return hi, a - hi
    p = k * z
    kh, kl = split(np.full_like(z, k))
    zh, zl = split(z)
    e = ((kh * zh - p) + kh * zl + kl * zh) + kl * zl
    return np.sin(p) + e * np.cos(p), p


def test_fused_sin_kz_of_the_phi_s_zero_kick():
    """sin(k z) with the product folded into the reduction (the phi_s = 0 kick): within a
    few ulp of the sine of the exact product, across the bucket, far outside it, through
    the fallback range, and NaN for non-finite z."""
    k = 2 * math.pi * 4620 / 6911.5038
    rng = np.random.default_rng(5)
    zb = math.pi / k
    parts = [np.linspace(-3 * zb, 3 * zb, 300001), rng.uniform(-1, 1, 100000) * 1400.0,
             rng.uniform(-1e-6, 1e-6, 20000),
             np.array([0.0, -0.0, 1e-300, -1e-300, zb, -zb, zb / 2, 5e-324])]
    z = np.concatenate(parts)
    t = torch.tensor(z, dtype=torch.float64, device="cuda:0")
    own = phtl.eval_sin_kz(k, t).cpu().numpy()
    ref, p = _sin_kz_reference(k, z)
    assert np.max(np.abs(own - ref)) <= 4 * 2.0 ** -53, np.max(np.abs(own - ref))
    big = np.abs(ref) > 1e-3
    assert np.max(np.abs(own[big] / ref[big] - 1)) < 4e-15
    tiny = (np.abs(p) < 1e-3) & (np.abs(p) > 1e-290)
    assert np.max(np.abs(own[tiny] / ref[tiny] - 1)) < 3e-16
    # particles that have left the bucket: the fused form holds to |k z| ~ 1e5 (quadrant
    # below 2^16); the reduction's q L term then carries L's own rounding times q, a few
    # ulp more
    out = rng.uniform(-1, 1, 200000) * 1.0e5 / k
    own_out = phtl.eval_sin_kz(k, torch.tensor(out, dtype=torch.float64, device="cuda:0")).cpu().numpy()
    ref_out, _ = _sin_kz_reference(k, out)
    assert np.max(np.abs(own_out - ref_out)) <= 8 * 2.0 ** -53, np.max(np.abs(own_out - ref_out))
    # beyond the fused range the kick uses the plain sine of the rounded product: bitwise
    # what phtl_eval_sin gives for k * z
    far = np.array([1.1e5, -2e5, 5e5, -1e6, 3e7, 1e300]) / k
    own_far = phtl.eval_sin_kz(k, torch.tensor(far, dtype=torch.float64, device="cuda:0")).cpu().numpy()
    ref_far = phtl.eval_sin(torch.tensor(k * far, dtype=torch.float64, device="cuda:0"), 0).cpu().numpy()
    assert np.array_equal(own_far, ref_far)
    bad = phtl.eval_sin_kz(k, torch.tensor([np.inf, -np.inf, np.nan], dtype=torch.float64,
                                           device="cuda:0")).cpu().numpy()
    assert np.all(np.isnan(bad))


def _float_pair_value(x):
    """The value of the float pair the double-float sine receives: x with its significand
    cut to 24 bits for the head and the next 24 significant bits for the tail (both
    truncated, as the device's integer split does)."""
    b = x.view(np.uint64)
    m29 = b & np.uint64(0x1FFFFFFF)
    msb = np.zeros(len(x), dtype=np.int64)
    nz = m29 != 0
    msb[nz] = np.floor(np.log2(m29[nz].astype(np.float64))).astype(np.int64)
    drop = np.maximum(msb - 23, 0).astype(np.uint64)
    kept = (m29 >> drop) << drop
    return ((b & ~np.uint64(0x1FFFFFFF)) | kept).view(np.float64)


def test_double_float_sine_of_the_f32c_kicks():
    """The double-float sine (FP32C / FP32CD kicks) against the FP64 sine of the exact pair
    value.  Bounds from its arithmetic: <= 4e-12 absolute on the bucket's phase range
    (|x| <= 2 pi: the trailing Horner terms are summed in FP32 and contribute up to
    |r^3 t tail| <= 6e-5, so 6e-5 * 2^-24 ~ 4e-12; the double-float steps ~1e-14),
    <= 1e-10 for |x| <= 1e3 (the FP32 reduction remainder grows with the quadrant q)."""
    rng = np.random.default_rng(7)
    near = np.concatenate([np.linspace(-2 * math.pi, 2 * math.pi, 200001),
                           rng.uniform(-1e-4, 1e-4, 20000), np.array([0.0, math.pi / 4, 1e-30])])
    far = rng.uniform(-1e3, 1e3, 100000)
    for x, bound in ((near, 4e-12), (far, 1e-10)):
        got = phtl.eval_sin(torch.tensor(x, dtype=torch.float64, device="cuda:0"), 2).cpu().numpy()
        ref = np.sin(_float_pair_value(x))
        err = np.max(np.abs(got - ref))
        assert err <= bound, (err, bound)
    assert phtl.eval_sin(torch.tensor([0.0], dtype=torch.float64, device="cuda:0"), 2).item() == 0.0
