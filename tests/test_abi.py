"""The C ABI on the host (no GPU): the library loads, exports every function that
include/phtl.h declares, validates parameters, derives the same FP64 constants as the
oracle (both written from the same definitions), converts monitor sums to moments,
and refuses to compute without an sm_103 device instead of falling back to the CPU."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1610_05801_gb300 import phtl, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "phtl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(phtl_\w+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1610_05801_gb300 import build

    build.build()
    lib = C.CDLL(phtl.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared functions
    assert set(names) == set(phtl.SIGNATURES), set(names) ^ set(phtl.SIGNATURES)


def test_version_and_strerror():
    lib = phtl.load()
    assert b"sm_103a" in lib.phtl_version()
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10):
        assert lib.phtl_strerror(code) != b"unknown error code", code
    assert lib.phtl_strerror(-99) == b"unknown error code"


def _create(**kw):
    p = phtl.make_params(**kw)
    h = C.c_void_p()
    rc = phtl.load().phtl_create(C.byref(p), C.byref(h))
    return rc, h


def test_create_validation():
    base = dict(synth.ring(2e6))
    rc, h = _create(**base)
    assert rc == phtl.OK
    lib = phtl.load()
    assert lib.phtl_destroy(h) == phtl.OK
    assert lib.phtl_destroy(h) == phtl.E_BADHANDLE           # double destroy
    assert lib.phtl_destroy(None) == phtl.E_BADHANDLE
    assert lib.phtl_get_derived(None, None) == phtl.E_BADHANDLE
    for bad in (dict(circumference_m=0.0), dict(p0_eVc=-1.0), dict(harmonic=0),
                dict(mass_eV=float("nan")), dict(beta_x_m=0.0), dict(gamma_t=0.0)):
        rc, h = _create(**dict(base, **bad))
        assert rc == phtl.E_INVALID, bad
    # below transition the phi_s = 0 bucket is unstable; phi_s = pi is stable
    rc, _ = _create(**dict(base, p0_eVc=10e9))
    assert rc == phtl.E_UNSTABLE
    rc, h = _create(**dict(base, p0_eVc=10e9, phi_s_rad=math.pi))
    assert rc == phtl.OK
    lib.phtl_destroy(h)
    # K >= 4 (no oscillation) is unstable too
    rc, _ = _create(**dict(base, voltage_V=1e10))
    assert rc == phtl.E_UNSTABLE
    assert lib.phtl_create(None, None) == phtl.E_INVALID


def test_double_rf_validation_and_strength():
    """A second RF system: harmonic2 must be positive when voltage2 is set, the combined
    linear strength K = eta C (A k cos phi_s + A2 k2 cos phi2) equals the oracle's, a
    flat bottom (K = 0) is accepted and an over-cancelling system is unstable -- for the
    handle and for a batched job's own voltage."""
    base = dict(synth.ring(4.5e6), harmonic2=2 * 4620, voltage2_V=1.35e6, phi2_rad=0.0)
    lib = phtl.load()
    rc, _ = _create(**dict(base, harmonic2=0))
    assert rc == phtl.E_INVALID
    for bad in (dict(voltage2_V=float("nan")), dict(phi2_rad=float("inf"))):
        rc, _ = _create(**dict(base, **bad))
        assert rc == phtl.E_INVALID, bad
    for ratio, phi2 in ((0.3, 0.0), (0.3, -0.4), (-0.5, 0.0)):
        ring = dict(base, voltage2_V=ratio * 4.5e6, phi2_rad=phi2)
        R = phtl.Ring(**ring)
        a, b = R.derived(), oracle.derive(ring)
        assert math.isclose(a.K, b.K, rel_tol=1e-13, abs_tol=1e-18), (ratio, a.K, b.K)
        R.close()
    rc, _ = _create(**dict(base, voltage2_V=-0.7 * 4.5e6))
    assert rc == phtl.E_UNSTABLE
    assert oracle.derive_rc(oracle.params(**dict(base, voltage2_V=-0.7 * 4.5e6))) == -2
    # a batched job whose own voltage over-cancels against the ring's second system
    R = phtl.Ring(**dict(base, voltage2_V=-0.3 * 4.5e6))
    z = np.zeros(8)
    J = (phtl.Job * 1)()
    J[0].c[0] = J[0].c[1] = z.ctypes.data
    J[0].n, J[0].turns, J[0].integrator, J[0].dtype = 8, 10, phtl.RK4, 0
    h = C.c_void_p()
    J[0].voltage_V = 1e6          # 1 MV - 1.35 MV at twice the harmonic: K < 0
    assert lib.phtl_batch_create(R.handle, J, 1, 1, C.byref(h)) == phtl.E_UNSTABLE
    J[0].integrator = 4
    assert lib.phtl_batch_create(R.handle, J, 1, 1, C.byref(h)) == phtl.E_INVALID
    R.close()


def test_programme_validation_needs_no_gpu():
    """phtl_set_programme checks the programme before it looks for a device: bad arrays
    and unstable turns are reported here; a valid programme then needs the GPU."""
    lib = phtl.load()
    R = phtl.Ring(**synth.ring(4.5e6))
    N = 100
    V = np.full(N, 4.5e6)
    p0 = 26e9 + 1e6 * np.arange(N + 1)

    def setp(V, p0, n=N):
        return lib.phtl_set_programme(R.handle, V.ctypes.data, p0.ctypes.data, n)

    assert lib.phtl_set_programme(R.handle, None, None, 5) == phtl.E_INVALID
    assert lib.phtl_set_programme(None, None, None, 0) == phtl.E_BADHANDLE
    bad = p0.copy()
    bad[7] = -1.0
    assert setp(V, bad) == phtl.E_INVALID
    bad = V.copy()
    bad[3] = 0.0                                             # no voltage, momentum changes
    assert setp(bad, p0) == phtl.E_INVALID
    assert setp(np.full(N, 1e5), p0) == phtl.E_UNSTABLE      # too little voltage for the gain
    assert lib.phtl_set_programme(R.handle, None, None, 0) == phtl.OK    # detach: no device needed
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert setp(V, p0) == phtl.E_NODEVICE
    R.close()
    # the programme runs the linear map only
    R = phtl.Ring(**synth.ring(4.5e6, eta1=0.05))
    assert lib.phtl_set_programme(R.handle, V.ctypes.data, p0.ctypes.data, N) == phtl.E_INVALID
    R.close()


def test_wake_validation_needs_no_gpu():
    """phtl_set_wake checks its arguments before it looks for a device."""
    lib = phtl.load()
    R = phtl.Ring(**synth.ring(4.5e6))
    w = np.ones(16)

    def setw(**over):
        kw = dict(z_lo=-0.5, z_hi=0.5, alpha=1e-6, w=w.ctypes.data, nslices=16, pad_=0)
        kw.update(over)
        wk = phtl.Wake(**kw)
        return lib.phtl_set_wake(R.handle, C.byref(wk))

    assert setw(nslices=0) == phtl.E_INVALID
    assert setw(nslices=phtl.MAX_SLICES + 1) == phtl.E_INVALID
    assert setw(z_hi=-0.5) == phtl.E_INVALID
    assert setw(alpha=float("nan")) == phtl.E_INVALID
    assert setw(alpha_sc=float("inf")) == phtl.E_INVALID
    assert setw(w=None) == phtl.E_INVALID
    bad = w.copy()
    bad[3] = float("inf")
    assert setw(w=bad.ctypes.data) == phtl.E_INVALID
    assert lib.phtl_set_wake(R.handle, None) == phtl.OK          # detach: nothing attached
    assert lib.phtl_set_wake(None, None) == phtl.E_BADHANDLE
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert setw() == phtl.E_NODEVICE
        z = np.zeros(8)
        assert lib.phtl_track_collective(R.handle, z.ctypes.data, z.ctypes.data, None, None, None,
                                         None, 8, 1, 1, 0, None) == phtl.E_NODEVICE
    R.close()


def test_derived_constants_match_oracle():
    for V in (2e6, 4.5e6):
        ring = synth.ring(V, transverse=True)
        R = phtl.Ring(**ring)
        a = R.derived()
        b = oracle.derive(ring)
        for name in ("betagamma", "gamma", "beta", "eta", "k", "A", "etaC", "K", "Qs"):
            assert math.isclose(getattr(a, name), getattr(b, name), rel_tol=1e-15), name
        assert list(a.mx) == list(b.mx) and list(a.my) == list(b.my)
        assert math.isclose(a.bucket_half_length_m, math.pi / b.k, rel_tol=1e-15)
        R.close()


def test_set_monitor_and_tuning_validation():
    R = phtl.Ring(**synth.ring(2e6))
    lib = phtl.load()
    h = R.handle
    buf = (C.c_double * 32)()
    assert lib.phtl_set_monitor(h, C.addressof(buf), 0, 1) == phtl.E_INVALID
    assert lib.phtl_set_monitor(h, C.addressof(buf), 2, 0) == phtl.E_INVALID
    assert lib.phtl_set_monitor(h, C.addressof(buf) + 4, 2, 1) == phtl.E_INVALID
    assert lib.phtl_set_monitor(h, None, 0, 0) == phtl.OK
    assert lib.phtl_set_tuning(h, 48, 0, 0) == phtl.E_INVALID
    assert lib.phtl_set_tuning(h, 512, 0, 0) == phtl.E_INVALID
    assert lib.phtl_set_tuning(h, 128, -1, 0) == phtl.E_INVALID
    assert lib.phtl_set_tuning(h, 128, 0, -1) == phtl.E_INVALID
    assert lib.phtl_set_tuning(h, 128, 100, 3) == phtl.OK
    assert lib.phtl_set_tuning(None, 0, 0, 0) == phtl.E_BADHANDLE
    R.close()


def test_track_argument_validation_needs_no_gpu():
    """Argument errors are reported before any device work."""
    R = phtl.Ring(**synth.ring(2e6))
    lib = phtl.load()
    h = R.handle
    z = np.zeros(8)
    p = z.ctypes.data
    args = lambda **k: dict(dict(z=p, dp=p, x=None, xp=None, y=None, yp=None, n=8, turns=10,
                                 integ=1, dt=0, s=None), **k)

    def call(a):
        return lib.phtl_track(h, a["z"], a["dp"], a["x"], a["xp"], a["y"], a["yp"], a["n"],
                              a["turns"], a["integ"], a["dt"], a["s"])

    assert call(args(integ=4)) == phtl.E_INVALID
    assert call(args(integ=-1)) == phtl.E_INVALID
    assert call(args(dt=7)) == phtl.E_INVALID
    assert call(args(n=-1)) == phtl.E_INVALID
    assert call(args(turns=-5)) == phtl.E_INVALID
    assert call(args(z=None)) == phtl.E_INVALID
    assert call(args(x=p)) == phtl.E_INVALID                 # x without x'
    assert call(args(z=p + 4)) == phtl.E_INVALID             # misaligned double
    assert lib.phtl_track(None, p, p, None, None, None, None, 8, 1, 1, 0, None) == phtl.E_BADHANDLE
    R.close()


def test_track_without_device_fails_loudly():
    """No CUDA device here: the library must refuse (no CPU fallback)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    R = phtl.Ring(**synth.ring(2e6))
    z = np.zeros(8)
    rc = phtl.load().phtl_track(R.handle, z.ctypes.data, z.ctypes.data, None, None, None, None,
                                8, 10, 1, 0, None)
    assert rc == phtl.E_NODEVICE
    R.close()


def test_moments_from_sums_matches_numpy():
    rng = np.random.default_rng(3)
    n = 777
    cols = [rng.normal(0.01, 0.2, n), rng.normal(-1e-4, 1e-3, n)]
    cols[1] = cols[1] + 0.003 * cols[0]
    x, xp = rng.normal(0, 1e-3, n), rng.normal(0, 3e-5, n)
    y, yp = rng.normal(0, 2e-3, n), rng.normal(0, 1e-5, n)
    row = [n]
    for a, b in ((cols[0], cols[1]), (x, xp), (y, yp)):
        row += [a.sum(), b.sum(), (a * a).sum(), (b * b).sum(), (a * b).sum()]
    m = phtl.moments_from_sums(np.array(row))
    ref = oracle.moments(cols[0], cols[1], x, xp, y, yp)
    assert np.allclose(m, ref, rtol=1e-9, atol=1e-15)
    assert np.all(phtl.moments_from_sums(np.zeros(16)) == 0)


def test_f32c_split_roundtrip():
    a = np.random.default_rng(1).normal(0, 0.3, 1001)
    b = phtl.split_f32c(a)
    assert b.dtype == np.float32 and b.shape == (2002,)
    assert np.max(np.abs(phtl.join_f32c(b) - a) / np.abs(a)) < 1e-14


def test_batch_validation_needs_no_gpu():
    """Job errors are reported before any device work."""
    R = phtl.Ring(**synth.ring(2e6))
    lib = phtl.load()
    z = np.zeros(8)
    p = z.ctypes.data

    def create(**over):
        J = (phtl.Job * 1)()
        J[0].c[0] = p
        J[0].c[1] = p
        J[0].n = 8
        J[0].turns = 10
        J[0].voltage_V = 2e6
        J[0].integrator = 1
        J[0].dtype = 0
        for k, v in over.items():
            setattr(J[0], k, v)
        h = C.c_void_p()
        return lib.phtl_batch_create(R.handle, J, 1, 1, C.byref(h))

    assert create(integrator=5) == phtl.E_INVALID
    assert create(dtype=9) == phtl.E_INVALID
    assert create(n=-1) == phtl.E_INVALID
    assert create(voltage_V=float("inf")) == phtl.E_INVALID
    assert create(voltage_V=1e10) == phtl.E_UNSTABLE      # K >= 4
    assert create(voltage_V=-2e6) == phtl.E_UNSTABLE      # wrong-sign bucket
    assert create(mon_rows=p, mon_capacity=2, mon_stride=1) == phtl.E_INVALID  # too few rows
    h = C.c_void_p()
    assert lib.phtl_batch_create(None, None, 0, 1, C.byref(h)) == phtl.E_BADHANDLE
    assert lib.phtl_batch_create(R.handle, None, 1, 1, C.byref(h)) == phtl.E_INVALID
    assert lib.phtl_batch_run(None, None) == phtl.E_BADHANDLE
    assert lib.phtl_batch_destroy(None) == phtl.E_BADHANDLE
    R.close()


def test_server_config_validation_without_a_gpu():
    """A bad serving configuration is refused before any device work: negative budget, slots,
    chunk turns, round target or SRPT wave cap, an unknown policy, an odd block size."""
    lib = phtl.load()
    rc, h = _create(**dict(synth.ring(2e6)))
    assert rc == phtl.OK
    good = dict(memory_budget_bytes=0, max_active=0, block_threads=0, chunk_turns_f64=0,
                chunk_turns_f32=0, target_round_ms=0.0, policy=0, waves=0)
    for field, bad in (("memory_budget_bytes", -1), ("max_active", -1), ("chunk_turns_f64", -5),
                       ("chunk_turns_f32", -5), ("target_round_ms", -1.0), ("waves", -1),
                       ("policy", 7), ("block_threads", 100)):
        cfg = phtl.ServerConfig(**dict(good, **{field: bad}))
        assert lib.phtl_server_start(h, C.byref(cfg)) == phtl.E_INVALID, field
    assert lib.phtl_destroy(h) == phtl.OK
