"""Thin ctypes binding of libphtl.so (C ABI in include/phtl.h).

Argument marshalling only: every step of the tracking runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams; tensors are passed as raw
device pointers.  There is no CPU fallback: if the library is missing or the GPU
is not an sm_103 device, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PHTL_LIB selects another build of the library (e.g. a compile-time variant)
LIB_PATH = os.environ.get("PHTL_LIB") or os.path.join(_HERE, "libphtl.so")

OK = 0
E_INVALID, E_UNSTABLE, E_NOMEM, E_CUDA, E_TIMEOUT, E_CANCELLED, E_BADHANDLE, E_NODEVICE = (
    -1, -2, -3, -4, -5, -6, -7, -8)
E_TOOBIG = -9
E_CAPTURE = -10
NOALLOC_MAX_JOBS = 256
EULER_CROMER, LEAPFROG, RUTH4, RK4 = 0, 1, 2, 3
F64, F32C, F32CD, F32CS = 0, 1, 2, 3
MON_FIELDS = 16
INTEGRATORS = {"euler_cromer": EULER_CROMER, "ec": EULER_CROMER, "leapfrog": LEAPFROG,
               "lf": LEAPFROG, "ruth4": RUTH4, "rk4": RK4}
DTYPES = {"f64": F64, "f32c": F32C, "f32cd": F32CD, "f32cs": F32CS}
MOMENT_NAMES = (
    "mean_z", "mean_dp", "rms_z", "rms_dp", "eps_z",
    "mean_x", "mean_xp", "rms_x", "rms_xp", "eps_x",
    "mean_y", "mean_yp", "rms_y", "rms_yp", "eps_y",
)


class PhtlError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


class Params(C.Structure):
    _fields_ = [("circumference_m", C.c_double), ("gamma_t", C.c_double), ("p0_eVc", C.c_double),
                ("mass_eV", C.c_double), ("charge_e", C.c_double), ("voltage_V", C.c_double),
                ("phi_s_rad", C.c_double), ("beta_x_m", C.c_double), ("beta_y_m", C.c_double),
                ("Qx", C.c_double), ("Qy", C.c_double), ("harmonic", C.c_int32),
                ("rf_linear", C.c_int32), ("eta1", C.c_double), ("eta2", C.c_double),
                ("xi_x", C.c_double), ("xi_y", C.c_double), ("voltage2_V", C.c_double),
                ("phi2_rad", C.c_double), ("harmonic2", C.c_int32), ("pad2_", C.c_int32)]


class Derived(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "betagamma", "gamma", "beta", "eta", "k", "A", "etaC", "sin_phis", "cos_phis", "K", "Qs",
        "bucket_half_length_m", "bucket_half_height")] + [("mx", C.c_double * 4),
                                                          ("my", C.c_double * 4)]


class Wake(C.Structure):
    _fields_ = [("z_lo", C.c_double), ("z_hi", C.c_double), ("alpha", C.c_double),
                ("alpha_sc", C.c_double), ("w", C.c_void_p), ("nslices", C.c_int32),
                ("pad_", C.c_int32)]


MAX_SLICES = 4096


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("particle_turns", C.c_int64), ("calls", C.c_int64),
                ("gate_launches", C.c_int64)]


class PhaseTimes(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("alloc_ms", "h2d_ms", "kernel_ms", "d2h_ms", "free_ms",
                                          "total_ms", "wall_ms")] + \
               [("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("launches", C.c_int64)]


class Job(C.Structure):
    _fields_ = [("c", C.c_void_p * 6), ("mon_rows", C.c_void_p), ("mon_capacity", C.c_int64),
                ("mon_stride", C.c_int64), ("n", C.c_int64), ("turns", C.c_int64),
                ("voltage_V", C.c_double), ("integrator", C.c_int32), ("dtype", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("pad_", C.c_int32), ("turns_per_launch", C.c_int64),
                ("particle_turns_per_s", C.c_double)]


class BatchInfo(C.Structure):
    _fields_ = [("njobs", C.c_int32), ("graph", C.c_int32), ("block_threads", C.c_int32 * 4),
                ("turns_per_launch", C.c_int64 * 4),
                ("probe_particle_turns_per_s", C.c_double * 4), ("launches_per_run", C.c_int64),
                ("tiles_first_launch", C.c_int64), ("particle_turns_per_run", C.c_int64)]


class ServerConfig(C.Structure):
    _fields_ = [("memory_budget_bytes", C.c_int64), ("max_active", C.c_int32),
                ("block_threads", C.c_int32), ("chunk_turns_f64", C.c_int64),
                ("chunk_turns_f32", C.c_int64), ("target_round_ms", C.c_double),
                ("policy", C.c_int32), ("waves", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("in_", C.c_void_p * 6), ("out", C.c_void_p * 6), ("mon_rows", C.c_void_p),
                ("mon_stride", C.c_int64), ("n", C.c_int64), ("turns", C.c_int64),
                ("voltage_V", C.c_double), ("integrator", C.c_int32), ("dtype", C.c_int32),
                ("resume_ticket", C.c_uint64), ("keep_resident", C.c_int32), ("pad_", C.c_int32)]


class Status(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("turns_done", C.c_int64),
                ("t_submit_ns", C.c_int64), ("t_admit_ns", C.c_int64), ("t_done_ns", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("submitted", "completed", "failed", "cancelled", "queued",
                                         "active", "bytes_in_use", "bytes_peak", "rounds",
                                         "launches")] + \
               [(n, C.c_double) for n in ("particle_turns", "busy_s", "p50_latency_s",
                                          "p99_latency_s", "mean_latency_s", "throughput_pts")]


QUEUED, RUNNING, DONE, FAILED, CANCELLED = 0, 1, 2, 3, 4
POLICY_SRPT, POLICY_SHARE = 0, 1

_lib = None
_lock = threading.Lock()
_vp, _i64, _int = C.c_void_p, C.c_int64, C.c_int

# name -> (restype, argtypes); every symbol include/phtl.h declares
SIGNATURES = {
    "phtl_create": (_int, [C.POINTER(Params), C.POINTER(_vp)]),
    "phtl_destroy": (_int, [_vp]),
    "phtl_get_derived": (_int, [_vp, C.POINTER(Derived)]),
    "phtl_strerror": (C.c_char_p, [_int]),
    "phtl_version": (C.c_char_p, []),
    "phtl_set_monitor": (_int, [_vp, _vp, _i64, _i64]),
    "phtl_set_tuning": (_int, [_vp, C.c_int32, _i64, C.c_int32]),
    "phtl_track": (_int, [_vp] + [_vp] * 6 + [_i64, _i64, _int, _int, _vp]),
    "phtl_track_perturn": (_int, [_vp] + [_vp] * 6 + [_i64, _i64, _int, _int, _vp]),
    "phtl_track_host": (_int, [_vp] + [_vp] * 6 + [_i64, _i64, _int, _int, _vp, _i64]),
    "phtl_moments_from_sums": (_int, [_vp, _vp]),
    "phtl_get_stats": (_int, [_vp, C.POINTER(Stats)]),
    "phtl_get_phase_times": (_int, [_vp, C.POINTER(PhaseTimes)]),
    "phtl_track_cancel": (_int, [_vp]),
    "phtl_track_status": (_int, [_vp, C.POINTER(C.c_int64)]),
    "phtl_eval_sin": (_int, [_vp, _vp, _i64, _int, _vp]),
    "phtl_eval_sin_kz": (_int, [C.c_double, _vp, _vp, _i64, _vp]),
    "phtl_set_programme": (_int, [_vp, _vp, _vp, _i64]),
    "phtl_track_programme": (_int, [_vp] + [_vp] * 6 + [_i64, _i64, _i64, _int, _int, _vp]),
    "phtl_set_wake": (_int, [_vp, C.POINTER(Wake)]),
    "phtl_collective_kick": (_int, [_vp, _vp, _vp, _i64, _int, _vp, _vp, _vp]),
    "phtl_track_collective": (_int, [_vp] + [_vp] * 6 + [_i64, _i64, _int, _int, _vp]),
    "phtl_autotune": (_int, [_vp, _int, _int, _i64, C.c_double, C.POINTER(Tuning)]),
    "phtl_batch_create": (_int, [_vp, C.POINTER(Job), C.c_int32, C.c_int32, C.POINTER(_vp)]),
    "phtl_batch_run": (_int, [_vp, _vp]),
    "phtl_batch_info_get": (_int, [_vp, C.POINTER(BatchInfo)]),
    "phtl_batch_destroy": (_int, [_vp]),
    "phtl_batch_run_noalloc": (_int, [_vp, C.POINTER(Job), C.c_int32, _vp]),
    "phtl_server_start": (_int, [_vp, C.POINTER(ServerConfig)]),
    "phtl_submit": (_int, [_vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "phtl_poll": (_int, [_vp, C.c_uint64, C.POINTER(Status)]),
    "phtl_wait": (_int, [_vp, C.c_uint64, _i64, C.POINTER(Status)]),
    "phtl_cancel": (_int, [_vp, C.c_uint64]),
    "phtl_release": (_int, [_vp, C.c_uint64]),
    "phtl_server_get_stats": (_int, [_vp, C.POINTER(ServerStats)]),
    "phtl_server_stop": (_int, [_vp]),
}


def load(path: str = LIB_PATH):
    """Load libphtl.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"{path} not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return load().phtl_strerror(int(code)).decode()
    except ImportError:
        return f"error {code}"


def _check(rc: int, what: str):
    if rc != OK:
        raise PhtlError(rc, what)


def make_params(**kw) -> Params:
    p = Params()
    defaults = dict(mass_eV=938.27208816e6, charge_e=1.0, phi_s_rad=0.0, beta_x_m=1.0,
                    beta_y_m=1.0, Qx=0.0, Qy=0.0, rf_linear=0, voltage_V=0.0)
    defaults.update(kw)
    for k, v in defaults.items():
        setattr(p, k, int(v) if k in ("harmonic", "rf_linear", "harmonic2") else float(v))
    return p


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(f"unsupported buffer type {type(t)}")


def _stream_ptr(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _integrator(i):
    return INTEGRATORS[i] if isinstance(i, str) else int(i)


def _dtype(d):
    return DTYPES[d] if isinstance(d, str) else int(d)


class Ring:
    """A phtl handle: ring/RF parameters plus derived FP64 constants (phtl_create)."""

    def __init__(self, **params):
        self._lib = load()
        self.params = make_params(**params)
        h = _vp()
        _check(self._lib.phtl_create(C.byref(self.params), C.byref(h)), "phtl_create")
        self._h = h
        self._monitor = None

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.phtl_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def derived(self) -> Derived:
        d = Derived()
        _check(self._lib.phtl_get_derived(self._h, C.byref(d)), "phtl_get_derived")
        return d

    def stats(self) -> Stats:
        st = Stats()
        _check(self._lib.phtl_get_stats(self._h, C.byref(st)), "phtl_get_stats")
        return st

    def cancel(self):
        """Stop the persistent tracking calls already enqueued on this ring at their next
        launch boundary (phtl_track_cancel); callable from any thread."""
        _check(self._lib.phtl_track_cancel(self._h), "phtl_track_cancel")

    def status(self):
        """(rc, turns_done) of the last tracking call once its stream work has completed:
        rc is OK, or E_CANCELLED when it was cut short (phtl_track_status)."""
        t = C.c_int64()
        rc = self._lib.phtl_track_status(self._h, C.byref(t))
        if rc not in (OK, E_CANCELLED):
            raise PhtlError(rc, "phtl_track_status")
        return rc, t.value

    def phase_times(self) -> dict:
        """Phase times (ms) of the last track_host call: alloc, h2d, kernel, d2h, free,
        total (CUDA events) and wall (host), with the bytes copied and the launches."""
        p = PhaseTimes()
        _check(self._lib.phtl_get_phase_times(self._h, C.byref(p)), "phtl_get_phase_times")
        return {name: getattr(p, name) for name, _ in PhaseTimes._fields_}

    def autotune(self, dtype="f32c", integrator="leapfrog", active_particles=1_000_000,
                 target_launch_ms=20.0) -> Tuning:
        t = Tuning()
        _check(self._lib.phtl_autotune(self._h, _dtype(dtype), _integrator(integrator),
                                       int(active_particles), float(target_launch_ms),
                                       C.byref(t)), "phtl_autotune")
        return t

    def set_tuning(self, block_threads: int = 0, turns_per_launch: int = 0, max_blocks: int = 0):
        _check(self._lib.phtl_set_tuning(self._h, int(block_threads), int(turns_per_launch),
                                         int(max_blocks)), "phtl_set_tuning")

    def set_monitor(self, rows=None, stride: int = 1):
        """rows: a CUDA float64 tensor of shape (capacity, 16), or None to detach."""
        if rows is None:
            _check(self._lib.phtl_set_monitor(self._h, None, 0, 1), "phtl_set_monitor")
            self._monitor = None
            return
        _check_tensor(rows, "float64", "monitor")
        assert rows.dim() == 2 and rows.shape[1] == MON_FIELDS
        _check(self._lib.phtl_set_monitor(self._h, rows.data_ptr(), rows.shape[0], int(stride)),
               "phtl_set_monitor")
        self._monitor = rows  # keep it alive while attached

    def _track(self, fn, z, dp, x, xp, y, yp, turns, integrator, dtype, stream):
        dt = _dtype(dtype)
        want = "float64" if dt == F64 else "float32"
        bufs = (z, dp, x, xp, y, yp)
        for name, b in zip(("z", "dp", "x", "xp", "y", "yp"), bufs):
            if b is not None:
                _check_tensor(b, want, name)
        n = z.numel() if dt == F64 else z.numel() // 2
        for b in bufs:
            if b is not None and b.numel() != z.numel():
                raise ValueError("all coordinate buffers must have the same length")
        rc = fn(self._h, *[_ptr(b) for b in bufs], n, int(turns), _integrator(integrator), dt,
                _stream_ptr(stream))
        _check(rc, fn.__name__)

    def track(self, z, dp, x=None, xp=None, y=None, yp=None, turns=1, integrator="leapfrog",
              dtype="f64", stream=None):
        """Persistent multi-turn tracking in place (phtl_track); stream-ordered."""
        self._track(self._lib.phtl_track, z, dp, x, xp, y, yp, turns, integrator, dtype, stream)

    def track_perturn(self, z, dp, x=None, xp=None, y=None, yp=None, turns=1,
                      integrator="leapfrog", dtype="f64", stream=None):
        """One launch per turn (phtl_track_perturn); stream-ordered."""
        self._track(self._lib.phtl_track_perturn, z, dp, x, xp, y, yp, turns, integrator, dtype,
                    stream)

    def set_programme(self, voltage_V=None, p0_eVc=None):
        """Attach a ramp programme (phtl_set_programme): voltage_V[n] for turns 0..N-1 and
        the reference momenta p0_eVc[0..N]; None detaches."""
        if voltage_V is None:
            _check(self._lib.phtl_set_programme(self._h, None, None, 0), "phtl_set_programme")
            return
        V = np.ascontiguousarray(voltage_V, dtype=np.float64)
        p0 = np.ascontiguousarray(p0_eVc, dtype=np.float64)
        if p0.shape[0] != V.shape[0] + 1:
            raise ValueError("p0_eVc needs one more entry than voltage_V")
        _check(self._lib.phtl_set_programme(self._h, V.ctypes.data, p0.ctypes.data, V.shape[0]),
               "phtl_set_programme")

    def track_programme(self, z, dp, x=None, xp=None, y=None, yp=None, turn0=0, turns=1,
                        integrator="leapfrog", dtype="f64", stream=None):
        """Track turns [turn0, turn0 + turns) of the attached programme
        (phtl_track_programme)."""
        dt = _dtype(dtype)
        want = "float64" if dt == F64 else "float32"
        bufs = (z, dp, x, xp, y, yp)
        for name, b in zip(("z", "dp", "x", "xp", "y", "yp"), bufs):
            if b is not None:
                _check_tensor(b, want, name)
        n = z.numel() if dt == F64 else z.numel() // 2
        rc = self._lib.phtl_track_programme(self._h, *[_ptr(b) for b in bufs], n, int(turn0),
                                            int(turns), _integrator(integrator), dt,
                                            _stream_ptr(stream))
        _check(rc, "phtl_track_programme")

    def set_wake(self, w=None, z_lo=0.0, z_hi=1.0, alpha=0.0, alpha_sc=0.0):
        """Attach a wake (phtl_set_wake): w[m] for m = 0..nslices-1 on the uniform slicing
        [z_lo, z_hi), kick alpha * V + alpha_sc * D (D: slope of the line density, the
        space-charge term); None detaches."""
        if w is None:
            _check(self._lib.phtl_set_wake(self._h, None), "phtl_set_wake")
            return
        wa = np.ascontiguousarray(w, dtype=np.float64)
        wk = Wake(float(z_lo), float(z_hi), float(alpha), float(alpha_sc), wa.ctypes.data,
                  wa.shape[0], 0)
        _check(self._lib.phtl_set_wake(self._h, C.byref(wk)), "phtl_set_wake")

    def collective_kick(self, z, dp, counts_out=None, V_out=None, dtype="f64", stream=None):
        """One collective step (slice, potential, kick) on device tensors z, dp (float64 for
        "f64", float32 [hi | comp] for the FP32 types); counts_out (int32/uint32 tensor) and
        V_out (float64 tensor) receive the step's counts and wake potential when given."""
        dt = _dtype(dtype)
        want = "float64" if dt == F64 else "float32"
        _check_tensor(z, want, "z")
        _check_tensor(dp, want, "dp")
        n = z.numel() if dt == F64 else z.numel() // 2
        rc = self._lib.phtl_collective_kick(self._h, _ptr(z), _ptr(dp), n, dt,
                                            _ptr(counts_out), _ptr(V_out), _stream_ptr(stream))
        _check(rc, "phtl_collective_kick")

    def track_collective(self, z, dp, x=None, xp=None, y=None, yp=None, turns=1,
                         integrator="leapfrog", dtype="f64", stream=None):
        """Turns of map + collective step (phtl_track_collective)."""
        self._track(self._lib.phtl_track_collective, z, dp, x, xp, y, yp, turns, integrator,
                    dtype, stream)

    def track_host(self, z, dp, x=None, xp=None, y=None, yp=None, turns=1,
                   integrator="leapfrog", dtype="f64", mon_rows=None, mon_stride=1):
        """End-to-end call on host buffers (numpy arrays or CPU tensors, ideally pinned):
        allocate, copy in, track, copy out, free (phtl_track_host); synchronous."""
        dt = _dtype(dtype)
        bufs = (z, dp, x, xp, y, yp)
        n = _numel(z) if dt == F64 else _numel(z) // 2
        rc = self._lib.phtl_track_host(self._h, *[_ptr(b) for b in bufs], n, int(turns),
                                       _integrator(integrator), dt, _ptr(mon_rows),
                                       int(mon_stride))
        _check(rc, "phtl_track_host")


def _numel(b):
    return b.numel() if hasattr(b, "numel") and callable(b.numel) else b.size


def _check_tensor(t, dtype: str, name: str):
    if not hasattr(t, "is_cuda") or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype}":
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def moments_from_sums(rows) -> np.ndarray:
    """Moments (mean, rms, emittance per plane; see MOMENT_NAMES) of monitor rows
    (array-like (..., 16) of raw sums) via phtl_moments_from_sums."""
    lib = load()
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.float64)).reshape(-1, MON_FIELDS)
    out = np.zeros((r.shape[0], 15))
    for i in range(r.shape[0]):
        _check(lib.phtl_moments_from_sums(r[i].ctypes.data, out[i].ctypes.data),
               "phtl_moments_from_sums")
    return out.reshape(np.asarray(rows).shape[:-1] + (15,))


def split_f32c(a: np.ndarray) -> np.ndarray:
    """FP64 values -> the FP32C layout [hi(n) | comp(n)] (hi = nearest float, comp = rest)."""
    a = np.asarray(a, dtype=np.float64)
    hi = a.astype(np.float32)
    lo = (a - hi.astype(np.float64)).astype(np.float32)
    return np.concatenate([hi, lo])


def join_f32c(b) -> np.ndarray:
    """FP32C layout [hi | comp] -> FP64 values hi + comp."""
    b = np.asarray(b, dtype=np.float32)
    n = b.shape[0] // 2
    return b[:n].astype(np.float64) + b[n:].astype(np.float64)


def eval_sin(x, which: int = 0, stream=None):
    """Device sine of a CUDA float64 tensor: which=0 the library's FP64 sine, 1 CUDA's."""
    import torch

    _check_tensor(x, "float64", "x")
    y = torch.empty_like(x)
    _check(load().phtl_eval_sin(x.data_ptr(), y.data_ptr(), x.numel(), int(which),
                                _stream_ptr(stream)), "phtl_eval_sin")
    return y


def eval_sin_kz(k: float, z, stream=None):
    """sin(k z) of a CUDA float64 tensor through the phi_s = 0 kick's fused form."""
    import torch

    _check_tensor(z, "float64", "z")
    y = torch.empty_like(z)
    _check(load().phtl_eval_sin_kz(float(k), z.data_ptr(), y.data_ptr(), z.numel(),
                                   _stream_ptr(stream)), "phtl_eval_sin_kz")
    return y


def make_job(z, dp, x=None, xp=None, y=None, yp=None, turns=1, voltage_V=None,
             integrator="leapfrog", dtype="f32c", monitor=None, stride=1) -> dict:
    """A batch job description (buffers are CUDA tensors; monitor a (rows, 16) float64
    tensor or None)."""
    return dict(c=[z, dp, x, xp, y, yp], turns=int(turns), voltage_V=voltage_V,
                integrator=integrator, dtype=dtype, monitor=monitor, stride=int(stride))


def job_array(ring: Ring, jobs):
    """phtl_job array for a list of make_job() dicts; returns (array, tensors to keep alive)."""
    keep = []
    arr = (Job * max(1, len(jobs)))()
    for i, j in enumerate(jobs):
        dt = _dtype(j["dtype"])
        want = "float64" if dt == F64 else "float32"
        for b in j["c"]:
            if b is not None:
                _check_tensor(b, want, "job buffer")
                keep.append(b)
        z = j["c"][0]
        n = z.numel() if dt == F64 else z.numel() // 2
        for k in range(6):
            arr[i].c[k] = _ptr(j["c"][k])
        mon = j.get("monitor")
        if mon is not None:
            _check_tensor(mon, "float64", "monitor")
            keep.append(mon)
            arr[i].mon_rows = mon.data_ptr()
            arr[i].mon_capacity = mon.shape[0]
            arr[i].mon_stride = int(j.get("stride", 1))
        arr[i].n = n
        arr[i].turns = int(j["turns"])
        v = j.get("voltage_V")
        arr[i].voltage_V = float(ring.params.voltage_V if v is None else v)
        arr[i].integrator = _integrator(j["integrator"])
        arr[i].dtype = dt
    return arr, keep


def batch_run_noalloc(ring: Ring, jobs, stream=None):
    """One run of `jobs` through phtl_batch_run_noalloc (no device allocation; the job
    table goes into the library's fixed device array).  Stream-ordered."""
    arr, _keep = job_array(ring, jobs)
    _check(load().phtl_batch_run_noalloc(ring.handle, arr, len(jobs), _stream_ptr(stream)),
           "phtl_batch_run_noalloc")


class Batch:
    """Many independent bunches tracked by shared, graph-captured launches
    (phtl_batch_create / phtl_batch_run)."""

    def __init__(self, ring: Ring, jobs, use_graph: bool = True):
        self._lib = load()
        self._ring = ring
        arr, self._keep = job_array(ring, jobs)
        self._jobs = arr
        h = _vp()
        _check(self._lib.phtl_batch_create(ring.handle, arr, len(jobs), 1 if use_graph else 0,
                                           C.byref(h)), "phtl_batch_create")
        self._h = h

    def run(self, stream=None):
        _check(self._lib.phtl_batch_run(self._h, _stream_ptr(stream)), "phtl_batch_run")

    def info(self) -> BatchInfo:
        b = BatchInfo()
        _check(self._lib.phtl_batch_info_get(self._h, C.byref(b)), "phtl_batch_info_get")
        return b

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.phtl_batch_destroy(self._h)
            self._h = _vp()
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The continuous-batching serving loop of a Ring (phtl_server_start ...).

    Requests carry host arrays (numpy, C-contiguous; float64 for "f64", float32 with the
    [hi | comp] layout for the FP32C types); results are written to `out` arrays (by
    default the inputs, in place) before the job turns DONE."""

    def __init__(self, ring: Ring, memory_budget_bytes=0, max_active=0, block_threads=0,
                 chunk_turns_f64=0, chunk_turns_f32=0, target_round_ms=0.0, policy="srpt",
                 waves=0):
        self._lib = load()
        self._ring = ring
        pol = {"srpt": POLICY_SRPT, "share": POLICY_SHARE}[policy] if isinstance(policy, str) else int(policy)
        cfg = ServerConfig(int(memory_budget_bytes), int(max_active), int(block_threads),
                           int(chunk_turns_f64), int(chunk_turns_f32), float(target_round_ms), pol,
                           int(waves))
        _check(self._lib.phtl_server_start(ring.handle, C.byref(cfg)), "phtl_server_start")
        self._keep = {}
        self._running = True

    def submit(self, z=None, dp=None, x=None, xp=None, y=None, yp=None, turns=1, voltage_V=None,
               integrator="leapfrog", dtype="f64", out=None, monitor=None, stride=1, n=None,
               resume=0, keep_resident=False) -> int:
        dt = _dtype(dtype)
        ins = [z, dp, x, xp, y, yp]
        outs = list(out) if out is not None else ins
        r = Request()
        for k in range(6):
            r.in_[k] = _ptr(ins[k]) if not resume else None
            r.out[k] = _ptr(outs[k])
        if n is None:
            ref = outs[0] if outs[0] is not None else ins[0]
            n = _numel(ref) if dt == F64 else _numel(ref) // 2
        r.n = int(n)
        r.turns = int(turns)
        r.voltage_V = float(self._ring.params.voltage_V if voltage_V is None else voltage_V)
        r.integrator = _integrator(integrator)
        r.dtype = dt
        if monitor is not None:
            r.mon_rows = _ptr(monitor)
            r.mon_stride = int(stride)
        r.resume_ticket = int(resume)
        r.keep_resident = 1 if keep_resident else 0
        t = C.c_uint64()
        _check(self._lib.phtl_submit(self._ring.handle, C.byref(r), C.byref(t)), "phtl_submit")
        self._keep[t.value] = (ins, outs, monitor)
        return t.value

    def poll(self, ticket) -> Status:
        st = Status()
        _check(self._lib.phtl_poll(self._ring.handle, int(ticket), C.byref(st)), "phtl_poll")
        return st

    def wait(self, ticket, timeout_ms=60000):
        """Returns (rc, Status): rc == OK when final, E_TIMEOUT otherwise."""
        st = Status()
        rc = self._lib.phtl_wait(self._ring.handle, int(ticket), int(timeout_ms), C.byref(st))
        if rc not in (OK, E_TIMEOUT):
            raise PhtlError(rc, "phtl_wait")
        if rc == OK and st.state != RUNNING:
            self._keep.pop(int(ticket), None)
        return rc, st

    def cancel(self, ticket):
        return self._lib.phtl_cancel(self._ring.handle, int(ticket))

    def release(self, ticket):
        _check(self._lib.phtl_release(self._ring.handle, int(ticket)), "phtl_release")

    def stats(self) -> ServerStats:
        s = ServerStats()
        _check(self._lib.phtl_server_get_stats(self._ring.handle, C.byref(s)), "phtl_server_get_stats")
        return s

    def stop(self):
        if self._running:
            self._lib.phtl_server_stop(self._ring.handle)
            self._running = False
            self._keep = {}
