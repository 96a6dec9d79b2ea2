"""Plain FP64 reference tracker -- TEST INFRASTRUCTURE, not the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (``paper_1610_05801_gb300``)
never imports it and shares no code with it.

The arithmetic lives in ``oracle/track_ref.c`` (plain C, FP64, compiled with
``-O2 -ffp-contract=off``); this module only compiles it with gcc, loads it with
ctypes and marshals numpy arrays.  What the C file computes, and which passage
of the paper each part follows, is stated in its header: the turn-by-turn
longitudinal map (Sec. 1.1.2: Euler-Cromer, leap-frog, 4th-order Ruth), the
linear transverse transfer matrix (Sec. 1.1.1) and per-turn bunch moments.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "track_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libphtl_oracle.so")
_lock = threading.Lock()
_lib = None

EULER_CROMER, LEAPFROG, RUTH4, RK4 = 0, 1, 2, 3
SCHEMES = {"euler_cromer": EULER_CROMER, "leapfrog": LEAPFROG, "ruth4": RUTH4, "rk4": RK4}
NMOM = 15
# per-turn constants of a ramp programme: eta_n C, A_n, phi_s,n, sin(phi_s,n),
# r_n = p0_n / p0_{n+1}, beta_n gamma_n
RAMP_NC = 6
MOMENT_NAMES = (
    "mean_z", "mean_dp", "rms_z", "rms_dp", "eps_z",
    "mean_x", "mean_xp", "rms_x", "rms_xp", "eps_x",
    "mean_y", "mean_yp", "rms_y", "rms_yp", "eps_y",
)


class RefParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "circumference_m", "gamma_t", "p0_eVc", "mass_eV", "charge_e", "harmonic",
        "voltage_V", "phi_s_rad", "rf_linear", "beta_x_m", "beta_y_m", "Qx", "Qy",
        "eta1", "eta2", "xi_x", "xi_y", "harmonic2", "voltage2_V", "phi2_rad")]


class RefDerived(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "betagamma", "gamma", "beta", "eta", "k", "A", "etaC", "phi_s", "sin_phis",
        "cos_phis", "K", "Qs", "rf_linear")] + [("mx", C.c_double * 4), ("my", C.c_double * 4)] + [
        (n, C.c_double) for n in ("eta1C", "eta2C", "qx", "qy", "bx", "by", "xi_x", "xi_y",
                                  "k2", "A2", "phi2", "sin_phi2", "cos_phi2")]


def build(openmp: bool = True, force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the C oracle into a shared library (gcc, -O2 -ffp-contract=off)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           src, "-o", tmp, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError as e:
        if openmp:  # a toolchain without OpenMP still gets the serial oracle
            return build(openmp=False, force=True, src=src, out=out)
        raise RuntimeError(f"oracle build failed: {e.stderr}") from e
    os.replace(tmp, out)
    return out


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params(**kw) -> RefParams:
    """Ring/RF parameters as the C struct; unspecified fields default to a proton,
    charge +1, phi_s = 0, the sine kick, and unit beta functions with zero tunes."""
    p = RefParams()
    defaults = dict(mass_eV=938.27208816e6, charge_e=1.0, phi_s_rad=0.0, rf_linear=0.0,
                    beta_x_m=1.0, beta_y_m=1.0, Qx=0.0, Qy=0.0)
    defaults.update(kw)
    for k, v in defaults.items():
        setattr(p, k, float(v))
    return p


class Oracle:
    """One loaded copy of the C oracle (the default one, or a test's mutated build)."""

    def __init__(self, path: str):
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.ref_derive.argtypes = [C.POINTER(RefParams), C.POINTER(RefDerived)]
        L.ref_derive.restype = C.c_int
        L.ref_track_signed.argtypes = [C.POINTER(RefDerived), C.c_int, C.c_double,
                                       dp, dp, dp, dp, dp, dp, C.c_long, C.c_long, dp, C.c_long]
        L.ref_track_signed.restype = C.c_int
        L.ref_moments.argtypes = [dp, dp, dp, dp, dp, dp, C.c_long, dp]
        L.ref_moments.restype = None
        L.ref_jacobian.argtypes = [C.POINTER(RefDerived), C.c_int, C.c_double, C.c_double,
                                   C.c_long, dp]
        L.ref_jacobian.restype = C.c_int
        L.ref_ramp_derive.argtypes = [C.POINTER(RefParams), dp, dp, C.c_long, dp]
        L.ref_ramp_derive.restype = C.c_int
        L.ref_track_ramp.argtypes = [C.POINTER(RefDerived), dp, C.c_long, C.c_long, C.c_int,
                                     dp, dp, dp, dp, dp, dp, C.c_long, C.c_long, dp, C.c_long]
        L.ref_track_ramp.restype = C.c_int
        lp = C.POINTER(C.c_long)
        L.ref_collective_kick.argtypes = [dp, dp, C.c_long, C.c_double, C.c_double, C.c_long, dp,
                                          C.c_double, C.c_double, lp, dp]
        L.ref_collective_kick.restype = C.c_int
        L.ref_track_collective.argtypes = [C.POINTER(RefDerived), C.c_int, dp, dp, dp, dp, dp, dp,
                                           C.c_long, C.c_long, C.c_double, C.c_double, C.c_long,
                                           dp, C.c_double, C.c_double, dp, C.c_long]
        L.ref_track_collective.restype = C.c_int
        L.ref_num_threads.argtypes = []
        L.ref_num_threads.restype = C.c_int
        L.ref_set_num_threads.argtypes = [C.c_int]
        L.ref_set_num_threads.restype = C.c_int
        self.lib = L
        self.path = path

    def derive_rc(self, p: RefParams) -> int:
        d = RefDerived()
        return int(self.lib.ref_derive(C.byref(p), C.byref(d)))

    def derive(self, p) -> RefDerived:
        if isinstance(p, dict):
            p = params(**p)
        d = RefDerived()
        rc = self.lib.ref_derive(C.byref(p), C.byref(d))
        if rc != 0:
            raise ValueError(f"ref_derive returned {rc}")
        return d

    def track(self, d: RefDerived, scheme, z, dp, x=None, xp=None, y=None, yp=None, turns=1,
              moments=False, stride=1, sign=1.0):
        """Track copies of the inputs; returns (z, dp, x, xp, y, yp, moments-or-None).

        moments: array (turns // stride + 1, NMOM); row r holds the moments after turn
        r*stride (row 0 = the initial state).  sign=-1 applies the exact inverse map."""
        if isinstance(scheme, str):
            scheme = SCHEMES[scheme]
        arrs = [None if a is None else np.array(a, dtype=np.float64, copy=True, order="C").reshape(-1)
                for a in (z, dp, x, xp, y, yp)]
        n = arrs[0].shape[0]
        mom = np.zeros((turns // stride + 1, NMOM)) if moments else None
        rc = self.lib.ref_track_signed(C.byref(d), int(scheme), float(sign),
                                       *[_ptr(a) for a in arrs], n, int(turns), _ptr(mom),
                                       int(stride))
        if rc != 0:
            raise ValueError(f"ref_track returned {rc}")
        return (*arrs, mom)

    def moments(self, z, dp, x=None, xp=None, y=None, yp=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
                for a in (z, dp, x, xp, y, yp)]
        out = np.zeros(NMOM)
        self.lib.ref_moments(*[_ptr(a) for a in arrs], arrs[0].shape[0], _ptr(out))
        return out

    def jacobian(self, d: RefDerived, scheme, z0, dp0, turns=1):
        if isinstance(scheme, str):
            scheme = SCHEMES[scheme]
        J = np.zeros(4)
        rc = self.lib.ref_jacobian(C.byref(d), int(scheme), float(z0), float(dp0), int(turns),
                                   _ptr(J))
        if rc != 0:
            raise ValueError(f"ref_jacobian returned {rc}")
        return J.reshape(2, 2)

    def ramp_derive_rc(self, p, V, p0):
        """(rc, per-turn constants (N, RAMP_NC)) of the programme V[0..N-1], p0[0..N]."""
        if isinstance(p, dict):
            p = params(**p)
        V = np.ascontiguousarray(V, dtype=np.float64)
        p0 = np.ascontiguousarray(p0, dtype=np.float64)
        if p0.shape[0] != V.shape[0] + 1:
            raise ValueError("p0 needs one more entry than V")
        out = np.zeros((V.shape[0], RAMP_NC))
        rc = self.lib.ref_ramp_derive(C.byref(p), _ptr(V), _ptr(p0), V.shape[0], _ptr(out))
        return int(rc), out

    def ramp_derive(self, p, V, p0):
        rc, out = self.ramp_derive_rc(p, V, p0)
        if rc != 0:
            raise ValueError(f"ref_ramp_derive returned {rc}")
        return out

    def track_ramp(self, d: RefDerived, tc, scheme, z, dp, x=None, xp=None, y=None, yp=None,
                   turn0=0, turns=None, moments=False, stride=1):
        """Track turns [turn0, turn0 + turns) of a programme (tc from ramp_derive) on copies of
        the inputs; returns (z, dp, x, xp, y, yp, moments-or-None) like track()."""
        if isinstance(scheme, str):
            scheme = SCHEMES[scheme]
        tc = np.ascontiguousarray(tc, dtype=np.float64)
        if turns is None:
            turns = tc.shape[0] - turn0
        arrs = [None if a is None else np.array(a, dtype=np.float64, copy=True, order="C").reshape(-1)
                for a in (z, dp, x, xp, y, yp)]
        n = arrs[0].shape[0]
        mom = np.zeros((turns // stride + 1, NMOM)) if moments else None
        rc = self.lib.ref_track_ramp(C.byref(d), _ptr(tc), tc.shape[0], int(turn0), int(scheme),
                                     *[_ptr(a) for a in arrs], n, int(turns), _ptr(mom),
                                     int(stride))
        if rc != 0:
            raise ValueError(f"ref_track_ramp returned {rc}")
        return (*arrs, mom)

    def collective_kick(self, z, dp, z_lo, inv_dz, w, alpha, alpha_sc=0.0):
        """One collective step on copies of (z, dp): returns (z, dp, counts, V)."""
        z = np.array(z, dtype=np.float64, copy=True, order="C").reshape(-1)
        dp = np.array(dp, dtype=np.float64, copy=True, order="C").reshape(-1)
        w = np.ascontiguousarray(w, dtype=np.float64)
        ns = w.shape[0]
        counts = np.zeros(ns, dtype=np.int64)
        V = np.zeros(ns)
        rc = self.lib.ref_collective_kick(_ptr(z), _ptr(dp), z.shape[0], float(z_lo), float(inv_dz),
                                          ns, _ptr(w), float(alpha), float(alpha_sc),
                                          counts.ctypes.data_as(C.POINTER(C.c_long)), _ptr(V))
        if rc != 0:
            raise ValueError(f"ref_collective_kick returned {rc}")
        return z, dp, counts, V

    def track_collective(self, d: RefDerived, scheme, z, dp, x=None, xp=None, y=None, yp=None,
                         turns=1, z_lo=-1.0, inv_dz=1.0, w=(0.0,), alpha=0.0, alpha_sc=0.0,
                         moments=False, stride=1):
        """Turns of map + collective step on copies of the inputs; returns like track()."""
        if isinstance(scheme, str):
            scheme = SCHEMES[scheme]
        arrs = [None if a is None else np.array(a, dtype=np.float64, copy=True, order="C").reshape(-1)
                for a in (z, dp, x, xp, y, yp)]
        n = arrs[0].shape[0]
        w = np.ascontiguousarray(w, dtype=np.float64)
        mom = np.zeros((turns // stride + 1, NMOM)) if moments else None
        rc = self.lib.ref_track_collective(C.byref(d), int(scheme), *[_ptr(a) for a in arrs], n,
                                           int(turns), float(z_lo), float(inv_dz), w.shape[0],
                                           _ptr(w), float(alpha), float(alpha_sc), _ptr(mom),
                                           int(stride))
        if rc != 0:
            raise ValueError(f"ref_track_collective returned {rc}")
        return (*arrs, mom)

    def num_threads(self) -> int:
        return int(self.lib.ref_num_threads())

    def set_num_threads(self, n: int) -> int:
        """Threads of this OS thread's later oracle calls (OpenMP); returns the count in
        effect.  Used to time the oracle on one core and on all cores."""
        return int(self.lib.ref_set_num_threads(int(n)))


def load() -> Oracle:
    """The default oracle (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
    return _lib


def derive(p):
    return load().derive(p)


def derive_rc(p) -> int:
    return load().derive_rc(p)


def track(*a, **k):
    return load().track(*a, **k)


def moments(*a, **k):
    return load().moments(*a, **k)


def jacobian(*a, **k):
    return load().jacobian(*a, **k)


def num_threads() -> int:
    return load().num_threads()


def collective_kick(*a, **k):
    return load().collective_kick(*a, **k)


def track_collective(*a, **k):
    return load().track_collective(*a, **k)


def ramp_derive(*a, **k):
    return load().ramp_derive(*a, **k)


def track_ramp(*a, **k):
    return load().track_ramp(*a, **k)
