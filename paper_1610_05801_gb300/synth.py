"""Seeded synthetic inputs for the tracker, shared by the tests, the oracle
checks and the benchmark.

This module holds no tracking arithmetic: no kick, drift, transfer matrix or
moment code.  It only draws initial coordinates and workload descriptions.
Where a recipe needs the bucket geometry (to keep particles inside a fraction of
the separatrix, or to match sigma_delta to sigma_z), the caller passes those
numbers in; they come from whichever side (oracle or library) is asking.

Random numbers: SplitMix64 (Steele, Lea & Flood 2014; the public-domain
reference by S. Vigna), written out here, feeding the Box-Muller transform.
The same seed always gives the same bytes on every machine.

The paper (Sec. 2.2) feeds both of its programs the same two-column (z, delta)
data file; here the same arrays are handed to the oracle and to the GPU.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASS_PROTON_EV = 938.27208816e6  # CODATA 2018


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 stream started at `seed`."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        s = (s ^ (s >> np.uint64(30))) * _M1
        s = (s ^ (s >> np.uint64(27))) * _M2
        return s ^ (s >> np.uint64(31))


class Stream:
    """Sequential draws from one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def u64(self, count: int) -> np.ndarray:
        out = splitmix64(self.seed, count, self.pos)
        self.pos += count
        return out

    def uniform(self, count: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, count: int) -> np.ndarray:
        """Standard normal deviates by Box-Muller (both outputs of each pair used)."""
        m = (count + 1) // 2
        u1 = 1.0 - self.uniform(m)  # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        out = np.empty(2 * m)
        out[0::2] = r * np.cos(2.0 * math.pi * u2)
        out[1::2] = r * np.sin(2.0 * math.pi * u2)
        return out[:count]


# --------------------------------------------------------------------------------------------
# Workload recipes (ring parameters, bunch shapes) of the benchmark configurations.

RING_SPS_LIKE = dict(circumference_m=6911.5, harmonic=4620, p0_eVc=26e9, gamma_t=22.77,
                     mass_eV=MASS_PROTON_EV, charge_e=1.0, phi_s_rad=0.0)


def ring(voltage_V: float, transverse: bool = False, **over) -> dict:
    """Ring/RF parameter dict of the proton-ring workloads (C = 6911.5 m, h = 4620,
    p0 = 26 GeV/c, gamma_t = 22.77, stationary bucket phi_s = 0)."""
    r = dict(RING_SPS_LIKE, voltage_V=float(voltage_V), rf_linear=0)
    if transverse:
        r.update(beta_x_m=50.0, beta_y_m=50.0, Qx=20.13, Qy=20.18)
    else:
        r.update(beta_x_m=1.0, beta_y_m=1.0, Qx=0.0, Qy=0.0)
    r.update(over)
    return r


@dataclasses.dataclass
class Bucket:
    """Bucket geometry supplied by the caller: k = 2 pi h / C, A = the kick amplitude,
    etaC = eta * C, Qs = small-amplitude synchrotron tune, betagamma."""
    k: float
    A: float
    etaC: float
    Qs: float
    betagamma: float = 1.0

    @property
    def half_length(self) -> float:
        return math.pi / self.k

    @property
    def half_height(self) -> float:
        return 2.0 * math.sqrt(self.A / (self.k * self.etaC))

    def contour(self, z, dp):
        """Value of the stationary-bucket invariant 0.5 etaC dp^2 + (A/k)(1 - cos kz):
        used only to select initial conditions inside a fraction of the separatrix."""
        return 0.5 * self.etaC * dp * dp + (self.A / self.k) * (1.0 - np.cos(self.k * z))

    def contour_at_amplitude(self, frac: float) -> float:
        """Contour value of the orbit whose z-amplitude is frac * half_length."""
        return (self.A / self.k) * (1.0 - math.cos(frac * math.pi))


def matched_bunch(seed: int, n: int, bucket: Bucket, sigma_z: float = 0.15,
                  z_cut_frac: float = 0.8, sep_frac: float = 1.0):
    """Gaussian bunch: z ~ N(0, sigma_z) truncated at |z| <= z_cut_frac * half_length,
    delta ~ N(0, sigma_dp) with sigma_dp = sigma_z * 2 pi Qs / |eta C| (linear matching);
    pairs outside sep_frac of the separatrix are redrawn.  Returns (z, dp, rejected)."""
    s = Stream(seed)
    sig_dp = sigma_z * 2.0 * math.pi * bucket.Qs / abs(bucket.etaC)
    zcut = z_cut_frac * bucket.half_length
    hmax = bucket.contour_at_amplitude(sep_frac)
    zs, ds, got, rejected = [], [], 0, 0
    while got < n:
        m = max(1024, int(1.3 * (n - got)))
        z = s.normal(m) * sigma_z
        d = s.normal(m) * sig_dp
        ok = (np.abs(z) <= zcut) & (bucket.contour(z, d) <= hmax)
        rejected += int(m - ok.sum())
        z, d = z[ok], d[ok]
        zs.append(z)
        ds.append(d)
        got += z.shape[0]
    z = np.concatenate(zs)[:n].copy()
    d = np.concatenate(ds)[:n].copy()
    return z, d, rejected


def halo_bunch(seed: int, n: int, bucket: Bucket, core_frac: float = 0.6,
               halo_sep_frac: float = 0.98, sigma_z: float = 0.15):
    """Precision-sweep bunch: core_frac of the particles from matched_bunch, the rest
    uniform in (z, delta) over the box [+-halo_sep_frac * half_length] x [+-half_height],
    kept only inside halo_sep_frac of the separatrix.  Core and halo are interleaved
    by a seeded permutation so any prefix is a fair subsample."""
    n_core = int(round(core_frac * n))
    zc, dc, _ = matched_bunch(seed, n_core, bucket, sigma_z=sigma_z)
    s = Stream(seed + 0x5A5A5A5A)
    hmax = bucket.contour_at_amplitude(halo_sep_frac)
    zh, dh, got = [], [], 0
    while got < n - n_core:
        m = max(1024, 2 * (n - n_core - got))
        z = (2.0 * s.uniform(m) - 1.0) * halo_sep_frac * bucket.half_length
        d = (2.0 * s.uniform(m) - 1.0) * bucket.half_height
        ok = bucket.contour(z, d) <= hmax
        zh.append(z[ok])
        dh.append(d[ok])
        got += int(ok.sum())
    z = np.concatenate([zc] + zh)[:n]
    d = np.concatenate([dc] + dh)[:n]
    perm = np.argsort(Stream(seed + 0x77).uniform(n), kind="stable")
    return z[perm].copy(), d[perm].copy()


def transverse_gaussian(seed: int, n: int, beta_m: float, eps_n: float, betagamma: float):
    """Matched Gaussian in one plane (alpha = 0): sigma_u = sqrt(beta eps),
    sigma_u' = sqrt(eps / beta), eps = eps_n / (beta gamma)."""
    eps = eps_n / betagamma
    s = Stream(seed)
    u = s.normal(n) * math.sqrt(beta_m * eps)
    up = s.normal(n) * math.sqrt(eps / beta_m)
    return u, up


def batched_jobs(seed: int = 3, nbunch: int = 64, total: float = 6e7, nmin: float = 1e3,
                 nmax: float = 4e6, vmin: float = 1e6, vmax: float = 6e6, tmin: int = 1000,
                 tmax: int = 100000):
    """Uneven bunches: n log-uniform in [nmin, nmax] then rescaled so the sum is about
    `total` (each clipped to [nmin, nmax]); V uniform in [vmin, vmax]; turns uniform
    integers in [tmin, tmax].  Returns a list of dicts (n, voltage_V, turns, seed)."""
    s = Stream(seed)
    ln = s.uniform(nbunch) * (math.log(nmax) - math.log(nmin)) + math.log(nmin)
    n = np.exp(ln)
    n = np.clip(n * (total / n.sum()), nmin, nmax)
    v = vmin + s.uniform(nbunch) * (vmax - vmin)
    t = tmin + (s.u64(nbunch) % np.uint64(tmax - tmin + 1)).astype(np.int64)
    return [dict(n=int(round(n[i])), voltage_V=float(v[i]), turns=int(t[i]), seed=1000 + i)
            for i in range(nbunch)]


def serving_trace(seed: int = 4, count: int = 2000, rate_hz: float = 200.0, nmin: float = 1e4,
                  nmax: float = 8e6, tmin: float = 1e2, tmax: float = 1e5):
    """Poisson arrivals at rate_hz; n and turns log-uniform; integrator uniform over the
    three schemes; FP64 or FP32-compensated with equal probability.
    Returns a list of dicts (t_arrive_s, n, turns, integrator, dtype, seed)."""
    s = Stream(seed)
    gaps = -np.log(1.0 - s.uniform(count)) / rate_hz
    t = np.cumsum(gaps)
    n = np.exp(math.log(nmin) + s.uniform(count) * (math.log(nmax) - math.log(nmin)))
    T = np.exp(math.log(tmin) + s.uniform(count) * (math.log(tmax) - math.log(tmin)))
    integ = (s.u64(count) % np.uint64(3)).astype(int)
    dt = (s.u64(count) % np.uint64(2)).astype(int)
    return [dict(t_arrive_s=float(t[i]), n=int(round(n[i])), turns=max(1, int(round(T[i]))),
                 integrator=int(integ[i]), dtype=int(dt[i]), seed=5000 + i)
            for i in range(count)]
