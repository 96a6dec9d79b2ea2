"""Shared test helpers: seeded inputs (from the synthetic generator) and the
per-particle error measure used by the parity tests.

Parity tolerance reading: the FP64 path must agree with the FP64 oracle to a
per-particle relative error of 1e-10 after 1e4 turns for particles inside 90 % of the
separatrix, where 'relative' is |dz| / zhat_p and |d delta| / dhat_p with zhat_p, dhat_p
the particle's own oscillation amplitudes (floored at 1e-3 of the bucket size), and
|du| / sqrt(beta eps_p) transversely.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from paper_1610_05801_gb300 import synth


def bucket_of(d) -> synth.Bucket:
    return synth.Bucket(k=d.k, A=d.A, etaC=d.etaC, Qs=d.Qs, betagamma=d.betagamma)


def inputs(n, seed=0, voltage=4.5e6, transverse=True, sep_frac=0.9, sigma_z=0.15):
    """Ring dict, oracle-derived constants and a matched bunch inside sep_frac of the
    separatrix (plus matched transverse Gaussians when transverse=True)."""
    ring = synth.ring(voltage, transverse=True)
    d = oracle.load().derive(ring)
    b = bucket_of(d)
    z, dp, _ = synth.matched_bunch(seed, n, b, sigma_z=sigma_z, sep_frac=sep_frac)
    out = dict(ring=ring, d=d, bucket=b, z=z, dp=dp, x=None, xp=None, y=None, yp=None)
    if transverse:
        out["x"], out["xp"] = synth.transverse_gaussian(seed + 101, n, 50.0, 2e-6, d.betagamma)
        out["y"], out["yp"] = synth.transverse_gaussian(seed + 202, n, 50.0, 2e-6, d.betagamma)
    return out


def amplitudes(d, z, dp):
    """Each particle's own z and delta amplitudes from its invariant (phi_s = 0 bucket),
    floored at 1e-3 of the bucket half-length / half-height."""
    H = 0.5 * d.etaC * dp * dp + (d.A / d.k) * (1 - np.cos(d.k * z))
    c = np.clip(1 - H * d.k / d.A, -1.0, 1.0)
    zh = np.arccos(c) / d.k
    dh = np.sqrt(np.maximum(2 * H / d.etaC, 0))
    zb, db = math.pi / d.k, 2 * math.sqrt(d.A / (d.k * d.etaC))
    return np.maximum(zh, 1e-3 * zb), np.maximum(dh, 1e-3 * db)


def rel_errors(d, ref, got, z0, dp0, beta=50.0):
    """Per-particle relative errors (longitudinal; transverse where present)."""
    zh, dh = amplitudes(d, z0, dp0)
    e = [np.abs(got[0] - ref[0]) / zh, np.abs(got[1] - ref[1]) / dh]
    for i in (2, 4):
        if ref[i] is not None and got[i] is not None:
            J = np.sqrt(ref[i] ** 2 + (beta * ref[i + 1]) ** 2)
            J = np.maximum(J, 1e-3 * np.max(J))
            e.append(np.abs(got[i] - ref[i]) / J)
            e.append(np.abs(got[i + 1] - ref[i + 1]) * beta / J)
    return np.max(np.vstack(e), axis=0)
