"""Write the regression fixtures of this directory from the FP64 oracle alone.

The paper prints no physics values (its tables are timings), so no fixture here holds a
value of the paper.  These files store the oracle's own results on the seeded synthetic
inputs of the small workload (1000 macro-particles, proton ring C = 6911.5 m, h = 4620,
p0 = 26 GeV/c, gamma_t = 22.77, V = 2 MV, phi_s = 0, matched bunch with sigma_z = 0.15 m
truncated at 80 % of the bucket half-length, seed 0): a change to the oracle's arithmetic
that moves them must be deliberate (the fixture is then rewritten by this script and the
change justified), and the GPU tests compare the library with them.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1610_05801_gb300 import synth  # noqa: E402

SCHEMES = ("euler_cromer", "leapfrog", "ruth4", "rk4")
TURNS = 1000
N_KEEP = 16


def inputs():
    ring = synth.ring(2e6)
    d = oracle.derive(ring)
    b = synth.Bucket(k=d.k, A=d.A, etaC=d.etaC, Qs=d.Qs, betagamma=d.betagamma)
    z, dp, _ = synth.matched_bunch(0, 1000, b)
    return ring, d, z, dp


def main():
    ring, d, z, dp = inputs()
    path = os.path.join(HERE, "oracle_small_workload_1000turns.txt")
    with open(path, "w") as f:
        f.write("# FP64 oracle, small workload (1000 particles, seed 0, V = 2 MV), after 1000 turns.\n")
        f.write("# Written by tests/golden/make_golden.py from oracle/ only; the paper prints no\n")
        f.write("# physics values.  Columns: scheme, particle index, z [m], delta; then per scheme\n")
        f.write("# the bunch moments (mean z, mean delta, rms z, rms delta, eps_z) of all 1000.\n")
        for s in SCHEMES:
            zf, df, *_, mom = oracle.track(d, s, z, dp, turns=TURNS, moments=True, stride=TURNS)
            for i in range(N_KEEP):
                f.write(f"particle {s} {i} {float(zf[i])!r} {float(df[i])!r}\n")
            f.write("moments " + s + " " + " ".join(repr(float(v)) for v in mom[-1, :5]) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
