"""Fit the polynomial coefficients of the library's FP64 sine (sin_f64.cuh) and, with
--f32, of the FP32 sine of the FP32-compensated kick (ops_f32c.cuh).

Method (textbook): after Cody-Waite reduction x = q pi/2 + r, |r| <= pi/4,
    sin r = r + r^3 S(r^2),          S(t) ~ (sin(sqrt t) - sqrt t) / t^(3/2)
    cos r = 1 - r^2/2 + r^4 C(r^2),   C(t) ~ (cos(sqrt t) - 1 + t/2) / t^2
with S and C of degree 5 in t on [0, (pi/4)^2].  Both are fitted by Chebyshev
interpolation at 60-digit precision (mpmath.chebyfit, a near-minimax fit) and rounded
to double.  Run once; the printed table is pasted into sin_f64.cuh.  Needs mpmath.
"""
import mpmath as mp


def fit(f, deg=5):
    mp.mp.dps = 60
    t1 = (mp.pi / 4) ** 2
    coeffs, err = mp.chebyfit(f, [mp.mpf(10) ** -30, t1], deg + 1, error=True)
    return [float(c) for c in reversed(coeffs)], float(err)  # c0 + c1 t + ...


def S(t):
    r = mp.sqrt(t)
    return (mp.sin(r) - r) / (t * r)


def Cc(t):
    r = mp.sqrt(t)
    return (mp.cos(r) - 1 + t / 2) / (t * t)


def check(sc, cc):
    """Max relative error of the double-rounded polynomials (evaluated at high precision)."""
    mp.mp.dps = 40
    worst_s = worst_c = 0
    for i in range(1, 4001):
        r = mp.pi / 4 * i / 4000
        t = r * r
        ps = sum(mp.mpf(c) * t ** k for k, c in enumerate(sc))
        pc = sum(mp.mpf(c) * t ** k for k, c in enumerate(cc))
        s = r + r ** 3 * ps
        c = 1 - t / 2 + t * t * pc
        worst_s = max(worst_s, abs(s / mp.sin(r) - 1))
        worst_c = max(worst_c, abs(c / mp.cos(r) - 1))
    return float(worst_s), float(worst_c)


def check_f32(sc, cc):
    """Max relative error of the float-rounded degree-2 polynomials on [0, pi/4]."""
    import numpy as np

    mp.mp.dps = 30
    sc32 = [float(np.float32(c)) for c in sc]
    cc32 = [float(np.float32(c)) for c in cc]
    ws = wc = 0
    for i in range(1, 4001):
        r = mp.pi / 4 * i / 4000
        t = r * r
        s = r + r ** 3 * sum(mp.mpf(c) * t ** k for k, c in enumerate(sc32))
        c = 1 - t / 2 + t * t * sum(mp.mpf(c) * t ** k for k, c in enumerate(cc32))
        ws = max(ws, abs(s / mp.sin(r) - 1))
        wc = max(wc, abs(c / mp.cos(r) - 1))
    return sc32, cc32, float(ws), float(wc)


if __name__ == "__main__":
    import sys

    if "--f32" in sys.argv:
        # the FP32 sine of the FP32-compensated kick: degree 2 in t for both S and C
        sc, es = fit(S, deg=2)
        cc, ec = fit(Cc, deg=2)
        sc32, cc32, ws, wc = check_f32(sc, cc)
        print("// FP32 S(t):", ", ".join(f"{c!r}f" for c in sc32), "(fit error %.2e)" % es)
        print("// FP32 C(t):", ", ".join(f"{c!r}f" for c in cc32), "(fit error %.2e)" % ec)
        print("// max relative error with float coefficients: sin %.2e, cos %.2e" % (ws, wc))
        sys.exit(0)
    sc, es = fit(S)
    cc, ec = fit(Cc)
    print("// S(t), t = r^2: c0 + c1 t + ... (fit error %.2e)" % es)
    for c in sc:
        print(f"    {c!r},")
    print("// C(t): (fit error %.2e)" % ec)
    for c in cc:
        print(f"    {c!r},")
    print("// max relative error of the polynomials on [0, pi/4]: sin %.2e, cos %.2e" % check(sc, cc))
