"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each pin takes an ``oracle.Oracle`` (the default build, or a deliberately mutated
copy in ``test_oracle_mutants.py``) and raises AssertionError when the oracle
disagrees with the mathematics.  The paper prints no formulas and no physics
results (Sec. 1.1.1 and 1.1.2 only name the schemes), so every pin here is a
closed form, an invariant, a textbook formula or a brute-force evaluation:

* textbook synchrotron tune and stationary-bucket height (in terms of h, eta, V,
  beta and E only);
* the closed-form one-turn matrices of the linearised Euler-Cromer and leap-frog
  maps and the Chebyshev form of their N-th power; the 4th-order tune error of
  the Ruth scheme;
* the pendulum's amplitude-dependent period (complete elliptic integral);
* the separatrix found by tracking, against the textbook bucket height;
* time-reversal symmetry of the palindromic schemes (and its absence for EC);
* the exact inverse map; det J = 1 (dual numbers and finite differences);
* order of the energy error under a change of RF voltage;
* oddness of the force and the fixed point; the exact transverse rotation;
* moments against numpy's mean / std / covariance;
* a 40-digit mpmath evaluation of the same maps on tiny inputs.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as _oracle

M_P = 938.27208816e6
RING = dict(circumference_m=6911.5, harmonic=4620.0, p0_eVc=26e9, gamma_t=22.77, mass_eV=M_P,
            charge_e=1.0, phi_s_rad=0.0, rf_linear=0.0, beta_x_m=50.0, beta_y_m=50.0,
            Qx=20.13, Qy=20.18)


def ring(**over):
    r = dict(RING, voltage_V=2e6)
    r.update(over)
    return r


def textbook(r):
    """Textbook quantities from the ring parameters only (charge +1 e)."""
    E = math.hypot(r["p0_eVc"], r["mass_eV"])
    gamma = E / r["mass_eV"]
    beta = r["p0_eVc"] / E
    eta = 1.0 / r["gamma_t"] ** 2 - 1.0 / gamma ** 2
    h, V, C = r["harmonic"], r["voltage_V"], r["circumference_m"]
    cphi = math.cos(r["phi_s_rad"])
    # small-amplitude synchrotron tune  Q_s = sqrt(h eta e V cos(phi_s) / (2 pi beta^2 E))
    Qs = math.sqrt(h * eta * V * cphi / (2.0 * math.pi * beta ** 2 * E))
    # stationary bucket half-height  (dp/p)_max = sqrt(2 e V / (pi beta^2 E h |eta|))
    dhat = math.sqrt(2.0 * V / (math.pi * beta ** 2 * E * h * abs(eta)))
    # linear one-turn quantities: eta C and the kick slope a = (e V / (beta p0 c)) (2 pi h / C) cos(phi_s)
    etaC = eta * C
    a = V / (beta * r["p0_eVc"]) * (2.0 * math.pi * h / C) * cphi
    zhat = C / (2.0 * h)  # bucket half-length
    return dict(E=E, gamma=gamma, beta=beta, eta=eta, Qs=Qs, dhat=dhat, etaC=etaC, a=a,
                K=etaC * a, zhat=zhat, k=2.0 * math.pi * h / C)


def _traj(O, d, scheme, z0, dp0, turns):
    """Turn-by-turn (z, dp) of one particle, via the single-particle moments (mean = value)."""
    *_, mom = O.track(d, scheme, [z0], [dp0], turns=turns, moments=True, stride=1)
    return mom[:, 0].copy(), mom[:, 1].copy()


def _tune_from_crossings(z):
    s = np.signbit(z)
    idx = np.nonzero(s[1:] != s[:-1])[0]
    assert idx.size >= 4, "no oscillation"
    tc = idx + z[idx] / (z[idx] - z[idx + 1])
    return (idx.size - 1) / (2.0 * (tc[-1] - tc[0]))


# --------------------------------------------------------------------------------------------


def pin_textbook_constants(O):
    for V in (2e6, 4.5e6):
        r = ring(voltage_V=V)
        tb = textbook(r)
        d = O.derive(r)
        assert abs(d.gamma / tb["gamma"] - 1) < 1e-14
        assert abs(d.beta / tb["beta"] - 1) < 1e-14
        assert abs(d.Qs / tb["Qs"] - 1) < 1e-12, (d.Qs, tb["Qs"])
        dhat_map = 2.0 * math.sqrt(d.A / (d.k * d.etaC))
        assert abs(dhat_map / tb["dhat"] - 1) < 1e-12, (dhat_map, tb["dhat"])
        assert abs(math.pi / d.k / tb["zhat"] - 1) < 1e-14


def pin_stability_rules(O):
    assert O.derive_rc(_oracle.params(**ring())) == 0
    # below transition (gamma < gamma_t) the stationary bucket needs phi_s = pi
    below = ring(p0_eVc=10e9)
    assert O.derive_rc(_oracle.params(**below)) == -2
    assert O.derive_rc(_oracle.params(**dict(below, phi_s_rad=math.pi))) == 0
    # zero voltage: a pure drift is allowed
    assert O.derive_rc(_oracle.params(**ring(voltage_V=0.0))) == 0


def _linear_matrix(O, d, scheme):
    sz, sd = 1e-2, 1e-5
    z1, d1, *_ = O.track(d, scheme, [sz, 0.0], [0.0, sd], turns=1)
    return np.array([[z1[0] / sz, z1[1] / sd], [d1[0] / sz, d1[1] / sd]])


def pin_linear_closed_form(O):
    """rf_linear: sin(phi) - sin(phi_s) -> cos(phi_s) k z makes every scheme a constant matrix."""
    for phis in (0.0, 0.3):
        _linear_closed_form_at(O, phis)


def _linear_closed_form_at(O, phis):
    r = ring(rf_linear=1.0, phi_s_rad=phis)
    tb = textbook(r)
    d = O.derive(r)
    eC, a, K = tb["etaC"], tb["a"], tb["K"]
    closed = {
        "euler_cromer": np.array([[1 - K, -eC], [a, 1.0]]),          # kick, then drift
        "leapfrog": np.array([[1 - K / 2, -eC * (1 - K / 4)], [a, 1 - K / 2]]),
    }
    for scheme, Mc in closed.items():
        M = _linear_matrix(O, d, scheme)
        assert np.all(np.abs(M / Mc - 1) < 1e-12), (scheme, M, Mc)
        # N-th power by the Chebyshev identity for det M = 1:
        # M^N = (sin(N mu) M - sin((N-1) mu) I) / sin(mu),  cos(mu) = tr(M)/2 = 1 - K/2,
        # i.e. mu = 2 asin(sqrt(K)/2) (the well-conditioned form near mu = 0)
        mu = 2.0 * math.asin(math.sqrt(K) / 2.0)
        N = 10000
        MN = (math.sin(N * mu) * Mc - math.sin((N - 1) * mu) * np.eye(2)) / math.sin(mu)
        z0, dp0 = 0.05, 2e-4
        zN, dN, *_ = O.track(d, scheme, [z0], [dp0], turns=N)
        ez, ed = MN @ np.array([z0, dp0])
        # relative to the orbit's extent in each coordinate
        zs = math.hypot(z0, dp0 * tb["etaC"] / (2 * math.pi * tb["Qs"]))
        ds = zs * 2 * math.pi * tb["Qs"] / tb["etaC"]
        assert abs(zN[0] - ez) / zs < 1e-11, (scheme, zN[0], ez)
        assert abs(dN[0] - ed) / ds < 1e-11, (scheme, dN[0], ed)
    # Ruth4: det 1 and a 4th-order tune: |mu - sqrt(K)| / sqrt(K) = O(K^2), i.e. ~16x smaller
    # per K/4 (a 2nd-order scheme gives K/24, ~4x)
    errs = []
    for V in (2e6, 0.5e6):
        rr = ring(rf_linear=1.0, voltage_V=V, phi_s_rad=phis)
        tbr = textbook(rr)
        M = _linear_matrix(O, O.derive(rr), "ruth4")
        assert abs(np.linalg.det(M) - 1) < 1e-13
        mu = 2.0 * math.asin(math.sqrt(max(0.0, 2.0 - np.trace(M))) / 2.0)
        errs.append(abs(mu - math.sqrt(tbr["K"])) / math.sqrt(tbr["K"]))
    assert errs[0] < 1e-5, errs
    assert 13 < errs[0] / errs[1] < 19, errs


def pin_pendulum_detuning(O):
    """Amplitude-dependent tune of the sine kick: Q(zhat) = Qs pi / (2 K_ell(sin^2(k zhat / 2)))."""
    from scipy.special import ellipk

    r = ring()
    tb = textbook(r)
    d = O.derive(r)
    for frac in (0.3, 0.6, 0.85):
        zh = frac * tb["zhat"]
        z, _ = _traj(O, d, "ruth4", zh, 0.0, 30000)
        Q = _tune_from_crossings(z)
        m = math.sin(tb["k"] * zh / 2.0) ** 2
        Qexp = tb["Qs"] * math.pi / (2.0 * ellipk(m))
        assert abs(Q / Qexp - 1) < 2e-5, (frac, Q, Qexp)


def pin_separatrix(O):
    """A particle started at z = 0 just inside the textbook bucket height stays in the bucket;
    just outside it slips out (checked with the 4th-order scheme at low voltage)."""
    r = ring(voltage_V=0.5e6)
    tb = textbook(r)
    d = O.derive(r)
    zin, _ = _traj(O, d, "ruth4", 0.0, 0.985 * tb["dhat"], 20000)
    zout, _ = _traj(O, d, "ruth4", 0.0, 1.015 * tb["dhat"], 20000)
    assert np.max(np.abs(zin)) < tb["zhat"]
    assert np.max(np.abs(zout)) > 1.5 * tb["zhat"]


def pin_time_reversal(O):
    """Palindromic compositions (LF, Ruth4) satisfy R M R = M^-1 with R: dp -> -dp;
    Euler-Cromer does not."""
    r = ring(voltage_V=4.5e6)
    tb = textbook(r)
    d = O.derive(r)
    z0 = np.array([0.1, 0.4, 0.6]) * tb["zhat"]
    d0 = np.array([0.3, -0.2, 0.1]) * tb["dhat"]
    N = 10000
    for scheme in ("leapfrog", "ruth4", "euler_cromer"):
        z1, d1, *_ = O.track(d, scheme, z0, d0, turns=N)
        z2, d2, *_ = O.track(d, scheme, z1, -d1, turns=N)
        err = max(np.max(np.abs(z2 - z0)) / tb["zhat"], np.max(np.abs(-d2 - d0)) / tb["dhat"])
        if scheme == "euler_cromer":
            assert err > 1e-6, err
        else:
            assert err < 1e-11, (scheme, err)


def pin_inverse_map(O):
    r = ring(voltage_V=4.5e6)
    tb = textbook(r)
    d = O.derive(r)
    z0 = np.array([0.05, 0.5, 0.85]) * tb["zhat"]
    d0 = np.array([0.1, -0.3, 0.02]) * tb["dhat"]
    x0, xp0 = np.array([1e-3, -2e-3, 5e-4]), np.array([2e-5, 1e-5, -3e-5])
    for scheme in ("euler_cromer", "leapfrog", "ruth4"):
        z1, d1, x1, xp1, *_ = O.track(d, scheme, z0, d0, x0, xp0, turns=10000)
        z2, d2, x2, xp2, *_ = O.track(d, scheme, z1, d1, x1, xp1, turns=10000, sign=-1.0)
        # 1e-12 of the bucket size for orbits up to half the bucket; near the separatrix
        # (85 %) the steep amplitude-dependence of the tune amplifies rounding: 1e-11
        tol = np.array([1e-12, 1e-12, 1e-11])
        assert np.all(np.abs(z2 - z0) / tb["zhat"] < tol), (scheme, z2 - z0)
        assert np.all(np.abs(d2 - d0) / tb["dhat"] < tol), (scheme, d2 - d0)
        assert np.max(np.abs(x2 - x0)) < 1e-12 * 3e-3


def pin_symplectic(O):
    r = ring(voltage_V=4.5e6)
    tb = textbook(r)
    d = O.derive(r)
    for scheme in ("euler_cromer", "leapfrog", "ruth4"):
        for fz, fd in ((0.0, 0.0), (0.3, 0.2), (0.8, -0.1), (0.5, 0.5)):
            z0, dp0 = fz * tb["zhat"], fd * tb["dhat"]
            J = O.jacobian(d, scheme, z0, dp0, 1)
            assert abs(np.linalg.det(J) - 1) < 1e-13, (scheme, J)
            J100 = O.jacobian(d, scheme, z0, dp0, 100)
            assert abs(np.linalg.det(J100) - 1) < 1e-10, (scheme, np.linalg.det(J100))
            # the dual-number Jacobian is the derivative of the tracked map
            hz, hd = 1e-6 * tb["zhat"], 1e-6 * tb["dhat"]
            zp, dpp, *_ = O.track(d, scheme, [z0 + hz, z0 - hz, z0, z0],
                                  [dp0, dp0, dp0 + hd, dp0 - hd], turns=1)
            Jfd = np.array([[(zp[0] - zp[1]) / (2 * hz), (zp[2] - zp[3]) / (2 * hd)],
                            [(dpp[0] - dpp[1]) / (2 * hz), (dpp[2] - dpp[3]) / (2 * hd)]])
            scale = np.array([[1.0, tb["zhat"] / tb["dhat"]], [tb["dhat"] / tb["zhat"], 1.0]])
            assert np.max(np.abs(J - Jfd) / scale) < 1e-6, (scheme, J, Jfd)


def _energy_err(O, scheme, V, turns):
    r = ring(voltage_V=V)
    tb = textbook(r)
    d = O.derive(r)
    z, dp = _traj(O, d, scheme, 0.5 * tb["zhat"], 0.0, turns)
    # pendulum invariant of the smooth motion (phi_s = 0)
    H = 0.5 * d.etaC * dp ** 2 + (d.A / d.k) * (1 - np.cos(d.k * z))
    return np.max(np.abs(H - H[0])) / H[0], np.max(np.abs(H[:1001] - H[0])) / H[0]


def pin_energy_order(O):
    """Symplectic schemes keep |H - H0| bounded; it scales with the step sqrt(K) to the
    scheme's order: quartering V (halving sqrt K) divides it by ~2, ~4, ~16."""
    expect = {"euler_cromer": (1.6, 2.6), "leapfrog": (3.2, 5.0), "ruth4": (12.0, 21.0)}
    for scheme, (lo, hi) in expect.items():
        e_hi, e_hi_short = _energy_err(O, scheme, 4e6, 10000)
        e_lo, _ = _energy_err(O, scheme, 1e6, 10000)
        assert e_hi < 1.5 * e_hi_short + 1e-13, (scheme, e_hi, e_hi_short)  # bounded, no drift
        assert lo < e_hi / e_lo < hi, (scheme, e_hi / e_lo)


def pin_symmetry_and_fixed_point(O):
    r = ring(voltage_V=4.5e6)
    tb = textbook(r)
    d = O.derive(r)
    z0 = np.array([0.1, 0.45, 0.7]) * tb["zhat"]
    d0 = np.array([0.2, -0.3, 0.05]) * tb["dhat"]
    for scheme in ("euler_cromer", "leapfrog", "ruth4"):
        za, da, *_ = O.track(d, scheme, z0, d0, turns=2000)
        zb, db, *_ = O.track(d, scheme, -z0, -d0, turns=2000)
        assert np.array_equal(za, -zb) and np.array_equal(da, -db), scheme
        zf, df, *_ = O.track(d, scheme, [0.0], [0.0], turns=2000)
        assert zf[0] == 0.0 and df[0] == 0.0
    # off-zero synchronous phase (stable above transition for |phi_s| < pi/2) and
    # phi_s = pi below transition: z = dp = 0 is still a fixed point of the map
    for rr in (ring(phi_s_rad=0.3), ring(p0_eVc=10e9, phi_s_rad=math.pi)):
        dd = O.derive(rr)
        for scheme in ("euler_cromer", "leapfrog", "ruth4"):
            zf, df, *_ = O.track(dd, scheme, [0.0], [0.0], turns=500)
            assert zf[0] == 0.0 and df[0] == 0.0, (scheme, zf, df)


def pin_transverse_rotation(O):
    r = ring(voltage_V=4.5e6)
    d = O.derive(r)
    N = 10000
    for beta, Q, key in ((50.0, 20.13, "x"), (50.0, 20.18, "y")):
        u0 = np.array([1e-3, -5e-4, 0.0])
        up0 = np.array([0.0, 2e-5, -1e-5])
        args = dict(x=u0, xp=up0) if key == "x" else dict(y=u0, yp=up0)
        out = O.track(d, "leapfrog", np.zeros(3), np.zeros(3), turns=N, **args)
        u, up = (out[2], out[3]) if key == "x" else (out[4], out[5])
        # exact N-turn rotation (alpha = 0) by the phase N * 2 pi frac(Q), evaluated at 30
        # digits from the double value of frac(Q) (Q - floor(Q) is exact in binary)
        import mpmath as mp

        with mp.workdps(30):
            ph = 2 * mp.pi * N * (mp.mpf(Q) - math.floor(Q))
            c, s = float(mp.cos(ph)), float(mp.sin(ph))
        ue = c * u0 + beta * s * up0
        upe = -s / beta * u0 + c * up0
        scale = 1e-3
        assert np.max(np.abs(u - ue)) / scale < N * 1e-15, key
        assert np.max(np.abs(up - upe)) * beta / scale < N * 1e-15, key
        # Courant-Snyder invariant
        J0 = u0 ** 2 / beta + beta * up0 ** 2
        J1 = u ** 2 / beta + beta * up ** 2
        assert np.max(np.abs(J1 - J0)) / np.max(J0) < 1e-12


def pin_moments(O):
    rng = np.random.default_rng(7)
    n = 1001
    z, dp = rng.normal(0.01, 0.1, n), rng.normal(-1e-5, 1e-3, n) + 0.002 * rng.normal(0, 0.1, n)
    x, xp = rng.normal(0, 1e-3, n), rng.normal(0, 2e-5, n)
    y, yp = rng.normal(0, 2e-3, n), rng.normal(0, 1e-5, n)
    m = O.moments(z, dp, x, xp, y, yp)
    for off, (a, b) in zip((0, 5, 10), ((z, dp), (x, xp), (y, yp))):
        cov = np.cov(np.vstack([a, b]), bias=True)
        exp = [a.mean(), b.mean(), a.std(), b.std(), math.sqrt(np.linalg.det(cov))]
        assert np.allclose(m[off:off + 5], exp, rtol=1e-12, atol=0), (off, m[off:off + 5], exp)
    # planes switched off report zeros; one particle has zero spread; empty bunch is all zero
    m2 = O.moments(z, dp)
    assert np.all(m2[5:] == 0)
    m1 = O.moments(z[:1], dp[:1], x[:1], xp[:1])
    assert m1[0] == z[0] and m1[1] == dp[0] and m1[2] == 0 and m1[4] == 0
    m0 = O.moments(np.zeros(0), np.zeros(0))
    assert np.all(m0 == 0)
    # the per-turn moment rows are the moments of the tracked state
    r = ring(voltage_V=4.5e6)
    d = O.derive(r)
    tb = textbook(r)
    z0 = rng.normal(0, 0.1, 64) * tb["zhat"] / 0.75
    d0 = rng.normal(0, 0.2, 64) * tb["dhat"]
    for scheme in ("euler_cromer", "leapfrog", "ruth4"):
        zz, dd, xx, xxp, *_, mom = O.track(d, scheme, z0, d0, x[:64], xp[:64], turns=30,
                                           moments=True, stride=10)
        assert mom.shape == (4, 15)
        assert np.allclose(mom[0, :5], [z0.mean(), d0.mean(), z0.std(), d0.std(),
                                        mom[0, 4]], rtol=1e-12)
        assert np.allclose(mom[3, :4], [zz.mean(), dd.mean(), zz.std(), dd.std()], rtol=1e-12)
        assert np.allclose(mom[3, 5:9], [xx.mean(), xxp.mean(), xx.std(), xxp.std()], rtol=1e-12)
    # a matched Gaussian in the linear map keeps its rms (to the map's O(K) mismatch)
    rl = ring(rf_linear=1.0)
    tbl = textbook(rl)
    dl = O.derive(rl)
    sz = 0.1
    sd = sz * 2 * math.pi * tbl["Qs"] / tbl["etaC"]
    zg, dg = rng.normal(0, sz, 20000), rng.normal(0, sd, 20000)
    *_, mom = O.track(dl, "leapfrog", zg, dg, turns=500, moments=True, stride=50)
    assert np.max(np.abs(mom[:, 2] / mom[0, 2] - 1)) < 0.02


def pin_brute_force(O, turns=(10000, 10000, 3000), nparticles=4):
    """FP64 oracle vs the same maps evaluated at 40 significant digits (mpmath)."""
    import mpmath as mp

    mp.mp.dps = 40
    r = ring(voltage_V=4.5e6)
    tb = textbook(r)
    d = O.derive(r)
    A, k, eC = mp.mpf(d.A), mp.mpf(d.k), mp.mpf(d.etaC)
    th = 1 / (2 - mp.cbrt(2))

    def kick(w, z, dp):
        return dp + w * A * mp.sin(k * z)

    def drift(w, z, dp):
        return z - w * eC * dp

    def turn(scheme, z, dp):
        if scheme == "euler_cromer":
            dp = kick(1, z, dp)
            z = drift(1, z, dp)
        elif scheme == "leapfrog":
            z = drift(mp.mpf(1) / 2, z, dp)
            dp = kick(1, z, dp)
            z = drift(mp.mpf(1) / 2, z, dp)
        else:
            for wd, wk in ((th / 2, th), ((1 - th) / 2, 1 - 2 * th), ((1 - th) / 2, th)):
                z = drift(wd, z, dp)
                dp = kick(wk, z, dp)
            z = drift(th / 2, z, dp)
        return z, dp

    fr = np.linspace(0.1, 0.9, nparticles)
    z0 = fr * tb["zhat"] * 0.9
    d0 = (0.5 - fr) * tb["dhat"] * 0.5
    for scheme, N in zip(("euler_cromer", "leapfrog", "ruth4"), turns):
        zf, df, *_ = O.track(d, scheme, z0, d0, turns=N)
        for i in range(nparticles):
            z, dp = mp.mpf(z0[i]), mp.mpf(d0[i])
            for _ in range(N):
                z, dp = turn(scheme, z, dp)
            ez = abs(float(z) - zf[i]) / tb["zhat"]
            ed = abs(float(dp) - df[i]) / tb["dhat"]
            assert ez < 1e-11 and ed < 1e-11, (scheme, i, ez, ed)


# ---- nonlinear slippage eta(delta) and chromaticity ---------------------------------------
# eta(delta) = eta0 + eta1 delta + eta2 delta^2 in the drift; per-particle transverse phase
# advance 2 pi (frac(Q) + xi delta) with delta after the turn's longitudinal step.
# Coefficients exaggerated so that every term moves the result far above rounding.
ETA1, ETA2 = 0.5, 20.0
XI_X, XI_Y = 5.0, -3.0
# milder coefficients for the pins that need bounded motion inside the bucket
ETA1_B, ETA2_B = 0.05, 2.0


def pin_nonlinear_slippage_closed_form(O):
    """RF off: delta is constant and the drift stages of every scheme add up to one turn,
    z_N = z_0 - N C (eta0 + eta1 d + eta2 d^2) d, with eta0 from the textbook formula."""
    r = ring(voltage_V=0.0, eta1=ETA1, eta2=ETA2)
    tb = textbook(r)
    d = O.derive(r)
    N = 1000
    z0 = np.array([0.0, 0.1, -0.2, 0.05])
    d0 = np.array([-1e-2, 3e-3, 7e-3, 0.0])
    C = r["circumference_m"]
    shift = N * C * (tb["eta"] + ETA1 * d0 + ETA2 * d0 ** 2) * d0
    for scheme in ("euler_cromer", "leapfrog", "ruth4", "rk4"):
        zf, df, *_ = O.track(d, scheme, z0, d0, turns=N)
        assert np.array_equal(df, d0), scheme
        err = np.abs(zf - (z0 - shift))
        assert np.all(err <= 1e-12 * np.abs(shift) + 1e-15), (scheme, err, shift)


def pin_nonlinear_slippage_fixed_points(O):
    """With RF on, (z, delta*) with eta(delta*) = 0 and sin(k z) = 0 is a fixed point of
    every scheme (no slip, no force); the roots come from the quadratic formula.  Half of
    these points are hyperbolic (rounding grows ~e^(0.06 t)), so 60 turns."""
    for e1, e2 in ((ETA1, 0.0), (ETA1, ETA2)):
        r = ring(voltage_V=4.5e6, eta1=e1, eta2=e2)
        tb = textbook(r)
        d = O.derive(r)
        e0 = tb["eta"]
        if e2 == 0.0:
            roots = [-e0 / e1]
        else:
            q = -0.5 * (e1 + math.sqrt(e1 * e1 - 4 * e2 * e0))
            roots = [e0 / q, q / e2]  # both roots, each in its stable form
        for ds in roots:
            for zs in (0.0, math.pi / d.k):
                for scheme in ("euler_cromer", "leapfrog", "ruth4"):
                    zf, df, *_ = O.track(d, scheme, [zs], [ds], turns=60)
                    assert abs(zf[0] - zs) < 1e-12 and abs(df[0] - ds) < 1e-14, \
                        (e1, e2, ds, zs, scheme, zf, df)


def _energy_err_nl(O, scheme, V, turns):
    r = ring(voltage_V=V, eta1=ETA1_B, eta2=ETA2_B)
    tb = textbook(r)
    d = O.derive(r)
    C = r["circumference_m"]
    z, dp = _traj(O, d, scheme, 0.4 * tb["zhat"], 0.0, turns)
    # invariant of the smooth motion with eta(delta): dz/dt = -dH/d delta, d delta/dt = dH/dz
    H = C * (tb["eta"] * dp ** 2 / 2 + ETA1_B * dp ** 3 / 3 + ETA2_B * dp ** 4 / 4) \
        + (d.A / d.k) * (1 - np.cos(d.k * z))
    return np.max(np.abs(H - H[0])) / H[0]


def pin_nonlinear_slippage_energy(O):
    """The maps with eta(delta) conserve the smooth Hamiltonian
    C (eta0 d^2/2 + eta1 d^3/3 + eta2 d^4/4) + (A/k)(1 - cos k z) to their order:
    quartering V divides the bounded error by ~2 (EC), ~4 (LF), ~16 (Ruth4; 25 measured at
    this amplitude, where the next order still contributes)."""
    expect = {"euler_cromer": (1.6, 2.8, 0.06), "leapfrog": (3.2, 5.5, 2e-3),
              "ruth4": (14.0, 34.0, 2e-6)}
    for scheme, (lo, hi, cap) in expect.items():
        e_hi = _energy_err_nl(O, scheme, 4e6, 6000)
        e_lo = _energy_err_nl(O, scheme, 1e6, 6000)
        assert e_hi < cap, (scheme, e_hi)
        assert lo < e_hi / e_lo < hi, (scheme, e_hi, e_lo, e_hi / e_lo)


def pin_chromatic_phase_sum(O):
    """Rotations about the same centre commute, so N chromatic turns rotate (u, u') by the
    summed angle 2 pi sum_t (frac(Q) + xi delta_t), delta_t being delta after turn t's
    longitudinal step.  The delta_t come from the achromatic map (the transverse push does
    not act back on (z, delta)); the angle sum and the rotation are evaluated at 30 digits."""
    import mpmath as mp

    r = ring(voltage_V=4.5e6, xi_x=XI_X, xi_y=XI_Y)
    tb = textbook(r)
    d = O.derive(r)
    d0 = O.derive(ring(voltage_V=4.5e6))
    N = 500
    z0 = np.array([0.3, -0.6]) * tb["zhat"]
    p0 = np.array([0.2, 0.4]) * tb["dhat"]
    u0, up0 = np.array([1e-3, -2e-3]), np.array([3e-5, 1e-5])
    v0, vp0 = np.array([-5e-4, 1.5e-3]), np.array([-2e-5, 4e-5])
    for scheme in ("euler_cromer", "leapfrog", "ruth4"):
        zf, df, xf, xpf, yf, ypf, _ = O.track(d, scheme, z0, p0, u0, up0, v0, vp0, turns=N)
        for i in range(2):
            _, dps = _traj(O, d0, scheme, z0[i], p0[i], N)
            for (Q, xi, beta, a0, b0, a1, b1) in ((r["Qx"], XI_X, r["beta_x_m"], u0[i], up0[i], xf[i], xpf[i]),
                                                  (r["Qy"], XI_Y, r["beta_y_m"], v0[i], vp0[i], yf[i], ypf[i])):
                with mp.workdps(30):
                    q = mp.mpf(Q) - math.floor(Q)
                    th = 2 * mp.pi * mp.fsum(q + mp.mpf(xi) * mp.mpf(float(x)) for x in dps[1:])
                    c, sn = mp.cos(th), mp.sin(th)
                    ae = float(c * a0 + beta * sn * b0)
                    be = float(-sn / beta * a0 + c * b0)
                amp = math.hypot(a0, beta * b0)
                assert abs(a1 - ae) < N * 1e-15 * amp, (scheme, i, a1, ae)
                assert abs(b1 - be) * beta < N * 1e-15 * amp, (scheme, i, b1, be)


def pin_nonlinear_inverse_map(O):
    """The inverse map undoes N turns with eta(delta) and chromaticity (it rotates back with
    the same delta before undoing the longitudinal step)."""
    r = ring(voltage_V=4.5e6, eta1=ETA1_B, eta2=ETA2_B, xi_x=XI_X, xi_y=XI_Y)
    tb = textbook(r)
    d = O.derive(r)
    z0 = np.array([0.05, 0.4, -0.3]) * tb["zhat"]
    d0 = np.array([0.1, -0.3, 0.2]) * tb["dhat"]
    x0, xp0 = np.array([1e-3, -2e-3, 5e-4]), np.array([2e-5, 1e-5, -3e-5])
    y0, yp0 = np.array([-1e-3, 1e-3, 2e-4]), np.array([1e-5, -2e-5, 3e-5])
    for scheme in ("euler_cromer", "leapfrog", "ruth4"):
        out = O.track(d, scheme, z0, d0, x0, xp0, y0, yp0, turns=5000)
        back = O.track(d, scheme, *out[:6], turns=5000, sign=-1.0)
        assert np.max(np.abs(back[0] - z0)) / tb["zhat"] < 1e-12, scheme
        assert np.max(np.abs(back[1] - d0)) / tb["dhat"] < 1e-12, scheme
        assert np.max(np.abs(back[2] - x0)) < 1e-12 * 3e-3, scheme
        assert np.max(np.abs(back[4] - y0)) < 1e-12 * 3e-3, scheme


def pin_nonlinear_symplectic(O):
    """det J = 1 with eta(delta) (the drift stays a shear), dual numbers against finite
    differences of the tracked map."""
    r = ring(voltage_V=4.5e6, eta1=ETA1_B, eta2=ETA2_B)
    tb = textbook(r)
    d = O.derive(r)
    for scheme in ("euler_cromer", "leapfrog", "ruth4"):
        for fz, fd in ((0.3, 0.2), (0.6, -0.4)):
            z0, dp0 = fz * tb["zhat"], fd * tb["dhat"]
            J = O.jacobian(d, scheme, z0, dp0, 1)
            assert abs(np.linalg.det(J) - 1) < 1e-13, (scheme, J)
            hz, hd = 1e-6 * tb["zhat"], 1e-6 * tb["dhat"]
            zp, dpp, *_ = O.track(d, scheme, [z0 + hz, z0 - hz, z0, z0],
                                  [dp0, dp0, dp0 + hd, dp0 - hd], turns=1)
            Jfd = np.array([[(zp[0] - zp[1]) / (2 * hz), (zp[2] - zp[3]) / (2 * hd)],
                            [(dpp[0] - dpp[1]) / (2 * hz), (dpp[2] - dpp[3]) / (2 * hd)]])
            scale = np.array([[1.0, tb["zhat"] / tb["dhat"]], [tb["dhat"] / tb["zhat"], 1.0]])
            assert np.max(np.abs(J - Jfd) / scale) < 1e-6, (scheme, J, Jfd)


# ---- classic RK4 and the second RF system ----------------------------------------------


def pin_rk4_linear_closed_form(O):
    """rf_linear: RK4 over one turn of y' = M y, M = [[0, -eta C], [a, 0]], is the 4th-order
    Taylor polynomial of exp(M): R = I (1 - K/2 + K^2/24) + M (1 - K/6) with K = eta C a
    (M^2 = -K I), so det R = 1 - K^3/72 + K^4/576 < 1 (not symplectic)."""
    for phis in (0.0, 0.3):
        r = ring(rf_linear=1.0, phi_s_rad=phis, voltage_V=4.5e6)
        tb = textbook(r)
        d = O.derive(r)
        eC, a, K = tb["etaC"], tb["a"], tb["K"]
        Mg = np.array([[0.0, -eC], [a, 0.0]])
        Rc = np.eye(2) * (1 - K / 2 + K * K / 24) + Mg * (1 - K / 6)
        R = _linear_matrix(O, d, "rk4")
        scale = np.array([[1.0, eC], [a, 1.0]])
        assert np.max(np.abs(R - Rc) / np.abs(scale)) < 1e-12, (phis, R, Rc)
        detc = 1 - K ** 3 / 72 + K ** 4 / 576
        assert abs(np.linalg.det(R) - detc) < 1e-14 and detc < 1, (np.linalg.det(R), detc)
        # the dual-number Jacobian agrees, and 100 turns multiply the determinant
        J = O.jacobian(d, "rk4", 0.01, 1e-4, 100)
        assert abs(np.linalg.det(J) / detc ** 100 - 1) < 1e-10


def _rk4_turn_error(O, V, fz):
    """Largest one-turn error of the oracle's RK4 against the exact flow of the pendulum
    dz/dn = -eta C d, d d/dn = A sin(k z), integrated by mpmath's Taylor-series solver."""
    import mpmath as mp

    r = ring(voltage_V=V)
    tb = textbook(r)
    d = O.derive(r)
    eC, A, k = d.etaC, d.A, d.k
    z0 = fz * tb["zhat"]
    out = []
    for z_init in z0:
        zf, df, *_ = O.track(d, "rk4", [z_init], [0.0], turns=1)
        with mp.workdps(25):
            f = mp.odefun(lambda t, y: [-mp.mpf(eC) * y[1], mp.mpf(A) * mp.sin(mp.mpf(k) * y[0])],
                          0, [mp.mpf(z_init), mp.mpf(0)])
            ze, de = f(1)
        # z alone would show the 6th-order cosine term (the start has delta = 0); delta
        # carries the 5th-order sine term that dominates the local error
        out.append(max(abs(float(ze) - zf[0]) / tb["zhat"], abs(float(de) - df[0]) / tb["dhat"]))
    return max(out)


def pin_rk4_order(O):
    """RK4 has local error O(h^5): with the step's phase advance halved (V / 4) the one-turn
    error against the exact flow drops ~2^5 = 32-fold at the same amplitude in z."""
    fz = np.array([0.2, 0.5])
    e_hi = _rk4_turn_error(O, 4e6, fz)
    e_lo = _rk4_turn_error(O, 1e6, fz)
    assert e_hi < 1e-7, e_hi
    assert 24 < e_hi / e_lo < 40, (e_hi, e_lo, e_hi / e_lo)


def pin_rk4_jacobian(O):
    """The dual-number Jacobian of one RK4 turn (nonlinear, with eta(delta) and a second RF
    system) is the derivative of the tracked map; its determinant is below 1."""
    r = ring(voltage_V=4.5e6, eta1=ETA1_B, eta2=ETA2_B, harmonic2=2 * RING["harmonic"],
             voltage2_V=1.5e6, phi2_rad=0.0)
    tb = textbook(r)
    d = O.derive(r)
    for fz, fd in ((0.3, 0.2), (0.6, -0.4)):
        z0, dp0 = fz * tb["zhat"], fd * tb["dhat"]
        J = O.jacobian(d, "rk4", z0, dp0, 1)
        hz, hd = 1e-6 * tb["zhat"], 1e-6 * tb["dhat"]
        zp, dpp, *_ = O.track(d, "rk4", [z0 + hz, z0 - hz, z0, z0],
                              [dp0, dp0, dp0 + hd, dp0 - hd], turns=1)
        Jfd = np.array([[(zp[0] - zp[1]) / (2 * hz), (zp[2] - zp[3]) / (2 * hd)],
                        [(dpp[0] - dpp[1]) / (2 * hz), (dpp[2] - dpp[3]) / (2 * hd)]])
        scale = np.array([[1.0, tb["zhat"] / tb["dhat"]], [tb["dhat"] / tb["zhat"], 1.0]])
        assert np.max(np.abs(J - Jfd) / scale) < 1e-6, (J, Jfd)
        assert 0 < np.linalg.det(J) < 1
    # no exact inverse: the oracle refuses sign = -1 for RK4
    try:
        O.track(d, "rk4", [0.1], [0.0], turns=1, sign=-1.0)
    except ValueError:
        pass
    else:
        raise AssertionError("RK4 has no exact inverse map")


def _double_rf(V=4.5e6, ratio=0.3, h2mul=2, phi2=0.0, **over):
    return ring(voltage_V=V, harmonic2=h2mul * RING["harmonic"], voltage2_V=ratio * V,
                phi2_rad=phi2, **over)


def pin_double_rf_linear(O):
    """rf_linear with a second RF system: the linear slope is a = A k cos(phi_s) +
    A2 k2 cos(phi_2) from the textbook constants of both systems, and EC / LF keep their
    closed-form one-turn matrices with that slope; a flat bottom (a = 0) is allowed."""
    for phis, phi2 in ((0.0, 0.0), (0.3, -0.4)):
        r = _double_rf(rf_linear=1.0, phi_s_rad=phis, phi2=phi2)
        tb = textbook(r)
        tb2 = textbook(dict(r, harmonic=r["harmonic2"], voltage_V=r["voltage2_V"], phi_s_rad=phi2))
        d = O.derive(r)
        eC = tb["etaC"]
        a = tb["a"] + tb2["a"]
        K = eC * a
        for scheme, Mc in (("euler_cromer", np.array([[1 - K, -eC], [a, 1.0]])),
                           ("leapfrog", np.array([[1 - K / 2, -eC * (1 - K / 4)], [a, 1 - K / 2]]))):
            M = _linear_matrix(O, d, scheme)
            assert np.all(np.abs(M / Mc - 1) < 1e-12), (scheme, M, Mc)
    # bunch-lengthening flat bottom: V2 = -V/2 at h2 = 2h cancels the linear slope
    flat = _double_rf(ratio=-0.5)
    d = O.derive(flat)
    assert abs(d.K) < 1e-15 and O.derive_rc(_oracle.params(**flat)) == 0
    # and a second system that over-cancels it has no bucket
    assert O.derive_rc(_oracle.params(**_double_rf(ratio=-0.7))) == -2


def _energy_err_rf2(O, scheme, V, turns):
    r = _double_rf(V=V)
    tb = textbook(r)
    d = O.derive(r)
    z, dp = _traj(O, d, scheme, 0.4 * tb["zhat"], 0.0, turns)
    # invariant of the smooth motion with both systems (phi_s = phi_2 = 0)
    H = 0.5 * d.etaC * dp ** 2 + (d.A / d.k) * (1 - np.cos(d.k * z)) \
        + (0.3 * d.A / (2 * d.k)) * (1 - np.cos(2 * d.k * z))
    return np.max(np.abs(H - H[0])) / H[0]


def pin_double_rf_energy(O):
    """The symplectic schemes conserve the two-harmonic Hamiltonian (A2 = 0.3 A at k2 = 2 k,
    both from the textbook scaling) to their order: quartering both voltages divides the
    bounded error by ~2 (EC), ~4 (LF), ~16 (Ruth4)."""
    expect = {"euler_cromer": (1.6, 2.7, 0.05), "leapfrog": (3.2, 5.2, 2e-3),
              "ruth4": (12.0, 24.0, 2e-6)}
    for scheme, (lo, hi, cap) in expect.items():
        e_hi = _energy_err_rf2(O, scheme, 4e6, 6000)
        e_lo = _energy_err_rf2(O, scheme, 1e6, 6000)
        assert e_hi < cap, (scheme, e_hi)
        assert lo < e_hi / e_lo < hi, (scheme, e_hi, e_lo, e_hi / e_lo)


# ---- ramp: a per-turn machine programme (accelerating bucket) ----------------------------


def _linear_ramp(pa, pb, N):
    """Reference momenta p0[0..N] of a linear momentum ramp."""
    return pa + (pb - pa) * np.arange(N + 1) / N


def _ramp_textbook(r, pn, pn1, V):
    """Textbook (a, eta C) of one turn of a ramp: the synchronous particle gains the energy
    E(p0[n+1]) - E(p0[n]) = q V sin(phi_s) per turn (exact energies), phi_s on the stable
    branch (eta cos phi_s > 0)."""
    E0, E1 = math.hypot(pn, r["mass_eV"]), math.hypot(pn1, r["mass_eV"])
    x = (E1 - E0) / V
    g = E0 / r["mass_eV"]
    above = 1.0 / r["gamma_t"] ** 2 - 1.0 / g ** 2 > 0
    phis = math.asin(x) if above else math.pi - math.asin(x)
    tb = textbook(dict(r, p0_eVc=pn, voltage_V=V, phi_s_rad=phis))
    return tb["a"], tb["etaC"], x


def pin_ramp_constant_programme(O):
    """A programme with constant momentum and voltage is the fixed machine: bitwise the
    same particles as the ring's own tracking, every scheme."""
    r = ring(voltage_V=4.5e6)
    d = O.derive(r)
    N = 300
    tc = O.ramp_derive(r, np.full(N, 4.5e6), np.full(N + 1, r["p0_eVc"]))
    z0, dp0 = np.array([0.1, -0.3, 0.5]), np.array([1e-3, 0.0, -2e-3])
    x0, xp0 = np.array([1e-3, 0.0, -2e-3]), np.array([1e-5, -2e-5, 0.0])
    for scheme in ("euler_cromer", "leapfrog", "ruth4"):
        a = O.track(d, scheme, z0, dp0, x0, xp0, x0, xp0, turns=N)
        b = O.track_ramp(d, tc, scheme, z0, dp0, x0, xp0, x0, xp0)
        for u, v in zip(a[:6], b[:6]):
            assert np.array_equal(u, v), scheme


def pin_ramp_synchronous_phase(O):
    """Each turn's synchronous phase gives the synchronous particle the programme's energy
    gain, q V sin(phi_s) = E(p0[n+1]) - E(p0[n]) (exact energies, so the momentum form
    beta dp agrees to second order, ~1e-8), on the branch with eta cos(phi_s) > 0; eta C
    and the kick slope are the textbook ones at the turn's starting momentum; the
    synchronous particle (0, 0) stays there exactly; a voltage too low for the gain has no
    bucket."""
    for pa, pb, label in ((26e9, 30e9, "above"), (10e9, 11e9, "below")):
        r = ring(voltage_V=4.5e6, p0_eVc=pa, phi_s_rad=0.0 if label == "above" else math.pi)
        N = 4000
        p0 = _linear_ramp(pa, pb, N)
        tc = O.ramp_derive(r, np.full(N, 4.5e6), p0)
        for n in (0, N // 2, N - 1):
            a, eC, x = _ramp_textbook(r, p0[n], p0[n + 1], 4.5e6)
            assert abs(tc[n, 3] / x - 1) < 1e-6, (label, n, tc[n, 3], x)
            assert abs(tc[n, 0] / eC - 1) < 1e-12, (label, n)
            # the kick slope A_n k cos(phi_s,n) of turn n is the textbook one at p0[n]
            k = 2 * math.pi * r["harmonic"] / r["circumference_m"]
            assert abs(tc[n, 1] * k * math.cos(tc[n, 2]) / a - 1) < 1e-7, (label, n)
            assert eC * math.cos(tc[n, 2]) > 0, (label, n)
            assert abs(tc[n, 4] * p0[n + 1] / p0[n] - 1) < 1e-15
        d = O.derive(r)
        z, dp, *_ = O.track_ramp(d, tc, "ruth4", [0.0], [0.0])
        assert z[0] == 0.0 and dp[0] == 0.0
    r = ring(voltage_V=4.5e6)
    rc, _ = O.ramp_derive_rc(r, np.full(10, 1e5), _linear_ramp(26e9, 26.01e9, 10))
    assert rc == -2


def pin_ramp_adiabatic_invariant(O):
    """Slow acceleration (rf_linear): the longitudinal action in (z, p0 delta) is an
    adiabatic invariant.  With the textbook invariant of each turn's linear leap-frog
    matrix, J = a z^2 + eta C (1 - K/4) delta^2 (K = eta C a), the action J / sqrt(a eta C
    (1 - K/4)) times p0 stays constant to 2e-3 over a 4e3-turn ramp (about 35 synchrotron
    periods), above and below transition, while the action without p0 changes by 9-13 %."""
    for pa, pb, label in ((26e9, 30e9, "above"), (10e9, 11e9, "below")):
        r = ring(voltage_V=4.5e6, rf_linear=1.0, p0_eVc=pa,
                 phi_s_rad=0.0 if label == "above" else math.pi)
        N = 4000
        p0 = _linear_ramp(pa, pb, N)
        tc = O.ramp_derive(r, np.full(N, 4.5e6), p0)
        d = O.derive(r)
        *_, mom = O.track_ramp(d, tc, "leapfrog", [0.05], [0.0], moments=True, stride=1)
        z, dp = mom[:, 0], mom[:, 1]
        I = np.empty(N + 1)
        for n in range(N + 1):
            pn1 = p0[n + 1] if n < N else p0[N] + (p0[N] - p0[N - 1])
            a, eC, _ = _ramp_textbook(r, p0[n], pn1, 4.5e6)
            b = eC * (1.0 - eC * a / 4.0)
            I[n] = (a * z[n] ** 2 + b * dp[n] ** 2) / math.sqrt(a * b)
        inv = I * p0
        assert np.max(np.abs(inv / inv[0] - 1)) < 2e-3, (label, np.max(np.abs(inv / inv[0] - 1)))
        assert abs(I[-1] / I[0] - 1) > 0.05, label


def pin_ramp_normalised_emittance(O):
    """Transverse adiabatic damping: the slopes follow the reference momentum, so the
    normalised emittance beta gamma eps (Liouville) is conserved through the ramp to
    rounding, while the geometric emittance shrinks as 1 / p0."""
    r = ring(voltage_V=4.5e6)
    N = 2000
    p0 = _linear_ramp(26e9, 30e9, N)
    tc = O.ramp_derive(r, np.full(N, 4.5e6), p0)
    d = O.derive(r)
    rng = np.random.default_rng(11)
    n = 500
    x, xp = rng.normal(0, 1.9e-3, n), rng.normal(0, 3.8e-5, n)
    y, yp = rng.normal(0, 1.9e-3, n), rng.normal(0, 3.8e-5, n)
    z, dp = rng.normal(0, 0.05, n), rng.normal(0, 4e-4, n)
    *_, mom = O.track_ramp(d, tc, "leapfrog", z, dp, x, xp, y, yp, moments=True, stride=N)
    for off in (9, 14):
        e0, e1 = mom[0, off], mom[-1, off]
        en0, en1 = e0 * p0[0] / r["mass_eV"], e1 * p0[N] / r["mass_eV"]
        assert abs(en1 / en0 - 1) < 1e-11, (off, en1 / en0)
        assert abs(e1 / e0 - p0[0] / p0[N]) < 1e-11


# ---- collective step: slicing and a wake kick ------------------------------------------


def _slices_setup(ns=64, lo=-0.8, hi=0.8):
    return ns, lo, hi, ns / (hi - lo), (hi - lo) / ns


def pin_collective_slicing(O):
    """Particles at slice centres with a seeded count pattern are counted slice by slice;
    z_lo belongs to the first slice, z_hi and beyond and below z_lo to none; the counts of
    the inside particles add up to their number; z itself is untouched."""
    ns, lo, hi, inv, dz = _slices_setup()
    rng = np.random.default_rng(5)
    pattern = rng.integers(0, 7, ns)
    z = np.concatenate([np.full(c, lo + (k + 0.5) * dz) for k, c in enumerate(pattern)])
    extra = np.array([lo, hi, hi + 0.3, lo - 1e-9, hi - 1e-9])
    zall = np.concatenate([z, extra])
    z1, dp1, counts, V = O.collective_kick(zall, np.zeros(zall.size), lo, inv, np.zeros(ns), 0.0)
    want = pattern.copy()
    want[0] += 1                     # z_lo
    want[-1] += 1                    # just below z_hi
    assert np.array_equal(counts, want), (counts, want)
    assert counts.sum() == z.size + 2
    assert np.array_equal(z1, zall) and np.all(dp1 == 0.0)


def pin_collective_wake_library(O):
    """The wake potential V_k = sum_{m >= 0} c_{k+m} w_m equals numpy's convolution of the
    reversed counts with the wake table; a delta wake returns the counts, a constant wake
    the number of particles at or ahead of each slice; the head slice feels only itself."""
    ns, lo, hi, inv, dz = _slices_setup()
    rng = np.random.default_rng(6)
    pattern = rng.integers(0, 9, ns)
    z = np.concatenate([np.full(c, lo + (k + 0.5) * dz) for k, c in enumerate(pattern)])
    w = rng.normal(0.0, 1.0, ns)
    _, _, counts, V = O.collective_kick(z, np.zeros(z.size), lo, inv, w, 1.0)
    ref = np.convolve(counts[::-1].astype(float), w)[:ns][::-1]
    assert np.max(np.abs(V - ref)) < 1e-12 * np.max(np.abs(ref)), np.max(np.abs(V - ref))
    delta = np.zeros(ns)
    delta[0] = 1.0
    assert np.array_equal(O.collective_kick(z, np.zeros(z.size), lo, inv, delta, 1.0)[3],
                          counts.astype(float))
    const = O.collective_kick(z, np.zeros(z.size), lo, inv, np.ones(ns), 1.0)[3]
    assert np.array_equal(const, np.cumsum(counts[::-1])[::-1].astype(float))
    # causality: one particle at the head, many behind it; it feels only its own wake
    zc = np.concatenate([np.full(50, lo + 0.5 * dz), [lo + (ns - 0.5) * dz]])
    _, dpc, _, _ = O.collective_kick(zc, np.zeros(zc.size), lo, inv, np.ones(ns), 2.0)
    assert dpc[-1] == 2.0 and np.all(dpc[:-1] == 2.0 * 51)


def pin_collective_kick(O):
    """The kick is alpha times the potential of the particle's own slice; particles outside
    the range are not kicked; alpha = 0 leaves delta bitwise unchanged."""
    ns, lo, hi, inv, dz = _slices_setup()
    rng = np.random.default_rng(7)
    z = rng.uniform(lo - 0.2, hi + 0.2, 3000)
    dp = rng.normal(0, 1e-3, z.size)
    w = np.exp(-np.arange(ns) / 10.0)
    z1, dp1, counts, V = O.collective_kick(z, dp, lo, inv, w, -3e-7)
    k = np.floor((z - lo) * inv).astype(int)
    inside = (k >= 0) & (k < ns)
    assert np.array_equal(dp1[~inside], dp[~inside])
    assert np.max(np.abs(dp1[inside] - (dp[inside] + (-3e-7) * V[k[inside]]))) == 0.0
    assert np.array_equal(O.collective_kick(z, dp, lo, inv, w, 0.0)[1], dp)


def pin_collective_turn_order(O):
    """A turn of the collective tracking is the one-turn map (and the transverse rotation)
    followed by the collective step on the whole bunch; with alpha = 0 it is the plain
    tracking, bitwise, every scheme."""
    ns, lo, hi, inv, dz = _slices_setup()
    r = ring(voltage_V=4.5e6)
    d = O.derive(r)
    rng = np.random.default_rng(8)
    z, dp = rng.normal(0, 0.1, 400), rng.normal(0, 5e-4, 400)
    x, xp = rng.normal(0, 1e-3, 400), rng.normal(0, 2e-5, 400)
    w = 1.0 / (1.0 + np.arange(ns))
    for scheme in ("euler_cromer", "leapfrog", "ruth4", "rk4"):
        a = O.track_collective(d, scheme, z, dp, x, xp, turns=1, z_lo=lo, inv_dz=inv, w=w,
                               alpha=1e-7)
        b = O.track(d, scheme, z, dp, x, xp, turns=1)
        c = O.collective_kick(b[0], b[1], lo, inv, w, 1e-7)
        assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]), scheme
        assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3]), scheme
        e = O.track_collective(d, scheme, z, dp, x, xp, turns=50, z_lo=lo, inv_dz=inv, w=w,
                               alpha=0.0)
        f = O.track(d, scheme, z, dp, x, xp, turns=50)
        for u, v in zip(e[:4], f[:4]):
            assert np.array_equal(u, v), scheme


def pin_collective_space_charge(O):
    """The space-charge term is the slope of the line density: for counts on an exact
    parabola c_k = A - B (k - k0)^2 (the parabolic bunch) the kick is exactly linear in the
    slice, alpha_sc (-2 B (k - k0)) in the interior; a linear profile gives the same slope
    everywhere, ends included (one-sided there); a symmetric profile an antisymmetric
    kick; a flat one none."""
    ns, lo, hi, inv, dz = _slices_setup(ns=41, lo=-1.025, hi=1.025)
    s = 2.0 ** -20
    k = np.arange(ns)

    def kicks(pattern):
        z = np.concatenate([np.full(c, lo + (i + 0.5) * dz) for i, c in enumerate(pattern)])
        _, dp1, counts, _ = O.collective_kick(z, np.zeros(z.size), lo, inv, np.zeros(ns), 0.0, s)
        assert np.array_equal(counts, pattern)
        per_slice = np.full(ns, np.nan)
        idx = np.floor((z - lo) * inv).astype(int)
        per_slice[idx] = dp1
        return per_slice

    B, k0 = 3, 20
    para = 1300 - B * (k - k0) ** 2
    kp = kicks(para)
    assert np.array_equal(kp[1:-1], s * (-2.0 * B * (k[1:-1] - k0)))
    assert np.array_equal(kp[:ns // 2], -kp[ns // 2 + 1:][::-1])
    lin = 5 + 7 * k
    assert np.all(kicks(lin) == s * 7.0)
    assert np.all(kicks(np.full(ns, 9)) == 0.0)


ALL_FAST = (pin_textbook_constants, pin_stability_rules, pin_linear_closed_form,
            pin_pendulum_detuning, pin_separatrix, pin_time_reversal, pin_inverse_map,
            pin_symplectic, pin_energy_order, pin_symmetry_and_fixed_point,
            pin_transverse_rotation, pin_moments, pin_nonlinear_slippage_closed_form,
            pin_nonlinear_slippage_fixed_points, pin_nonlinear_slippage_energy,
            pin_chromatic_phase_sum, pin_nonlinear_inverse_map, pin_nonlinear_symplectic,
            pin_rk4_linear_closed_form, pin_rk4_jacobian, pin_double_rf_linear,
            pin_double_rf_energy, pin_ramp_constant_programme, pin_ramp_synchronous_phase,
            pin_ramp_adiabatic_invariant, pin_ramp_normalised_emittance,
            pin_collective_slicing, pin_collective_wake_library, pin_collective_kick,
            pin_collective_turn_order, pin_collective_space_charge)
# pins that need mpmath (skipped where it is missing)
ALL_MPMATH = (pin_rk4_order,)
