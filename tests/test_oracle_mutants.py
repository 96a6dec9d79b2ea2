"""Each pin set must have teeth: a copy of the oracle with one plausible mistake planted
(a flipped sign, a dropped term, a wrong coefficient, a transposed operand) must fail at
least one of the independent pins in pins.py.  The mistakes are planted in a temporary
copy of the C source, on the CPU; the real oracle is never modified."""
import os

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "track_ref.c")

MUTANTS = {
    "drift_sign": ("*z = *z - (w * etaC) * dp;", "*z = *z + (w * etaC) * dp;"),
    "eta1_sign": ("d->etaC + d->eta1C * dp + d->eta2C * dp * dp; /* eta(delta) C */",
                  "d->etaC - d->eta1C * dp + d->eta2C * dp * dp; /* eta(delta) C */"),
    "eta2_wrong_power": ("d->etaC + d->eta1C * dp + d->eta2C * dp * dp; /* eta(delta) C */",
                         "d->etaC + d->eta1C * dp + d->eta2C * dp; /* eta(delta) C */"),
    "eta1_from_eta2": ("d->eta1C = p->eta1 * p->circumference_m;",
                       "d->eta1C = p->eta2 * p->circumference_m;"),
    "chroma_sign": ("double mu = 2.0 * REF_PI * (q + xi * dp);",
                    "double mu = 2.0 * REF_PI * (q - xi * dp);"),
    "chroma_no_2pi": ("double mu = 2.0 * REF_PI * (q + xi * dp);",
                      "double mu = 2.0 * REF_PI * q + xi * dp;"),
    "chroma_beta_misplaced": ("double un = c * *u + b * s * *up;\n    double upn = -s / b * *u + c * *up;",
                              "double un = c * *u + s / b * *up;\n    double upn = -s * b * *u + c * *up;"),
    "chroma_old_delta": ("""            if (sign > 0) {
                ref_turn(d, scheme, sign, &z[i], &dp[i]);
                ref_transverse(d, sign, dox, doy, dp[i], dox ? &x[i] : 0, dox ? &xp[i] : 0,
                               doy ? &y[i] : 0, doy ? &yp[i] : 0);""",
                         """            if (sign > 0) {
                ref_transverse(d, sign, dox, doy, dp[i], dox ? &x[i] : 0, dox ? &xp[i] : 0,
                               doy ? &y[i] : 0, doy ? &yp[i] : 0);
                ref_turn(d, scheme, sign, &z[i], &dp[i]);"""),
    "chroma_plane_swapped": ("if (d->xi_x != 0.0) ref_rotate_chroma(d->qx, d->xi_x, d->bx, dp, sign, x, xp);",
                             "if (d->xi_x != 0.0) ref_rotate_chroma(d->qx, d->xi_y, d->bx, dp, sign, x, xp);"),
    "rk4_k2_weight": ("*z = *z + (k1z + 2.0 * k2z + 2.0 * k3z + k4z) / 6.0;",
                      "*z = *z + (k1z + 1.0 * k2z + 2.0 * k3z + k4z) / 6.0;"),
    "rk4_midpoint": ("ref_rhs(d, *z + 0.5 * k1z, *dp + 0.5 * k1d, &k2z, &k2d);",
                     "ref_rhs(d, *z + k1z, *dp + k1d, &k2z, &k2d);"),
    "rk4_last_stage_half": ("ref_rhs(d, *z + k3z, *dp + k3d, &k4z, &k4d);",
                            "ref_rhs(d, *z + 0.5 * k3z, *dp + 0.5 * k3d, &k4z, &k4d);"),
    "rk4_rhs_linear_slip": ("    *fz = -etaC * dp;", "    *fz = -d->etaC * dp;"),
    "rf2_k2_from_h": ("d->k2 = 2.0 * REF_PI * p->harmonic2 / p->circumference_m;",
                      "d->k2 = 2.0 * REF_PI * p->harmonic / p->circumference_m;"),
    "rf2_A2_without_beta": ("d->A2 = p->charge_e * p->voltage2_V / (d->beta * p->p0_eVc);",
                            "d->A2 = p->charge_e * p->voltage2_V / (p->p0_eVc);"),
    "rf2_kick_sign": ("if (d->A2 != 0.0) *dp = *dp + (w * d->A2) * ref_force2(d, z);",
                      "if (d->A2 != 0.0) *dp = *dp - (w * d->A2) * ref_force2(d, z);"),
    "rf2_linear_drops_cos": ("if (d->rf_linear != 0.0) return d->cos_phi2 * d->k2 * z;",
                             "if (d->rf_linear != 0.0) return d->k2 * z;"),
    "inverse_order_chroma": ("""            } else {
                ref_transverse(d, sign, dox, doy, dp[i], dox ? &x[i] : 0, dox ? &xp[i] : 0,
                               doy ? &y[i] : 0, doy ? &yp[i] : 0);
                ref_turn(d, scheme, sign, &z[i], &dp[i]);
            }""",
                             """            } else {
                ref_turn(d, scheme, sign, &z[i], &dp[i]);
                ref_transverse(d, sign, dox, doy, dp[i], dox ? &x[i] : 0, dox ? &xp[i] : 0,
                               doy ? &y[i] : 0, doy ? &yp[i] : 0);
            }"""),
    "lf_half_weight": ("ref_drift(d, 0.5 * sign, z, *dp);\n        ref_kick(d, 1.0 * sign",
                       "ref_drift(d, 0.45 * sign, z, *dp);\n        ref_kick(d, 1.0 * sign"),
    "ruth_theta": ("cbrt(2.0)", "sqrt(2.0)"),
    "ruth_middle_kick": ("ref_kick(d, (1.0 - 2.0 * t) * sign", "ref_kick(d, (1.0 - t) * sign"),
    "A_without_beta": ("(d->beta * p->p0_eVc)", "(p->p0_eVc)"),
    "k_without_2": ("d->k = 2.0 * REF_PI * p->harmonic", "d->k = REF_PI * p->harmonic"),
    "kick_drops_sin_phis": ("return sin(d->phi_s + d->k * z) - d->sin_phis;",
                            "return sin(d->phi_s + d->k * z);"),
    "linear_drops_cos_phis": ("return d->cos_phis * d->k * z;", "return d->k * z;"),
    "beta_misplaced": ("d->mx[1] = bx * sin(mux);", "d->mx[1] = sin(mux) / bx;"),
    "tune_plane_swapped": ("double mux = 2.0 * REF_PI * (p->Qx - floor(p->Qx));",
                           "double mux = 2.0 * REF_PI * (p->Qy - floor(p->Qy));"),
    "ec_drift_first": ("if (sign > 0) { ref_kick(d, 1.0, *z, dp); ref_drift(d, 1.0, z, *dp); }",
                       "if (sign > 0) { ref_drift(d, 1.0, z, *dp); ref_kick(d, 1.0, *z, dp); }"),
    "variance_n_minus_1": ("saa /= (double)n;", "saa /= (double)(n - 1);"),
    "emittance_drops_cov": ("double e2 = saa * sbb - sab * sab;", "double e2 = saa * sbb;"),
    "eta_sign": ("d->eta = 1.0 / (p->gamma_t * p->gamma_t) - 1.0 / (d->gamma * d->gamma);",
                 "d->eta = 1.0 / (d->gamma * d->gamma) - 1.0 / (p->gamma_t * p->gamma_t);"),
    "gamma_from_p_over_m": ("d->gamma = sqrt(1.0 + d->betagamma * d->betagamma);",
                            "d->gamma = d->betagamma;"),
    "ramp_no_rescale": ("            dp[i] = r * dp[i];\n", "            dp[i] = dp[i];\n"),
    "ramp_rescale_inverted": ("        o[4] = pa / pb;", "        o[4] = pb / pa;"),
    "ramp_slopes_not_damped": ("            if (dox) xp[i] = r * xp[i];", "            if (dox) xp[i] = xp[i];"),
    "ramp_phis_branch": ("o[2] = eta > 0 ? asin(x) : REF_PI - asin(x);", "o[2] = asin(x);"),
    "ramp_gain_without_beta": ("double x = b * (pb - pa) / (p->charge_e * V[t]);",
                               "double x = (pb - pa) / (p->charge_e * V[t]);"),
    "ramp_eta_from_end_momentum": ("double bg = pa / p->mass_eV;", "double bg = pb / p->mass_eV;"),
    "wake_direction_reversed": ("for (j = k; j < nslices; j++) s = s + (double)counts[j] * w[j - k];",
                                "for (j = 0; j <= k; j++) s = s + (double)counts[j] * w[k - j];"),
    "wake_index_off_by_one": ("s = s + (double)counts[j] * w[j - k];",
                              "s = s + (double)counts[j] * w[j - k + (j + 1 < nslices)];"),
    "slice_round_not_floor": ("            k = (long)floor(u);\n            if (k < nslices) counts[k]++;",
                              "            k = (long)floor(u + 0.5);\n            if (k < nslices) counts[k]++;"),
    "slice_includes_z_hi": ("        if (u >= 0.0 && u < (double)nslices) {\n            k = (long)floor(u);",
                            "        if (u >= 0.0 && u <= (double)nslices) {\n            k = (long)floor(u) - (u == (double)nslices);"),
    "collective_kick_sign": ("if (k < nslices) dp[i] = dp[i] + (alpha * v[k] + alpha_sc * sd[k]);",
                             "if (k < nslices) dp[i] = dp[i] + (-alpha * v[k] + alpha_sc * sd[k]);"),
    "space_charge_sign": ("if (k < nslices) dp[i] = dp[i] + (alpha * v[k] + alpha_sc * sd[k]);",
                          "if (k < nslices) dp[i] = dp[i] + (alpha * v[k] - alpha_sc * sd[k]);"),
    "space_charge_forward_difference": ("D[k] = 0.5 * (double)(counts[k + 1] - counts[k - 1]);",
                                        "D[k] = (double)(counts[k + 1] - counts[k]);"),
    "space_charge_end_zero": ("D[0] = (double)(counts[1] - counts[0]);", "D[0] = 0.0;"),
    "collective_before_map": ("""        for (i = 0; i < n; i++) {
            ref_turn(d, scheme, 1.0, &z[i], &dp[i]);
            ref_transverse(d, 1.0, dox, doy, dp[i], dox ? &x[i] : 0, dox ? &xp[i] : 0,
                           doy ? &y[i] : 0, doy ? &yp[i] : 0);
        }
        ref_collective_kick(z, dp, n, z_lo, inv_dz, nslices, w, alpha, alpha_sc, c, v);""",
                              """        ref_collective_kick(z, dp, n, z_lo, inv_dz, nslices, w, alpha, alpha_sc, c, v);
        for (i = 0; i < n; i++) {
            ref_turn(d, scheme, 1.0, &z[i], &dp[i]);
            ref_transverse(d, 1.0, dox, doy, dp[i], dox ? &x[i] : 0, dox ? &xp[i] : 0,
                           doy ? &y[i] : 0, doy ? &yp[i] : 0);
        }"""),
    "ramp_A_from_end_momentum": ("o[1] = p->charge_e * V[t] / (b * pa);",
                                 "o[1] = p->charge_e * V[t] / (b * pb);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation site for {name} not found"
    src = tmp_path / "track_ref.c"
    src.write_text(text.replace(old, new, 1))
    lib = oracle.build(openmp=False, force=True, src=str(src), out=str(tmp_path / "libm.so"))
    O = oracle.Oracle(lib)
    caught = []
    extra = ()
    try:
        import mpmath  # noqa: F401
        extra = pins.ALL_MPMATH
    except ImportError:
        pass
    for pin in pins.ALL_FAST + extra:
        try:
            pin(O)
        except (AssertionError, ValueError, ZeroDivisionError, FloatingPointError):
            caught.append(pin.__name__)
    assert caught, f"no independent pin catches the mutant {name}"
