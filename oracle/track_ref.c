/*
 * oracle/track_ref.c -- plain FP64 reference tracker (TEST INFRASTRUCTURE).
 *
 * This file is the oracle that the GPU library is checked against.  It is not
 * part of the product path: only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two meet only in the seeded input
 * generator (which holds no tracking arithmetic).
 *
 * What it computes (Oeftiger 2014, "Parallelisation of PyHEADTAIL"):
 *   - Sec. 1.1.2: each macro-particle's longitudinal coordinates (z, delta) are
 *     integrated turn by turn with Euler-Cromer (1st order), leap-frog (2nd
 *     order Verlet) or a 4th-order Ruth scheme; particles are independent.
 *   - Sec. 1.1.1: the transverse coordinates are pushed by the same linear
 *     transfer matrix every turn.
 *   - Sec. 2.3: two nested loops, turns (sequential) outside, particles
 *     (independent) inside.
 * The paper prints none of the formulas.  The readings used here are the
 * textbook single-harmonic synchrotron map:
 *   kick  K(w):  phi = phi_s + k z;  delta <- delta + w A (sin phi - sin phi_s)
 *   drift D(w):  z <- z - w eta(delta) C delta,  eta(delta) = eta0 + eta1 delta + eta2 delta^2
 *                (the slippage expansion; eta1 = eta2 = 0 is the linear slippage)
 *   EC    = K(1) then D(1)           (momentum first, then position)
 *   LF    = D(1/2) K(1) D(1/2)       (Verlet drift-kick-drift)
 *   RUTH4 = D(t/2) K(t) D((1-t)/2) K(1-2t) D((1-t)/2) K(t) D(t/2),
 *           t = 1/(2 - 2^(1/3))      (Forest & Ruth 1990; Yoshida 1990)
 *   RK4   = classic Runge-Kutta on dz/dn = -eta(delta) C delta, d delta/dn = F(z) over one
 *           turn (Sec. 1.1.2's "Runge-Kutta" read literally; not symplectic, no exact
 *           inverse), F the kick's force per unit weight
 *   double RF (optional): the kick adds w A2 (sin(phi_2 + k2 z) - sin phi_2) with
 *           k2 = 2 pi h2 / C and A2 = q V2 / (beta p0)
 *   transverse, per plane: [u; u'] <- [[cos mu, b sin mu], [-sin mu / b, cos mu]] [u; u']
 *           mu = 2 pi (frac(Q) + xi delta), alpha = 0, with the particle's delta after the
 *           turn's longitudinal step (xi = dQ/d delta, the chromaticity; xi = 0 gives the
 *           same matrix for every particle).
 *   ramp (optional): per-turn eta_n, A_n, phi_s,n from a programme V_n, p0_n, with delta and
 *           the slopes re-expressed by p0_n / p0_{n+1} after each turn
 *   collective step (optional, after each turn): slice counts on a uniform grid, wake
 *           potential V_k = sum_{j >= k} c_j w[j - k], line-density slope D_k (central
 *           difference of the counts), kick delta += alpha V_k + alpha_sc D_k
 * Derived constants (all FP64, from the ring parameters):
 *   beta*gamma = p0/m; gamma = sqrt(1 + (beta gamma)^2); beta = beta gamma / gamma
 *   eta = 1/gamma_t^2 - 1/gamma^2;  k = 2 pi h / C;  A = q V / (beta p0)   [p0 in eV/c]
 * Moments after each recorded turn: means, population rms (two-pass) and the
 * rms emittance sqrt(<u^2><u'^2> - <u u'>^2) of the centred coordinates.
 *
 * Compiled with -O2 -ffp-contract=off (no fused multiply-add): every operation
 * rounds as written.  Parity status: pinned (closed-form linear map, textbook
 * synchrotron tune and bucket height, pendulum detuning, time-reversal
 * symmetry, symplecticity, order scaling, high-precision brute force, exact
 * transverse rotation; for eta(delta): the closed-form drift with the RF off, the
 * fixed points at eta(delta) = 0 and the order of the smooth Hamiltonian's error;
 * for the chromaticity: the summed-angle rotation; for RK4: the Taylor polynomial of
 * the linear flow, its determinant and the 5th-order local error against an
 * mpmath Taylor-series flow; for the second RF system: the combined linear slope and
 * the two-harmonic Hamiltonian's order; for the ramp: the textbook synchronous energy
 * gain, the adiabatic invariant and the normalised emittance; for the collective step:
 * counts of particles placed at slice centres, numpy's convolution, causality and the
 * map-then-kick order); see the tests.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define REF_OK 0
#define REF_E_INVALID (-1)
#define REF_E_UNSTABLE (-2)

enum { REF_EULER_CROMER = 0, REF_LEAPFROG = 1, REF_RUTH4 = 2, REF_RK4 = 3 };

/* Number of moment values per recorded turn, in this order:
 *  0 mean z   1 mean delta   2 rms z   3 rms delta   4 eps_z
 *  5 mean x   6 mean x'      7 rms x   8 rms x'      9 eps_x
 * 10 mean y  11 mean y'     12 rms y  13 rms y'     14 eps_y            */
#define REF_NMOM 15

typedef struct {
    double circumference_m; /* C */
    double gamma_t;         /* transition gamma */
    double p0_eVc;          /* reference momentum in eV/c */
    double mass_eV;         /* rest mass in eV/c^2 */
    double charge_e;        /* charge in units of e */
    double harmonic;        /* RF harmonic number h */
    double voltage_V;       /* RF voltage V */
    double phi_s_rad;       /* synchronous phase */
    double rf_linear;       /* nonzero: sin(phi) - sin(phi_s) -> cos(phi_s) k z */
    double beta_x_m, beta_y_m, Qx, Qy;
    double eta1, eta2;      /* slippage expansion: eta(delta) = eta0 + eta1 delta + eta2 delta^2 */
    double xi_x, xi_y;      /* chromaticities dQ/d delta */
    double harmonic2, voltage2_V, phi2_rad; /* second RF system (voltage2 = 0: none) */
} ref_params;

typedef struct {
    double betagamma, gamma, beta, eta, k, A, etaC, phi_s, sin_phis, cos_phis;
    double K, Qs; /* linear strength eta C A k cos(phi_s) and sqrt(K)/(2 pi) */
    double rf_linear;
    double mx[4], my[4]; /* transverse one-turn matrices, row-major */
    double eta1C, eta2C; /* eta1 C, eta2 C */
    double qx, qy;       /* frac(Qx), frac(Qy) */
    double bx, by;       /* beta functions used by the rotations */
    double xi_x, xi_y;
    double k2, A2, phi2, sin_phi2, cos_phi2; /* second RF system */
} ref_derived;

static const double REF_PI = 3.14159265358979323846;

int ref_derive(const ref_params* p, ref_derived* d)
{
    if (!p || !d) return REF_E_INVALID;
    if (!(p->circumference_m > 0) || !(p->p0_eVc > 0) || !(p->mass_eV > 0) ||
        !(p->gamma_t > 0) || !(p->harmonic > 0))
        return REF_E_INVALID;
    if (!isfinite(p->eta1) || !isfinite(p->eta2) || !isfinite(p->xi_x) || !isfinite(p->xi_y))
        return REF_E_INVALID;
    if (!isfinite(p->voltage2_V) || !isfinite(p->phi2_rad) ||
        (p->voltage2_V != 0.0 && !(p->harmonic2 > 0)))
        return REF_E_INVALID;
    memset(d, 0, sizeof(*d));
    d->betagamma = p->p0_eVc / p->mass_eV;
    d->gamma = sqrt(1.0 + d->betagamma * d->betagamma);
    d->beta = d->betagamma / d->gamma;
    d->eta = 1.0 / (p->gamma_t * p->gamma_t) - 1.0 / (d->gamma * d->gamma);
    d->k = 2.0 * REF_PI * p->harmonic / p->circumference_m;
    d->A = p->charge_e * p->voltage_V / (d->beta * p->p0_eVc);
    d->etaC = d->eta * p->circumference_m;
    d->phi_s = p->phi_s_rad;
    d->sin_phis = sin(p->phi_s_rad);
    d->cos_phis = cos(p->phi_s_rad);
    d->rf_linear = p->rf_linear;
    if (p->voltage2_V != 0.0) {
        d->k2 = 2.0 * REF_PI * p->harmonic2 / p->circumference_m;
        d->A2 = p->charge_e * p->voltage2_V / (d->beta * p->p0_eVc);
        d->phi2 = p->phi2_rad;
        d->sin_phi2 = sin(p->phi2_rad);
        d->cos_phi2 = cos(p->phi2_rad);
    }
    /* linear strength of both systems together */
    d->K = d->etaC * (d->A * d->k * d->cos_phis + d->A2 * d->k2 * d->cos_phi2);
    d->Qs = d->K > 0 ? sqrt(d->K) / (2.0 * REF_PI) : 0.0;

    double mux = 2.0 * REF_PI * (p->Qx - floor(p->Qx));
    double muy = 2.0 * REF_PI * (p->Qy - floor(p->Qy));
    double bx = p->beta_x_m > 0 ? p->beta_x_m : 1.0;
    double by = p->beta_y_m > 0 ? p->beta_y_m : 1.0;
    d->mx[0] = cos(mux);       d->mx[1] = bx * sin(mux);
    d->mx[2] = -sin(mux) / bx; d->mx[3] = cos(mux);
    d->my[0] = cos(muy);       d->my[1] = by * sin(muy);
    d->my[2] = -sin(muy) / by; d->my[3] = cos(muy);
    d->eta1C = p->eta1 * p->circumference_m;
    d->eta2C = p->eta2 * p->circumference_m;
    d->qx = p->Qx - floor(p->Qx);
    d->qy = p->Qy - floor(p->Qy);
    d->bx = bx;
    d->by = by;
    d->xi_x = p->xi_x;
    d->xi_y = p->xi_y;

    /* a zero voltage is a pure drift: allowed.  Otherwise the linearised
     * motion must oscillate: eta cos(phi_s) > 0 and 0 < K < 4; with a second RF system
     * the flat-bottomed bucket K = 0 is allowed too. */
    if (p->voltage_V != 0.0 && p->voltage2_V == 0.0 && !(d->K > 0.0 && d->K < 4.0))
        return REF_E_UNSTABLE;
    if (p->voltage2_V != 0.0 && !(d->K >= 0.0 && d->K < 4.0)) return REF_E_UNSTABLE;
    return REF_OK;
}

/* ---- one stage of the longitudinal map -------------------------------- */

static double ref_force(const ref_derived* d, double z)
{
    if (d->rf_linear != 0.0) return d->cos_phis * d->k * z;
    return sin(d->phi_s + d->k * z) - d->sin_phis;
}

/* the second RF system's force per unit A2 */
static double ref_force2(const ref_derived* d, double z)
{
    if (d->rf_linear != 0.0) return d->cos_phi2 * d->k2 * z;
    return sin(d->phi2 + d->k2 * z) - d->sin_phi2;
}

static void ref_kick(const ref_derived* d, double w, double z, double* dp)
{
    *dp = *dp + (w * d->A) * ref_force(d, z);
    if (d->A2 != 0.0) *dp = *dp + (w * d->A2) * ref_force2(d, z);
}

/* Right-hand side of the smooth motion per turn: dz/dn = -eta(delta) C delta,
 * d delta/dn = A F1(z) + A2 F2(z). */
static void ref_rhs(const ref_derived* d, double z, double dp, double* fz, double* fd)
{
    double etaC = d->etaC + d->eta1C * dp + d->eta2C * dp * dp;
    *fz = -etaC * dp;
    *fd = d->A * ref_force(d, z);
    if (d->A2 != 0.0) *fd = *fd + d->A2 * ref_force2(d, z);
}

/* One classic RK4 step of one turn. */
static void ref_rk4(const ref_derived* d, double* z, double* dp)
{
    double k1z, k1d, k2z, k2d, k3z, k3d, k4z, k4d;
    ref_rhs(d, *z, *dp, &k1z, &k1d);
    ref_rhs(d, *z + 0.5 * k1z, *dp + 0.5 * k1d, &k2z, &k2d);
    ref_rhs(d, *z + 0.5 * k2z, *dp + 0.5 * k2d, &k3z, &k3d);
    ref_rhs(d, *z + k3z, *dp + k3d, &k4z, &k4d);
    *z = *z + (k1z + 2.0 * k2z + 2.0 * k3z + k4z) / 6.0;
    *dp = *dp + (k1d + 2.0 * k2d + 2.0 * k3d + k4d) / 6.0;
}

static void ref_drift(const ref_derived* d, double w, double* z, double dp)
{
    double etaC = d->etaC + d->eta1C * dp + d->eta2C * dp * dp; /* eta(delta) C */
    *z = *z - (w * etaC) * dp;
}

/* Forest-Ruth coefficient t = 1/(2 - 2^(1/3)). */
static double ref_ruth_theta(void) { return 1.0 / (2.0 - cbrt(2.0)); }

/* One turn of the chosen scheme; sign = +1 forward, -1 the exact inverse
 * (stages in reverse order with negated weights). */
static void ref_turn(const ref_derived* d, int scheme, double sign, double* z, double* dp)
{
    if (scheme == REF_RK4) {
        ref_rk4(d, z, dp); /* forward only (no exact inverse) */
    } else if (scheme == REF_EULER_CROMER) {
        if (sign > 0) { ref_kick(d, 1.0, *z, dp); ref_drift(d, 1.0, z, *dp); }
        else          { ref_drift(d, -1.0, z, *dp); ref_kick(d, -1.0, *z, dp); }
    } else if (scheme == REF_LEAPFROG) {
        /* palindromic: the inverse has the same order */
        ref_drift(d, 0.5 * sign, z, *dp);
        ref_kick(d, 1.0 * sign, *z, dp);
        ref_drift(d, 0.5 * sign, z, *dp);
    } else {
        double t = ref_ruth_theta();
        ref_drift(d, 0.5 * t * sign, z, *dp);
        ref_kick(d, t * sign, *z, dp);
        ref_drift(d, 0.5 * (1.0 - t) * sign, z, *dp);
        ref_kick(d, (1.0 - 2.0 * t) * sign, *z, dp);
        ref_drift(d, 0.5 * (1.0 - t) * sign, z, *dp);
        ref_kick(d, t * sign, *z, dp);
        ref_drift(d, 0.5 * t * sign, z, *dp);
    }
}

static void ref_rotate(const double* m, double sign, double* u, double* up)
{
    /* the inverse of [[c, b s], [-s/b, c]] is [[c, -b s], [s/b, c]] */
    double m1 = sign > 0 ? m[1] : -m[1];
    double m2 = sign > 0 ? m[2] : -m[2];
    double un = m[0] * *u + m1 * *up;
    double upn = m2 * *u + m[3] * *up;
    *u = un;
    *up = upn;
}

/* Chromatic rotation of one plane: the phase advance 2 pi (q + xi delta) of this
 * particle; sign = -1 rotates back by the same angle. */
static void ref_rotate_chroma(double q, double xi, double b, double dp, double sign, double* u,
                              double* up)
{
    double mu = 2.0 * REF_PI * (q + xi * dp);
    double c = cos(mu), s = sign * sin(mu);
    double un = c * *u + b * s * *up;
    double upn = -s / b * *u + c * *up;
    *u = un;
    *up = upn;
}

static void ref_transverse(const ref_derived* d, double sign, int dox, int doy, double dp,
                           double* x, double* xp, double* y, double* yp)
{
    if (dox) {
        if (d->xi_x != 0.0) ref_rotate_chroma(d->qx, d->xi_x, d->bx, dp, sign, x, xp);
        else ref_rotate(d->mx, sign, x, xp);
    }
    if (doy) {
        if (d->xi_y != 0.0) ref_rotate_chroma(d->qy, d->xi_y, d->by, dp, sign, y, yp);
        else ref_rotate(d->my, sign, y, yp);
    }
}

/* Two-pass moments of (a, b): mean, population rms and emittance. */
static void ref_pair_moments(const double* a, const double* b, long n, double* out5)
{
    double ma = 0, mb = 0, saa = 0, sbb = 0, sab = 0;
    long i;
    if (n <= 0) { out5[0] = out5[1] = out5[2] = out5[3] = out5[4] = 0.0; return; }
    for (i = 0; i < n; i++) { ma += a[i]; mb += b[i]; }
    ma /= (double)n;
    mb /= (double)n;
    for (i = 0; i < n; i++) {
        double da = a[i] - ma, db = b[i] - mb;
        saa += da * da;
        sbb += db * db;
        sab += da * db;
    }
    saa /= (double)n;
    sbb /= (double)n;
    sab /= (double)n;
    double e2 = saa * sbb - sab * sab;
    out5[0] = ma;
    out5[1] = mb;
    out5[2] = sqrt(saa);
    out5[3] = sqrt(sbb);
    out5[4] = e2 > 0 ? sqrt(e2) : 0.0;
}

void ref_moments(const double* z, const double* dp, const double* x, const double* xp,
                 const double* y, const double* yp, long n, double* out)
{
    int j;
    for (j = 0; j < REF_NMOM; j++) out[j] = 0.0;
    ref_pair_moments(z, dp, n, out);
    if (x && xp) ref_pair_moments(x, xp, n, out + 5);
    if (y && yp) ref_pair_moments(y, yp, n, out + 10);
}

/*
 * Track n particles for `turns` turns.  Any of x..yp may be NULL (plane off).
 * moments: NULL, or an array of (turns/stride + 1) * REF_NMOM doubles; row r
 * holds the moments after turn r*stride (row 0 = the initial state).
 * sign = +1 tracks forward, -1 applies the inverse map.
 */
int ref_track_signed(const ref_derived* d, int scheme, double sign, double* z, double* dp,
                     double* x, double* xp, double* y, double* yp, long n, long turns,
                     double* moments, long stride)
{
    long t, i;
    if (!d || n < 0 || turns < 0 || scheme < 0 || scheme > 3) return REF_E_INVALID;
    if (scheme == REF_RK4 && sign < 0) return REF_E_INVALID; /* no exact inverse */
    if (n > 0 && (!z || !dp)) return REF_E_INVALID;
    if (moments && stride <= 0) return REF_E_INVALID;
    int dox = x && xp, doy = y && yp;
    if (moments) ref_moments(z, dp, dox ? x : 0, dox ? xp : 0, doy ? y : 0, doy ? yp : 0, n, moments);
    for (t = 1; t <= turns; t++) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (i = 0; i < n; i++) {
            /* forward: longitudinal step, then the transverse rotation with the new delta;
             * the inverse undoes them in the opposite order */
            if (sign > 0) {
                ref_turn(d, scheme, sign, &z[i], &dp[i]);
                ref_transverse(d, sign, dox, doy, dp[i], dox ? &x[i] : 0, dox ? &xp[i] : 0,
                               doy ? &y[i] : 0, doy ? &yp[i] : 0);
            } else {
                ref_transverse(d, sign, dox, doy, dp[i], dox ? &x[i] : 0, dox ? &xp[i] : 0,
                               doy ? &y[i] : 0, doy ? &yp[i] : 0);
                ref_turn(d, scheme, sign, &z[i], &dp[i]);
            }
        }
        if (moments && t % stride == 0)
            ref_moments(z, dp, dox ? x : 0, dox ? xp : 0, doy ? y : 0, doy ? yp : 0, n,
                        moments + (t / stride) * REF_NMOM);
    }
    return REF_OK;
}

int ref_track(const ref_derived* d, int scheme, double* z, double* dp, double* x, double* xp,
              double* y, double* yp, long n, long turns, double* moments, long stride)
{
    return ref_track_signed(d, scheme, 1.0, z, dp, x, xp, y, yp, n, turns, moments, stride);
}

/* ---- ramp: a per-turn machine programme (accelerating bucket) ---------- */

/* Per-turn constants of a programme, REF_RAMP_NC doubles per turn:
 *  0 eta_n C   1 A_n = q V_n / (beta_n p0_n)   2 phi_s,n   3 sin(phi_s,n)
 *  4 r_n = p0_n / p0_{n+1}                     5 beta_n gamma_n = p0_n / m       */
#define REF_RAMP_NC 6

/*
 * Derive the per-turn constants of a ramp from the voltage programme V[0..N-1] and the
 * reference momenta p0[0..N] (p0[n] at the start of turn n, p0[n+1] at its end).
 * Reading (the paper changes machine parameters between runs but prints no formulas):
 *   - a particle's momentum grows by q V_n sin(phi) / beta_n per turn (dE = beta c dp),
 *     the synchronous particle's by p0[n+1] - p0[n], so
 *     sin(phi_s,n) = beta_n (p0[n+1] - p0[n]) / (q V_n),
 *     phi_s,n on the branch with eta_n cos(phi_s,n) > 0 (asin above transition,
 *     pi - asin below it);
 *   - turn n runs the scheme's stages with eta_n, A_n and phi_s,n (measured against p0[n],
 *     so the synchronous particle stays at (0, 0) within the turn), then delta and the
 *     transverse slopes are re-expressed against p0[n+1]: delta <- r_n delta,
 *     u' <- r_n u' (for a single kick this is exact: p0[n](1 + delta + A(sin phi -
 *     sin phi_s)) / p0[n+1] - 1 = r_n (delta + A (sin phi - sin phi_s)) - 1 + 1 when the
 *     synchronous gain is p0[n] A sin phi_s).
 * Returns REF_E_INVALID (non-finite or non-positive momenta, V = 0 with a momentum change)
 * or REF_E_UNSTABLE (|sin phi_s| >= 1, or a turn's linear strength outside (0, 4)).
 */
int ref_ramp_derive(const ref_params* p, const double* V, const double* p0, long nturns,
                    double* out)
{
    long t;
    if (!p || nturns < 0 || (nturns > 0 && (!V || !p0 || !out))) return REF_E_INVALID;
    if (!(p->circumference_m > 0) || !(p->mass_eV > 0) || !(p->gamma_t > 0) || !(p->harmonic > 0))
        return REF_E_INVALID;
    double k = 2.0 * REF_PI * p->harmonic / p->circumference_m;
    for (t = 0; t < nturns; t++) {
        double pa = p0[t], pb = p0[t + 1];
        if (!(pa > 0) || !(pb > 0) || !isfinite(pa) || !isfinite(pb) || !isfinite(V[t]))
            return REF_E_INVALID;
        double bg = pa / p->mass_eV;
        double g = sqrt(1.0 + bg * bg);
        double b = bg / g;
        double eta = 1.0 / (p->gamma_t * p->gamma_t) - 1.0 / (g * g);
        double* o = out + t * REF_RAMP_NC;
        o[0] = eta * p->circumference_m;
        o[1] = p->charge_e * V[t] / (b * pa);
        if (V[t] == 0.0) {
            if (pb != pa) return REF_E_INVALID;
            o[2] = 0.0;
            o[3] = 0.0;
        } else {
            double x = b * (pb - pa) / (p->charge_e * V[t]);
            if (!(fabs(x) < 1.0)) return REF_E_UNSTABLE;
            o[2] = eta > 0 ? asin(x) : REF_PI - asin(x);
            o[3] = sin(o[2]); /* the kick's own sin(phi_s): (0, 0) stays fixed exactly */
            double K = o[0] * o[1] * k * cos(o[2]);
            if (!(K > 0.0 && K < 4.0)) return REF_E_UNSTABLE;
        }
        o[4] = pa / pb;
        o[5] = bg;
    }
    return REF_OK;
}

/*
 * Track turns [turn0, turn0 + turns) of a programme (tc from ref_ramp_derive).  The
 * ring's own voltage, phi_s and p0 are replaced turn by turn; the harmonic, gamma_t,
 * the transverse optics and the rf_linear flag are the ring's.  Monitor rows as
 * ref_track.  The programme runs the linear map only (single RF, eta0, no chromaticity).
 */
int ref_track_ramp(const ref_derived* d, const double* tc, long nprog, long turn0, int scheme,
                   double* z, double* dp, double* x, double* xp, double* y, double* yp, long n,
                   long turns, double* moments, long stride)
{
    long t, i;
    if (!d || !tc || n < 0 || turns < 0 || scheme < 0 || scheme > 2) return REF_E_INVALID;
    if (turn0 < 0 || turn0 + turns > nprog) return REF_E_INVALID;
    if (n > 0 && (!z || !dp)) return REF_E_INVALID;
    if (moments && stride <= 0) return REF_E_INVALID;
    if (d->eta1C != 0.0 || d->eta2C != 0.0 || d->xi_x != 0.0 || d->xi_y != 0.0 || d->A2 != 0.0)
        return REF_E_INVALID;
    int dox = x && xp, doy = y && yp;
    if (moments) ref_moments(z, dp, dox ? x : 0, dox ? xp : 0, doy ? y : 0, doy ? yp : 0, n, moments);
    for (t = 1; t <= turns; t++) {
        const double* c = tc + (turn0 + t - 1) * REF_RAMP_NC;
        ref_derived dt = *d;
        dt.etaC = c[0];
        dt.A = c[1];
        dt.phi_s = c[2];
        dt.sin_phis = c[3];
        dt.cos_phis = cos(c[2]);
        double r = c[4];
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (i = 0; i < n; i++) {
            ref_turn(&dt, scheme, 1.0, &z[i], &dp[i]);
            ref_transverse(&dt, 1.0, dox, doy, dp[i], dox ? &x[i] : 0, dox ? &xp[i] : 0,
                           doy ? &y[i] : 0, doy ? &yp[i] : 0);
            /* re-express against the next turn's reference momentum */
            dp[i] = r * dp[i];
            if (dox) xp[i] = r * xp[i];
            if (doy) yp[i] = r * yp[i];
        }
        if (moments && t % stride == 0)
            ref_moments(z, dp, dox ? x : 0, dox ? xp : 0, doy ? y : 0, doy ? yp : 0, n,
                        moments + (t / stride) * REF_NMOM);
    }
    return REF_OK;
}

/* ---- collective step: longitudinal slicing and a wake kick ------------- */

/*
 * The paper's conclusion names collective effects as the next workload after single-
 * particle tracking; it prints no formulas.  The reading (a wake field acting through the
 * bunch's own longitudinal line density):
 *   - slicing: nslices uniform slices on [z_lo, z_hi); particle i lies in slice
 *     k = floor((z_i - z_lo) * inv_dz), inv_dz = nslices / (z_hi - z_lo), when
 *     0 <= k < nslices; c_k counts the particles of slice k;
 *   - wake potential: V_k = sum over j >= k of c_j w[j - k] (z > 0 is ahead: a slice is
 *     affected by the slices ahead of it and by itself, w[m] being the wake of one
 *     macro-particle m slices ahead), summed in order of increasing j;
 *   - space charge: D_k = (c_{k+1} - c_{k-1}) / 2, one-sided (c_1 - c_0, c_{N-1} - c_{N-2})
 *     at the ends and 0 for a single slice: the slope of the line density in counts per
 *     slice (the longitudinal space-charge field is proportional to it);
 *   - kick: delta_i <- delta_i + (alpha V_k(i) + alpha_sc D_k(i)) for the particles inside
 *     the range.
 * inv_dz is passed in (computed once by the caller) so that both implementations decide
 * the slice index from the same two operations.
 */
void ref_slice_counts(const double* z, long n, double z_lo, double inv_dz, long nslices,
                      long* counts)
{
    long i, k;
    for (k = 0; k < nslices; k++) counts[k] = 0;
    for (i = 0; i < n; i++) {
        double u = (z[i] - z_lo) * inv_dz;
        if (u >= 0.0 && u < (double)nslices) {
            k = (long)floor(u);
            if (k < nslices) counts[k]++;
        }
    }
}

void ref_wake_potential(const long* counts, const double* w, long nslices, double* V)
{
    long j, k;
    for (k = 0; k < nslices; k++) {
        double s = 0.0;
        for (j = k; j < nslices; j++) s = s + (double)counts[j] * w[j - k];
        V[k] = s;
    }
}

/* Slope of the line density: central differences of the counts, one-sided at the ends. */
void ref_density_slope(const long* counts, long nslices, double* D)
{
    long k;
    if (nslices == 1) { D[0] = 0.0; return; }
    D[0] = (double)(counts[1] - counts[0]);
    D[nslices - 1] = (double)(counts[nslices - 1] - counts[nslices - 2]);
    for (k = 1; k < nslices - 1; k++) D[k] = 0.5 * (double)(counts[k + 1] - counts[k - 1]);
}

/* One collective step on (z, dp): slice, wake potential, density slope, kick.  counts / V
 * (optional) receive the step's slice counts and wake potential. */
int ref_collective_kick(double* z, double* dp, long n, double z_lo, double inv_dz, long nslices,
                        const double* w, double alpha, double alpha_sc, long* counts, double* V)
{
    long i;
    if (n < 0 || nslices < 1 || !w || (n > 0 && (!z || !dp))) return REF_E_INVALID;
    long* c = counts ? counts : (long*)malloc(sizeof(long) * nslices);
    double* v = V ? V : (double*)malloc(sizeof(double) * nslices);
    double* sd = (double*)malloc(sizeof(double) * nslices);
    if (!c || !v || !sd) return REF_E_INVALID;
    ref_slice_counts(z, n, z_lo, inv_dz, nslices, c);
    ref_wake_potential(c, w, nslices, v);
    ref_density_slope(c, nslices, sd);
    for (i = 0; i < n; i++) {
        double u = (z[i] - z_lo) * inv_dz;
        if (u >= 0.0 && u < (double)nslices) {
            long k = (long)floor(u);
            if (k < nslices) dp[i] = dp[i] + (alpha * v[k] + alpha_sc * sd[k]);
        }
    }
    free(sd);
    if (!counts) free(c);
    if (!V) free(v);
    return REF_OK;
}

/* Track `turns` turns, each the scheme's one-turn map and the transverse rotation
 * (as ref_track), then the collective step on the whole bunch.  Monitor rows after each
 * full turn (collective kick included), as ref_track. */
int ref_track_collective(const ref_derived* d, int scheme, double* z, double* dp, double* x,
                         double* xp, double* y, double* yp, long n, long turns, double z_lo,
                         double inv_dz, long nslices, const double* w, double alpha,
                         double alpha_sc, double* moments, long stride)
{
    long t, i;
    if (!d || n < 0 || turns < 0 || scheme < 0 || scheme > 3) return REF_E_INVALID;
    if (n > 0 && (!z || !dp)) return REF_E_INVALID;
    if (moments && stride <= 0) return REF_E_INVALID;
    if (nslices < 1 || !w) return REF_E_INVALID;
    int dox = x && xp, doy = y && yp;
    long* c = (long*)malloc(sizeof(long) * nslices);
    double* v = (double*)malloc(sizeof(double) * nslices);
    if (!c || !v) { free(c); free(v); return REF_E_INVALID; }
    if (moments) ref_moments(z, dp, dox ? x : 0, dox ? xp : 0, doy ? y : 0, doy ? yp : 0, n, moments);
    for (t = 1; t <= turns; t++) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (i = 0; i < n; i++) {
            ref_turn(d, scheme, 1.0, &z[i], &dp[i]);
            ref_transverse(d, 1.0, dox, doy, dp[i], dox ? &x[i] : 0, dox ? &xp[i] : 0,
                           doy ? &y[i] : 0, doy ? &yp[i] : 0);
        }
        ref_collective_kick(z, dp, n, z_lo, inv_dz, nslices, w, alpha, alpha_sc, c, v);
        if (moments && t % stride == 0)
            ref_moments(z, dp, dox ? x : 0, dox ? xp : 0, doy ? y : 0, doy ? yp : 0, n,
                        moments + (t / stride) * REF_NMOM);
    }
    free(c);
    free(v);
    return REF_OK;
}

/* ---- one-turn Jacobian by forward-mode dual numbers -------------------- */

typedef struct { double v, dz, dd; } ref_dual; /* value and d/dz0, d/ddelta0 */

/* the kick's force A F1(z) + A2 F2(z) and its slope d/dz */
static void ref_force_slope(const ref_derived* d, double z, double* f, double* fp)
{
    if (d->rf_linear != 0.0) { *f = d->A * d->cos_phis * d->k * z; *fp = d->A * d->cos_phis * d->k; }
    else { double ph = d->phi_s + d->k * z; *f = d->A * (sin(ph) - d->sin_phis); *fp = d->A * d->k * cos(ph); }
    if (d->A2 != 0.0) {
        if (d->rf_linear != 0.0) { *f += d->A2 * d->cos_phi2 * d->k2 * z; *fp += d->A2 * d->cos_phi2 * d->k2; }
        else { double ph = d->phi2 + d->k2 * z; *f += d->A2 * (sin(ph) - d->sin_phi2); *fp += d->A2 * d->k2 * cos(ph); }
    }
}

/* dual right-hand side of the smooth motion (RK4) */
static void ref_dual_rhs(const ref_derived* d, ref_dual z, ref_dual dp, ref_dual* fz, ref_dual* fd)
{
    double x = dp.v, f, fp;
    double etaC = d->etaC + d->eta1C * x + d->eta2C * x * x;
    double gp = d->etaC + 2.0 * d->eta1C * x + 3.0 * d->eta2C * x * x;
    fz->v = -etaC * x; fz->dz = -gp * dp.dz; fz->dd = -gp * dp.dd;
    ref_force_slope(d, z.v, &f, &fp);
    fd->v = f; fd->dz = fp * z.dz; fd->dd = fp * z.dd;
}

static ref_dual ref_dual_axpy(double a, ref_dual x, ref_dual y) /* y + a x */
{
    ref_dual r = {y.v + a * x.v, y.dz + a * x.dz, y.dd + a * x.dd};
    return r;
}

static void ref_dual_rk4(const ref_derived* d, ref_dual* z, ref_dual* dp)
{
    ref_dual k1z, k1d, k2z, k2d, k3z, k3d, k4z, k4d;
    ref_dual_rhs(d, *z, *dp, &k1z, &k1d);
    ref_dual_rhs(d, ref_dual_axpy(0.5, k1z, *z), ref_dual_axpy(0.5, k1d, *dp), &k2z, &k2d);
    ref_dual_rhs(d, ref_dual_axpy(0.5, k2z, *z), ref_dual_axpy(0.5, k2d, *dp), &k3z, &k3d);
    ref_dual_rhs(d, ref_dual_axpy(1.0, k3z, *z), ref_dual_axpy(1.0, k3d, *dp), &k4z, &k4d);
    ref_dual sz = ref_dual_axpy(2.0, k3z, ref_dual_axpy(2.0, k2z, k1z));
    ref_dual sd = ref_dual_axpy(2.0, k3d, ref_dual_axpy(2.0, k2d, k1d));
    *z = ref_dual_axpy(1.0 / 6.0, ref_dual_axpy(1.0, k4z, sz), *z);
    *dp = ref_dual_axpy(1.0 / 6.0, ref_dual_axpy(1.0, k4d, sd), *dp);
}

static void ref_dual_turn(const ref_derived* d, int scheme, ref_dual* z, ref_dual* dp)
{
    /* the same stage sequence as ref_turn, carrying the tangent vectors */
    double ws_d[4], ws_k[3];
    int nd, nk, s;
    if (scheme == REF_RK4) { ref_dual_rk4(d, z, dp); return; }
    if (scheme == REF_EULER_CROMER) { nk = 1; ws_k[0] = 1.0; nd = 1; ws_d[0] = 1.0; }
    else if (scheme == REF_LEAPFROG) { nd = 2; ws_d[0] = ws_d[1] = 0.5; nk = 1; ws_k[0] = 1.0; }
    else {
        double t = ref_ruth_theta();
        nd = 4; ws_d[0] = ws_d[3] = 0.5 * t; ws_d[1] = ws_d[2] = 0.5 * (1.0 - t);
        nk = 3; ws_k[0] = ws_k[2] = t; ws_k[1] = 1.0 - 2.0 * t;
    }
    /* EC starts with a kick; LF and RUTH4 alternate starting with a drift */
    int di = 0, ki = 0;
    int nstages = nd + nk;
    for (s = 0; s < nstages; s++) {
        int is_kick = (scheme == REF_EULER_CROMER) ? (s == 0) : (s % 2 == 1);
        if (is_kick) {
            double w = ws_k[ki++], f, fp;
            ref_force_slope(d, z->v, &f, &fp);
            dp->v = dp->v + w * f;
            dp->dz = dp->dz + w * fp * z->dz;
            dp->dd = dp->dd + w * fp * z->dd;
        } else {
            /* z -= w g(delta), g(delta) = eta(delta) C delta, g' = etaC + 2 eta1C delta + 3 eta2C delta^2 */
            double w = ws_d[di++];
            double x = dp->v;
            double etaC = d->etaC + d->eta1C * x + d->eta2C * x * x;
            double gp = d->etaC + 2.0 * d->eta1C * x + 3.0 * d->eta2C * x * x;
            z->v = z->v - (w * etaC) * x;
            z->dz = z->dz - w * gp * dp->dz;
            z->dd = z->dd - w * gp * dp->dd;
        }
    }
}

/* J = d(z1, delta1)/d(z0, delta0) after `turns` turns, row-major 2x2. */
int ref_jacobian(const ref_derived* d, int scheme, double z0, double dp0, long turns, double* J)
{
    if (!d || !J || scheme < 0 || scheme > 3 || turns < 0) return REF_E_INVALID;
    ref_dual z = {z0, 1.0, 0.0}, dp = {dp0, 0.0, 1.0};
    long t;
    for (t = 0; t < turns; t++) ref_dual_turn(d, scheme, &z, &dp);
    J[0] = z.dz; J[1] = z.dd; J[2] = dp.dz; J[3] = dp.dd;
    return REF_OK;
}

int ref_num_threads(void)
{
#ifdef _OPENMP
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    return 1;
#endif
}

/* Threads of the calling thread's later parallel loops (n >= 1), for timing the oracle
 * single-threaded and on all cores; returns the count now in effect.  Test
 * infrastructure only: it changes no arithmetic. */
int ref_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return ref_num_threads();
}
