/*
 * phtl.h -- C ABI of libphtl.so: GB300-native (sm_103a) turn-by-turn macro-particle
 * tracking, after A. Oeftiger, "Parallelisation of PyHEADTAIL" (2014).
 *
 * What the library computes (the paper names the schemes but prints no formulas; the
 * readings below are the textbook synchrotron map):
 *   Sec. 1.1.2  longitudinal phase space (z, delta), integrated turn by turn for each
 *               macro-particle independently, by Euler-Cromer (1st order), leap-frog
 *               (2nd-order Verlet, drift-kick-drift), a 4th-order Ruth scheme or classic
 *               RK4 (see PHTL_RK4):
 *                 kick  K(w): phi = phi_s + k z;  delta += w A (sin phi - sin phi_s)
 *                 drift D(w): z -= w eta(delta) C delta,
 *                             eta(delta) = eta0 + eta1 delta + eta2 delta^2
 *                 EC = K(1) D(1);  LF = D(1/2) K(1) D(1/2);
 *                 RUTH4 = D(t/2) K(t) D((1-t)/2) K(1-2t) D((1-t)/2) K(t) D(t/2),
 *                         t = 1/(2 - 2^(1/3))  (Forest & Ruth 1990)
 *               with k = 2 pi h / C, A = q V / (beta p0) [p0 in eV/c],
 *               eta0 = 1/gamma_t^2 - 1/gamma^2 (eta1 = eta2 = 0: linear slippage; the
 *               paper's profile evaluates eta per drift from delta, Fig. cprof).
 *   Sec. 1.1.1  transverse (x, x', y, y'): the same linear transfer matrix every turn,
 *               [u; u'] <- [[cos mu, b sin mu], [-sin mu / b, cos mu]] [u; u'],
 *               mu = 2 pi (frac(Q) + xi delta), alpha = 0; with a chromaticity xi != 0
 *               each particle turns by its own angle, delta taken after the turn's
 *               longitudinal step (xi = 0: one matrix for all).
 *   Sec. 2.3    particles are independent, turns are sequential; the turn loop runs
 *               inside the kernel (state in registers), bounded per launch.
 * Per-turn bunch moments are accumulated into a caller-owned monitor buffer.  Beyond the
 * single-harmonic map: a second RF system (phtl_params.voltage2_V), a ramp programme
 * (phtl_set_programme) and a collective step of slicing, wake and space-charge kick
 * (phtl_set_wake), each stated where it is declared.
 *
 * Logging: with the environment variable PHTL_LOG set to 1 (or higher) when the library is
 * first used, each tracking call, batch and serving event prints one line to stderr
 * ("phtl: ..."): the entry point, sizes, integrator, arithmetic and launch shape.
 *
 * Conventions for every entry point:
 *   - Return value: PHTL_OK (0) or a negative PHTL_E_* code.  No C++ exception
 *     crosses this boundary.  phtl_strerror() names a code.
 *   - Particle and monitor buffers are owned by the caller and are never freed by the
 *     library.  "Device pointer" means memory the current CUDA device can address
 *     (cudaMalloc / PyTorch CUDA tensors).  The library owns handles, internal
 *     tables, CUDA graphs and pinned staging buffers, and frees them in phtl_destroy.
 *   - Stream-ordered calls (phtl_track, phtl_track_perturn, phtl_track_batched) only
 *     enqueue work on the given stream (NULL = the legacy default stream) and return;
 *     device-side faults surface at the caller's next synchronisation.  The caller
 *     must not free or reuse the buffers until that work has completed.
 *   - n == 0 or turns == 0 is a valid no-op (PHTL_OK), except that a monitor row 0
 *     is still written when a monitor is set.
 *   - A handle may be used from one host thread at a time; the serving calls
 *     (phtl_server_*, phtl_submit, phtl_poll, phtl_cancel) are internally locked and
 *     may be called from any thread.
 */
#ifndef PHTL_H
#define PHTL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------------------ */
#define PHTL_OK 0
#define PHTL_E_INVALID (-1)   /* null pointer, bad enum, negative size, misalignment */
#define PHTL_E_UNSTABLE (-2)  /* RF parameters give no stable bucket (0 < K < 4 fails) */
#define PHTL_E_NOMEM (-3)     /* device or host allocation failed / over the budget   */
#define PHTL_E_CUDA (-4)      /* a CUDA runtime call failed                           */
#define PHTL_E_TIMEOUT (-5)   /* a wait reached its deadline                          */
#define PHTL_E_CANCELLED (-6) /* the job was cancelled                                */
#define PHTL_E_BADHANDLE (-7) /* null, destroyed or foreign handle / unknown ticket   */
#define PHTL_E_NODEVICE (-8)  /* no CUDA device, or not an sm_103 device              */
#define PHTL_E_TOOBIG (-9)    /* more jobs than phtl_batch_run_noalloc's fixed table   */
#define PHTL_E_CAPTURE (-10)  /* the stream is capturing a CUDA graph and the call      */
                              /* cannot be recorded into one                          */

/* ---- enums ------------------------------------------------------------------------- */
/* PHTL_RK4: classic 4th-order Runge-Kutta on the smooth motion per turn, dz/dn = -eta(d) C d,
 * dd/dn = A F1(z) + A2 F2(z) (Sec. 1.1.2's "Runge-Kutta" read literally): four force
 * evaluations per turn, not symplectic, forward only.  It runs in the widened map's
 * kernels (every dtype).                                                             */
enum { PHTL_EULER_CROMER = 0, PHTL_LEAPFROG = 1, PHTL_RUTH4 = 2, PHTL_RK4 = 3 };

/* Arithmetic of the particle state.
 *  PHTL_F64   : every coordinate buffer holds n doubles.
 *  PHTL_F32C  : FP32 compensated (double-float, ~48 bits).  Every coordinate buffer
 *               holds 2n floats: [hi(0..n-1) | comp(0..n-1)]; the value of particle i is
 *               hi[i] + comp[i].  Increments are double-float products of the FP64
 *               coefficients (split into hi + lo floats) and the pair, added with
 *               TwoSum and renormalised with Fast2Sum.  The RF phase argument is formed
 *               in FP64 from hi + comp; the sine is the library's double-float sine
 *               (~4e-12 absolute on the bucket).
 *  PHTL_F32CD : as PHTL_F32C, but the phase argument is formed in double-float (FP32
 *               pair) arithmetic instead of FP64 (no FP64 instruction on the path).
 *  PHTL_F32CS : FP32 increments (coefficients split into hi + lo, TwoSum accumulation),
 *               the phase rounded to FP32 and the SFU's sine (__sinf, absolute error
 *               ~2^-21 on [-pi, pi]): fastest, least accurate over long horizons.    */
enum { PHTL_F64 = 0, PHTL_F32C = 1, PHTL_F32CD = 2, PHTL_F32CS = 3 };

/* ---- machine description ----------------------------------------------------------- */
typedef struct phtl_params {
    double circumference_m; /* C > 0                                                  */
    double gamma_t;         /* transition gamma > 0                                   */
    double p0_eVc;          /* reference momentum [eV/c] > 0                          */
    double mass_eV;         /* rest mass [eV/c^2] > 0                                 */
    double charge_e;        /* charge [e]                                             */
    double voltage_V;       /* RF voltage [V]; 0 = pure drift                         */
    double phi_s_rad;       /* synchronous phase                                      */
    double beta_x_m;        /* beta functions for the transverse matrices (> 0)       */
    double beta_y_m;
    double Qx;              /* betatron tunes; only frac(Q) enters                    */
    double Qy;
    int32_t harmonic;       /* RF harmonic number h > 0                               */
    int32_t rf_linear;      /* nonzero: sin(phi) - sin(phi_s) -> cos(phi_s) k z      */
    /* Widened map (all 0 = the linear slippage and achromatic rotation above):      */
    double eta1, eta2;      /* slippage expansion eta(d) = eta0 + eta1 d + eta2 d^2 in  */
                            /* the drift, z <- z - w eta(d) C d (eta0 from gamma_t)    */
    double xi_x, xi_y;      /* chromaticities dQ/dd: per plane the phase advance is     */
                            /* 2 pi (frac(Q) + xi d), d after the turn's longitudinal  */
                            /* step                                                    */
    /* Second RF system (double RF; voltage2_V = 0: none).  Each kick K(w) adds        */
    /* w A2 (sin(phi2 + k2 z) - sin(phi2)), k2 = 2 pi harmonic2 / C,                   */
    /* A2 = q voltage2_V / (beta p0); in rf_linear mode the bracket is cos(phi2) k2 z.  */
    /* It belongs to the ring: batched and served jobs override voltage_V only.        */
    double voltage2_V;      /* second system's voltage [V]                             */
    double phi2_rad;        /* its phase at z = 0                                       */
    int32_t harmonic2;      /* its harmonic number (> 0 when voltage2_V != 0)           */
    int32_t pad2_;
} phtl_params;

/* Constants derived in FP64 on the host by phtl_create. */
typedef struct phtl_derived {
    double betagamma, gamma, beta;
    double eta;        /* slip factor                                              */
    double k;          /* 2 pi h / C [1/m]                                         */
    double A;          /* kick amplitude q V / (beta p0)                           */
    double etaC;       /* eta * C [m]                                              */
    double sin_phis, cos_phis;
    double K;          /* linear strength eta C (A k cos(phi_s) + A2 k2 cos(phi2))  */
    double Qs;         /* sqrt(K) / (2 pi)                                         */
    double bucket_half_length_m; /* pi / k                                        */
    double bucket_half_height;   /* 2 sqrt(A / (k eta C)) (stationary bucket)      */
    double mx[4], my[4];         /* transverse one-turn matrices, row-major        */
} phtl_derived;

typedef struct phtl_handle phtl_handle; /* opaque, library-owned */

/* ---- monitor ------------------------------------------------------------------------ */
/* One monitor row = PHTL_MON_FIELDS doubles of raw sums over the particles:
 *   0 n      1 sum z    2 sum d    3 sum z^2   4 sum d^2   5 sum z d
 *   6 sum x  7 sum x'   8 sum x^2  9 sum x'^2 10 sum x x'
 *  11 sum y 12 sum y'  13 sum y^2 14 sum y'^2 15 sum y y'
 * (d = delta).  Row r holds the sums after turn r*stride of the call (row 0 = the
 * state the call started from).  Sums are FP64, accumulated with device atomics,
 * so their last bits depend on the order the GPU happens to add them in.          */
#define PHTL_MON_FIELDS 16

/* ---- lifetime ----------------------------------------------------------------------- */

/* Validate the parameters and derive the FP64 constants (Sec. 1.1.2 map, see above).
 * Pure host work: touches no GPU.  *out receives a new handle on PHTL_OK.
 * Errors: PHTL_E_INVALID (null, non-positive C/p0/mass/gamma_t/h/beta, a non-finite
 *         eta1/eta2/xi/voltage2/phi2, voltage2 != 0 with harmonic2 <= 0),
 *         PHTL_E_UNSTABLE (single RF: V != 0 and not 0 < K < 4; double RF: not
 *         0 <= K < 4, K = 0 being the flat-bottomed bucket).                          */
int phtl_create(const phtl_params* params, phtl_handle** out);

/* Stop the server if running, wait for the handle's streams, free everything the
 * library owns.  Caller buffers are not touched.  Errors: PHTL_E_BADHANDLE.       */
int phtl_destroy(phtl_handle* h);

/* Copy the derived constants.  Host only.                                        */
int phtl_get_derived(const phtl_handle* h, phtl_derived* out);

/* Human-readable name of an error code (static string, never NULL).              */
const char* phtl_strerror(int code);

/* ---- configuration ------------------------------------------------------------------- */

/* Attach a monitor to subsequent phtl_track / phtl_track_perturn calls.
 * rows: device pointer to capacity_rows * PHTL_MON_FIELDS doubles, caller-owned, or
 * NULL to detach.  stride >= 1: record every stride-th turn.  Each tracking call
 * first zeroes the rows it will write (turns/stride + 1 rows, stream-ordered) and
 * fails with PHTL_E_INVALID if capacity_rows is smaller than that.               */
int phtl_set_monitor(phtl_handle* h, double* rows, int64_t capacity_rows, int64_t stride);

/* Kernel shape: block_threads in {32..256, multiple of 32} or 0 = automatic;
 * turns_per_launch >= 1 or 0 = automatic (bounded launch time, Sec. 2.3's hybrid
 * loop); max_blocks >= 1 caps the grid of the persistent kernel (its blocks then walk
 * the particle chunks in a grid-stride loop) or 0 = the device's resident capacity.
 * Host only.                                                                      */
int phtl_set_tuning(phtl_handle* h, int32_t block_threads, int64_t turns_per_launch,
                    int32_t max_blocks);

/* ---- tracking (stream-ordered) ------------------------------------------------------- */

/* Track n particles for `turns` turns with the persistent multi-turn kernel
 * (Sec. 2.3: turn loop inside the kernel, state in registers; the host splits the
 * turns into bounded launches).
 * z, dp: device pointers (required when n > 0).  x, xp / y, yp: device pointers, or
 * both NULL to leave that plane out.  Layout: PHTL_F64 -> n doubles per coordinate;
 * PHTL_F32C / PHTL_F32CD / PHTL_F32CS -> 2n floats per coordinate ([hi | comp]).  Pointers must be
 * aligned to the element size; 16-byte alignment enables 128-bit loads.
 * integrator: PHTL_EULER_CROMER | PHTL_LEAPFROG | PHTL_RUTH4 | PHTL_RK4.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Updates the buffers in place.  Errors: PHTL_E_BADHANDLE, PHTL_E_INVALID,
 * PHTL_E_NODEVICE, PHTL_E_CUDA (launch failure).                                   */
int phtl_track(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
               int64_t n, int64_t turns, int integrator, int dtype, void* cuda_stream);

/* Stop the persistent tracking calls already enqueued on this handle (phtl_track,
 * phtl_track_programme and the kernels of phtl_track_host), from any host thread, at the
 * next boundary between their launches.  Each launch is preceded on the stream by a
 * one-thread gate kernel that reads the handle's cancel word (host-mapped memory) and lets
 * the launch run whole or skip it, so the particles are left exactly as after the last
 * launch that ran: bitwise the state of the same call with fewer turns, its later monitor
 * rows zero.  Calls enqueued after phtl_track_cancel returns run normally.  The first
 * device call of a handle allocates the cancel and gate words (8 pinned host words, one
 * device word); a handle's calls share them, so calls that can overlap on the GPU must not
 * be cancelled independently.  A call enqueued on a stream that is capturing a CUDA graph
 * gets no gates (a replay would reuse its epoch): phtl_track_cancel does not stop the
 * graph's replays, and phtl_track_status reports such a call as complete.
 * Errors: PHTL_E_BADHANDLE.                                                            */
int phtl_track_cancel(phtl_handle* h);

/* Outcome of the handle's last phtl_track / phtl_track_programme / phtl_track_host call,
 * to be read after that call's stream work has completed: PHTL_OK with *turns_done = its
 * turns, or PHTL_E_CANCELLED with *turns_done = the turns of the launches that ran before
 * phtl_track_cancel took effect (a multiple of the turns per launch).  Host only.
 * Errors: PHTL_E_BADHANDLE, PHTL_E_INVALID (turns_done NULL).                          */
int phtl_track_status(const phtl_handle* h, int64_t* turns_done);

/* Same arguments and results as phtl_track, but one kernel launch per turn, so the
 * state makes a round trip through HBM every turn (Sec. 2.3's host-side turn loop):
 * the memory-bound reference point.                                               */
int phtl_track_perturn(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y,
                       void* yp, int64_t n, int64_t turns, int integrator, int dtype,
                       void* cuda_stream);

/* End-to-end call on HOST buffers (the paper's Fig. cuprof phases: allocate, copy in,
 * kernel, copy out, free).  Same layout rules as phtl_track, but every pointer is host
 * memory; mon_rows (or NULL) is a host array of turns/mon_stride + 1 rows.  The call
 * is synchronous: on return the host buffers hold the result.  Device memory is
 * allocated and freed inside.  Errors: as phtl_track, plus PHTL_E_NOMEM.            */
int phtl_track_host(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
                    int64_t n, int64_t turns, int integrator, int dtype, double* mon_rows,
                    int64_t mon_stride);

/* Phase times of the last phtl_track_host call on a handle: the phases of the paper's CUDA
 * profile (Sec. 2.4.2, Fig. cuprof: allocate, copy in, kernel, copy out, free), each
 * measured with CUDA events recorded on the call's stream between the phases (device
 * time, ms), plus the call's host wall time from entry to return.  Zeros before the first
 * call.  Host only.  Errors: PHTL_E_BADHANDLE, PHTL_E_INVALID (out NULL).               */
typedef struct phtl_phase_times {
    double alloc_ms;   /* stream-ordered device allocations                            */
    double h2d_ms;     /* host -> device copies of the coordinates                      */
    double kernel_ms;  /* monitor clear and the tracking launches                       */
    double d2h_ms;     /* device -> host copies of the coordinates and monitor rows     */
    double free_ms;    /* stream-ordered frees                                          */
    double total_ms;   /* first event to last                                           */
    double wall_ms;    /* host wall time of the call                                    */
    int64_t h2d_bytes, d2h_bytes;
    int64_t launches;  /* tracking kernels of the call                                  */
} phtl_phase_times;

int phtl_get_phase_times(const phtl_handle* h, phtl_phase_times* out);

/* ---- ramp programme (accelerating bucket) ---------------------------------------------- */

/* Attach a machine programme to the handle: the RF voltage voltage_V[n] of every turn
 * n = 0 .. nturns-1 and the reference momentum p0_eVc[n] at the start of turn n
 * (nturns + 1 values; p0_eVc[nturns] is the momentum after the last turn).  Host arrays,
 * read during the call.  The paper's runs change the machine parameters (hollow-bunch
 * studies); it prints no formulas, so the per-turn reading is:
 *   - turn n uses beta_n, gamma_n, eta_n from p0_eVc[n] and A_n = q V_n / (beta_n p0_n);
 *   - a particle gains q V_n sin(phi) / beta_n of momentum per turn (dE = beta c dp) and
 *     the synchronous one p0[n+1] - p0[n], so sin(phi_s,n) = beta_n (p0[n+1] - p0[n]) /
 *     (q V_n), phi_s,n on the stable branch (asin above transition, pi - asin below);
 *   - the turn runs the scheme's stages with eta_n C, A_n and phi_s,n (the synchronous
 *     particle stays at (0, 0)), then the transverse rotation, then delta, x' and y' are
 *     re-expressed against the next reference momentum: multiplied by
 *     r_n = p0[n] / p0[n+1] (for a single kick exactly the momentum bookkeeping
 *     p0[n] (1 + delta + A (sin phi - sin phi_s)) = p0[n+1] (1 + delta')).
 * The ring's harmonic, gamma_t, transverse optics and rf_linear flag apply to every turn;
 * the ring's own voltage_V, phi_s_rad and p0_eVc do not.  The constants of all turns are
 * derived in FP64 on the host (the long-horizon reference bookkeeping) and kept in a
 * library-owned device table of 192 bytes per turn (replacing any previous programme; freed
 * by phtl_destroy or a call with nturns == 0).  Synchronous.
 * Errors: PHTL_E_BADHANDLE; PHTL_E_INVALID (null arrays with nturns > 0, non-positive or
 * non-finite momenta, V = 0 on a turn whose momentum changes, a ring with eta1, eta2,
 * a chromaticity or a second RF system -- the programme runs the linear map only);
 * PHTL_E_UNSTABLE (|sin phi_s,n| >= 1, or a turn's linear strength outside (0, 4));
 * PHTL_E_NODEVICE; PHTL_E_NOMEM.                                                          */
int phtl_set_programme(phtl_handle* h, const double* voltage_V, const double* p0_eVc,
                       int64_t nturns);

/* Track turns [turn0, turn0 + turns) of the attached programme with the persistent
 * kernel (turn loop inside the kernel; each turn's constants read from the device table).
 * Buffers, layout, dtypes, monitor and tuning as phtl_track; integrator PHTL_EULER_CROMER
 * | PHTL_LEAPFROG | PHTL_RUTH4.  Stream-ordered.  Splitting a range into consecutive calls
 * gives bitwise the same particles.  Errors: as phtl_track, plus PHTL_E_INVALID (no
 * programme, a programme set on another device, turn0 + turns beyond it, PHTL_RK4).     */
int phtl_track_programme(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
                         int64_t n, int64_t turn0, int64_t turns, int integrator, int dtype,
                         void* cuda_stream);

/* ---- collective step: slicing and a wake kick ------------------------------------------- */

#define PHTL_MAX_SLICES 4096

/* A wake and longitudinal space charge acting through the bunch's own line density.  The
 * paper's conclusion names collective effects as the next workload after single-particle
 * tracking and prints no formulas; the reading:
 *   - slicing: nslices uniform slices on [z_lo, z_hi); particle i lies in slice
 *     k = floor((z_i - z_lo) * inv_dz), inv_dz = nslices / (z_hi - z_lo) (both FP64,
 *     subtract then multiply), when 0 <= k < nslices; c_k counts slice k's particles;
 *   - wake potential: V_k = sum over j >= k of c_j w[j - k] (z > 0 is ahead: a slice feels
 *     the slices ahead of it and itself; w[m] is the wake of one macro-particle m slices
 *     ahead, in units chosen with alpha);
 *   - space charge: D_k = (c_{k+1} - c_{k-1}) / 2, one-sided (c_1 - c_0, c_{N-1} - c_{N-2})
 *     at the ends, 0 for a single slice: the slope of the line density in counts per slice,
 *     to which the longitudinal space-charge field is proportional;
 *   - kick: delta_i += alpha V_k(i) + alpha_sc D_k(i) for the particles inside the grid
 *     (others unchanged). */
typedef struct phtl_wake {
    double z_lo, z_hi;  /* slicing range [z_lo, z_hi), z_hi > z_lo                     */
    double alpha;       /* kick per unit wake potential                              */
    double alpha_sc;    /* kick per unit density slope (space charge; 0 = none)       */
    const double* w;    /* host array of nslices wake samples w[0 .. nslices-1]       */
    int32_t nslices;    /* 1 .. PHTL_MAX_SLICES                                       */
    int32_t pad_;
} phtl_wake;

/* Attach a wake to the handle (NULL detaches).  The table is copied into library-owned
 * device memory together with the slice counts (two buffers), the wake potential and the
 * per-slice kick (in FP64 and as a float pair): 40 bytes per slice, freed by phtl_destroy
 * or a detaching call.  The
 * collective calls below also keep each particle's slice between two launches in
 * library-owned memory (2 bytes per particle, allocated by the first call with more
 * particles than before, which synchronises the device; freed with the wake).  These
 * buffers belong to the handle: collective calls on one handle must be ordered (one
 * stream, or streams synchronised between the calls); use one handle per concurrent bunch.
 * Synchronous.
 * Errors: PHTL_E_BADHANDLE; PHTL_E_INVALID (nslices out of range, z_hi <= z_lo,
 * non-finite values, w NULL); PHTL_E_NODEVICE; PHTL_E_NOMEM.                           */
int phtl_set_wake(phtl_handle* h, const phtl_wake* wake);

/* One collective step on (z, dp) without the map: slice the bunch, form the wake
 * potential and the density slope, kick.  Buffers and layout as phtl_track (every dtype;
 * the potential and the kick are formed in FP64, the FP32 types add the kick as a float
 * pair; PHTL_F32C decides the slice in FP64 from hi + comp, PHTL_F32CD / PHTL_F32CS in
 * double-float).  counts_out (nslices uint32) and V_out (nslices doubles): device
 * pointers or NULL, receive the step's counts and wake potential.  Stream-ordered.
 * Errors: as phtl_track, plus PHTL_E_INVALID (no wake attached, or attached on another
 * device).                                                                              */
int phtl_collective_kick(phtl_handle* h, void* z, void* dp, int64_t n, int dtype,
                         uint32_t* counts_out, double* V_out, void* cuda_stream);

/* Track `turns` turns, each the scheme's one-turn map and the transverse rotation (as
 * phtl_track, widened map included) followed by the collective step on the whole bunch.
 * Every dtype (as phtl_collective_kick) and every integrator (RK4 included); the monitor
 * (phtl_set_monitor) records after each full turn, collective kick included.  Each turn
 * is two kernel launches (turn + slicing, potential), the state making one HBM round
 * trip per turn.
 * Stream-ordered.  Errors: as phtl_collective_kick.                                     */
int phtl_track_collective(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
                          int64_t n, int64_t turns, int integrator, int dtype, void* cuda_stream);

/* ---- batched launch (many independent bunches in one graph-captured launch) ------------ */

/* One bunch of a batch.  Particles are independent and turns sequential (Sec. 2.3), so
 * bunches of different sizes, turn counts, RF voltages, integrators and arithmetic can
 * share launches.  The ring (C, h, p0, gamma_t, phi_s, transverse optics) is the handle's;
 * voltage_V is this bunch's own RF voltage.                                            */
typedef struct phtl_job {
    void* c[6];           /* z, dp, x, xp, y, yp: device pointers, layout as phtl_track;
                             x/xp and y/yp pairs may be NULL                              */
    double* mon_rows;     /* device monitor rows of this bunch, or NULL                   */
    int64_t mon_capacity; /* rows at mon_rows (>= turns / mon_stride + 1)                  */
    int64_t mon_stride;   /* >= 1 when mon_rows is set                                     */
    int64_t n;            /* macro-particles                                               */
    int64_t turns;        /* turns tracked by each run of the batch                        */
    double voltage_V;     /* RF voltage of this bunch                                      */
    int32_t integrator;   /* PHTL_EULER_CROMER | PHTL_LEAPFROG | PHTL_RUTH4 | PHTL_RK4      */
    int32_t dtype;        /* PHTL_F64 | PHTL_F32C | PHTL_F32CD | PHTL_F32CS                 */
} phtl_job;

typedef struct phtl_batch phtl_batch; /* opaque, library-owned */

/* Launch shape chosen by the autotuner (or set with phtl_set_tuning). */
typedef struct phtl_tuning {
    int32_t block_threads;
    int32_t pad_;
    int64_t turns_per_launch;
    double particle_turns_per_s; /* the probe's measured throughput                        */
} phtl_tuning;

typedef struct phtl_batch_info {
    int32_t njobs;
    int32_t graph;                       /* 1: runs replay a captured CUDA graph          */
    int32_t block_threads[4];            /* per arithmetic (PHTL_F64 .. PHTL_F32CS); 0 = none */
    int64_t turns_per_launch[4];
    double probe_particle_turns_per_s[4];
    int64_t launches_per_run;            /* kernel launches in one run (known after a run) */
    int64_t tiles_first_launch;          /* blocks of the first chunk launch, all groups   */
    int64_t particle_turns_per_run;      /* sum of n * turns                              */
} phtl_batch_info;

/* Project-written autotuner: times the batched kernel of `dtype`/`integrator` at block
 * sizes 64, 96, 128, 192 and 256 on scratch particles that fill the GPU once (the library
 * allocates and frees them; the call synchronises), keeps the fastest block, and picks
 * the turns per launch that make a launch over `active_particles` particles last about
 * target_launch_ms.  Errors: PHTL_E_BADHANDLE, PHTL_E_INVALID, PHTL_E_NODEVICE,
 * PHTL_E_CUDA.                                                                          */
int phtl_autotune(phtl_handle* h, int dtype, int integrator, int64_t active_particles,
                  double target_launch_ms, phtl_tuning* out);

/* Build a batch: validates every job (as phtl_track, plus a stability check of each
 * bunch's voltage -> PHTL_E_UNSTABLE), groups the jobs by arithmetic, sorts each group by
 * turns (longest first), uploads a device job table, and fixes the launch shape (the
 * handle's tuning if both block and turns per launch are set, else phtl_autotune with a
 * 20 ms target).  use_graph != 0: the first run captures its launches into a CUDA graph
 * that later runs replay.  The caller's buffers must stay valid until
 * phtl_batch_destroy.  Synchronous set-up.                                             */
int phtl_batch_create(phtl_handle* h, const phtl_job* jobs, int32_t njobs, int32_t use_graph,
                      phtl_batch** out);

/* Enqueue one run on cuda_stream: every job advances by its `turns`, its monitor (if
 * any) rewritten from row 0.  A job's particles come out bitwise as phtl_track would give
 * them.  Stream-ordered.  Errors: PHTL_E_BADHANDLE, PHTL_E_CUDA.                         */
int phtl_batch_run(phtl_batch* b, void* cuda_stream);

int phtl_batch_info_get(const phtl_batch* b, phtl_batch_info* out);

/* Synchronise the device, free the job tables and graph.  Errors: PHTL_E_BADHANDLE.     */
int phtl_batch_destroy(phtl_batch* b);

/* Capacity of the fixed job table used by phtl_batch_run_noalloc. */
#define PHTL_NOALLOC_MAX_JOBS 256

/* One run of a batch that allocates nothing.  No counterpart in the paper: this entry
 * point exists for callers that cannot let the library allocate device memory -- an
 * application whose device memory is owned and budgeted by its own allocator or pool,
 * or a loop that must never pay for cudaMalloc / cudaFree, which can block the host and
 * synchronise the device.  It tracks the same jobs with the same kernels and gives the
 * same particles as phtl_batch_create + phtl_batch_run (monitor sums equal to FP64
 * rounding), but it calls no cudaMalloc, cudaFree or other allocating routine: the job
 * table is written into a fixed device array of PHTL_NOALLOC_MAX_JOBS entries that lives
 * in the library for as long as the process runs, on every GPU that loads it.  The
 * launch shape is the handle's tuning (phtl_set_tuning), else 128 threads per block and
 * the library's default turns per launch; no autotuner probe and no CUDA graph.
 * jobs: as for phtl_batch_create (caller-owned device buffers, updated in place).
 * The call is stream-ordered on cuda_stream.  The first call on a device looks up the
 * array's device address (one-time set-up).  The table is copied from host memory that
 * lives only during the call, so the call cannot be recorded into a CUDA graph: on a
 * stream that is capturing it returns PHTL_E_CAPTURE and enqueues nothing.  Every call
 * shares the array and it keeps the last call's contents; each call rewrites all entries
 * it uses.  Calls that can overlap on the GPU (for example on two streams with no
 * ordering between them) race on the array: order them on one stream.  Every check runs
 * before the first enqueue, so a rejected call leaves the jobs untouched; only a CUDA
 * error during the enqueue (PHTL_E_CUDA) can leave some arithmetic groups advanced.
 * Errors: PHTL_E_TOOBIG (njobs > PHTL_NOALLOC_MAX_JOBS), PHTL_E_CAPTURE,
 * PHTL_E_BADHANDLE, PHTL_E_INVALID, PHTL_E_UNSTABLE, PHTL_E_NODEVICE, PHTL_E_CUDA.      */
int phtl_batch_run_noalloc(phtl_handle* h, const phtl_job* jobs, int32_t njobs,
                           void* cuda_stream);

/* ---- serving loop (continuous batching) ------------------------------------------------- */

/* Job states reported by phtl_poll / phtl_wait. */
enum { PHTL_QUEUED = 0, PHTL_RUNNING = 1, PHTL_DONE = 2, PHTL_FAILED = 3, PHTL_CANCELLED = 4 };

typedef struct phtl_server_config {
    int64_t memory_budget_bytes; /* device bytes admitted jobs may hold (state + monitor),
                                    resident states included; 0 = 150e9                  */
    int32_t max_active;          /* jobs tracked concurrently (slots); 0 = 64              */
    int32_t block_threads;       /* 0 = autotuned per arithmetic                          */
    int64_t chunk_turns_f64;     /* turns per scheduling round for FP64 jobs; 0 = chosen
                                    every round for a ~target_round_ms round               */
    int64_t chunk_turns_f32;     /* the same for the FP32-compensated jobs                 */
    double target_round_ms;      /* 0 = 20 ms                                              */
    int32_t policy;              /* PHTL_POLICY_SRPT (0, default) or PHTL_POLICY_SHARE     */
    int32_t waves;               /* SRPT: particles of one arithmetic a round carries, in
                                    resident waves of its batched kernel; 0 = 8            */
} phtl_server_config;

/* Which admitted jobs a scheduling round advances.
 *  PHTL_POLICY_SRPT : per arithmetic, the jobs with the least remaining work
 *                     (n x turns left) first, up to `waves` resident waves of particles,
 *                     plus always the longest-admitted one (no starvation): short jobs
 *                     finish early, lowering the median latency.
 *  PHTL_POLICY_SHARE: every admitted job advances every round (processor sharing).    */
enum { PHTL_POLICY_SRPT = 0, PHTL_POLICY_SHARE = 1 };

/* One tracking request: host buffers in, host buffers out. */
typedef struct phtl_request {
    const void* in[6];      /* host inputs z, dp, x, xp, y, yp (layout as phtl_track;
                               x/xp and y/yp pairs may be NULL).  Ignored on resume.       */
    void* out[6];           /* host outputs, same planes as in[] (may alias in[]), written
                               before the job turns PHTL_DONE                              */
    double* mon_rows;       /* host rows for turns/mon_stride + 1 monitor rows, or NULL    */
    int64_t mon_stride;
    int64_t n;              /* macro-particles                                            */
    int64_t turns;
    double voltage_V;       /* this job's RF voltage (the ring is the handle's)           */
    int32_t integrator;
    int32_t dtype;
    uint64_t resume_ticket; /* nonzero: continue from that PHTL_DONE job's resident device
                               state (same n, dtype and planes; given by out[])            */
    int32_t keep_resident;  /* nonzero: keep the device state after DONE for a resume;
                               it counts against the budget until phtl_release           */
    int32_t pad_;
} phtl_request;

typedef struct phtl_status {
    int32_t state;          /* PHTL_QUEUED .. PHTL_CANCELLED                              */
    int32_t error;          /* PHTL_OK, or the error of a FAILED / CANCELLED job           */
    int64_t turns_done;
    int64_t t_submit_ns, t_admit_ns, t_done_ns; /* steady clock                          */
} phtl_status;

typedef struct phtl_server_stats {
    int64_t submitted, completed, failed, cancelled, queued, active;
    int64_t bytes_in_use, bytes_peak;
    int64_t rounds, launches;
    double particle_turns;  /* completed work                                            */
    double busy_s;          /* time spent in scheduling rounds                            */
    double p50_latency_s, p99_latency_s, mean_latency_s; /* submit -> done, DONE jobs     */
    double throughput_pts;  /* particle_turns / (last done - first submit)               */
} phtl_server_stats;

/* Start the serving loop of a handle: a worker thread that admits queued requests in
 * arrival order while a slot is free and their device bytes fit the budget, tracks all
 * admitted jobs together in scheduling rounds of batched launches (every job advances by
 * up to one chunk of turns per round), and retires finished jobs between rounds (results
 * copied to the request's host buffers, device memory freed unless kept resident).  A
 * job's particles are bitwise the same as phtl_track would give; its monitor sums agree
 * to FP64 rounding.  cfg NULL = defaults.  Synchronous set-up (runs the autotuner).
 * Errors: PHTL_E_BADHANDLE, PHTL_E_INVALID (bad config or already started),
 * PHTL_E_NODEVICE, PHTL_E_CUDA, PHTL_E_NOMEM.                                        */
int phtl_server_start(phtl_handle* h, const phtl_server_config* cfg);

/* Queue a request; *ticket identifies it.  Host buffers must stay valid until the job is
 * final.  Errors: PHTL_E_BADHANDLE (no server / unknown resume ticket), PHTL_E_INVALID,
 * PHTL_E_UNSTABLE (voltage), PHTL_E_NOMEM (larger than the whole budget).            */
int phtl_submit(phtl_handle* h, const phtl_request* req, uint64_t* ticket);

/* Current status of a ticket.  Errors: PHTL_E_BADHANDLE.                               */
int phtl_poll(phtl_handle* h, uint64_t ticket, phtl_status* out);

/* Wait until the ticket is final or timeout_ms passes (0 = do not wait): PHTL_OK, or
 * PHTL_E_TIMEOUT with *out the current status.                                         */
int phtl_wait(phtl_handle* h, uint64_t ticket, int64_t timeout_ms, phtl_status* out);

/* Cancel a queued or running job; it leaves at the next round boundary with state
 * PHTL_CANCELLED and turns_done at that boundary.  Errors: PHTL_E_BADHANDLE,
 * PHTL_E_INVALID (already final).                                                      */
int phtl_cancel(phtl_handle* h, uint64_t ticket);

/* Free the resident device state of a PHTL_DONE job kept with keep_resident.           */
int phtl_release(phtl_handle* h, uint64_t ticket);

int phtl_server_get_stats(phtl_handle* h, phtl_server_stats* out);

/* Stop the loop: the running round completes, jobs not yet DONE end CANCELLED, resident
 * states are freed.  phtl_destroy does this too.                                       */
int phtl_server_stop(phtl_handle* h);

/* ---- host helpers -------------------------------------------------------------------- */

/* Cumulative counters of a handle since phtl_create (host only). */
typedef struct phtl_stats {
    int64_t launches;       /* tracking kernels enqueued by this handle          */
    int64_t particle_turns; /* sum over tracking calls of n * turns              */
    int64_t calls;          /* tracking calls that enqueued work                 */
    int64_t gate_launches;  /* one-thread cancellation gates in front of the     */
                            /* persistent launches (phtl_track_cancel)           */
} phtl_stats;

int phtl_get_stats(const phtl_handle* h, phtl_stats* out);

/* Moments of one monitor row: out[15] = mean z, mean d, rms z, rms d, eps_z,
 * mean x, mean x', rms x, rms x', eps_x, mean y, mean y', rms y, rms y', eps_y
 * (population rms; eps = sqrt(<u^2><u'^2> - <u u'>^2) of centred coordinates).
 * A row with n == 0 gives zeros.  Host only.                                      */
int phtl_moments_from_sums(const double* row, double* out15);

/* Diagnostic: y[i] = sine of x[i] on the device, for n device doubles, stream-ordered.
 * which = 0: the library's own FP64 sine used by the FP64 kick (Cody-Waite reduction
 * plus a fitted polynomial); which = 1: CUDA's sin(), for comparison; which = 2: the
 * double-float sine of the PHTL_F32C / PHTL_F32CD kicks, applied to x[i] truncated to
 * a float pair (48 bits) and returned as hi + lo.
 * Errors: PHTL_E_INVALID, PHTL_E_NODEVICE, PHTL_E_CUDA.                           */
int phtl_eval_sin(const double* x, double* y, int64_t n, int which, void* cuda_stream);

/* Diagnostic: y[i] = sin(k * z[i]) for n device doubles, stream-ordered, through the
 * form the FP64 kick takes for phi_s = 0 (Sec. 1.1.2's kick with a stationary bucket):
 * the product k z is folded into the sine's argument reduction, so it is never rounded
 * on its own.  |k z| beyond ~1e5, Inf and NaN use which = 0 of phtl_eval_sin on the
 * rounded product.  Errors: PHTL_E_INVALID (n < 0, null pointer with n > 0, k not
 * finite), PHTL_E_NODEVICE, PHTL_E_CUDA.                                           */
int phtl_eval_sin_kz(double k, const double* z, double* y, int64_t n, void* cuda_stream);

/* Library version string, e.g. "phtl 0.1 sm_103a".                                 */
const char* phtl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PHTL_H */
