/*
 * phtl.h -- C ABI of libphtl.so: GB300-native (sm_103a) turn-by-turn macro-particle
 * tracking, after A. Oeftiger, "Parallelisation of PyHEADTAIL" (2014).
 *
 * What the library computes (the paper names the schemes but prints no formulas; the
 * readings below are the textbook single-harmonic synchrotron map):
 *   Sec. 1.1.2  longitudinal phase space (z, delta), integrated turn by turn for each
 *               macro-particle independently, by Euler-Cromer (1st order), leap-frog
 *               (2nd-order Verlet, drift-kick-drift) or a 4th-order Ruth scheme:
 *                 kick  K(w): phi = phi_s + k z;  delta += w A (sin phi - sin phi_s)
 *                 drift D(w): z -= w eta C delta
 *                 EC = K(1) D(1);  LF = D(1/2) K(1) D(1/2);
 *                 RUTH4 = D(t/2) K(t) D((1-t)/2) K(1-2t) D((1-t)/2) K(t) D(t/2),
 *                         t = 1/(2 - 2^(1/3))  (Forest & Ruth 1990)
 *               with k = 2 pi h / C, A = q V / (beta p0) [p0 in eV/c],
 *               eta = 1/gamma_t^2 - 1/gamma^2.
 *   Sec. 1.1.1  transverse (x, x', y, y'): the same linear transfer matrix every turn,
 *               [u; u'] <- [[cos mu, b sin mu], [-sin mu / b, cos mu]] [u; u'],
 *               mu = 2 pi frac(Q), alpha = 0, no chromaticity.
 *   Sec. 2.3    particles are independent, turns are sequential; the turn loop runs
 *               inside the kernel (state in registers), bounded per launch.
 * Per-turn bunch moments are accumulated into a caller-owned monitor buffer.
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

/* ---- enums ------------------------------------------------------------------------- */
enum { PHTL_EULER_CROMER = 0, PHTL_LEAPFROG = 1, PHTL_RUTH4 = 2 };

/* Arithmetic of the particle state.
 *  PHTL_F64   : every coordinate buffer holds n doubles.
 *  PHTL_F32C  : FP32 with compensated (Kahan/TwoSum) accumulation.  Every coordinate
 *               buffer holds 2n floats: [hi(0..n-1) | comp(0..n-1)]; the value of
 *               particle i is hi[i] + comp[i].  The RF phase argument k z is formed in
 *               FP64 from hi + comp, then rounded to FP32 for the SFU sine.
 *  PHTL_F32CD : as PHTL_F32C, but the phase argument is formed in double-float
 *               (FP32 pair) arithmetic instead of FP64.                               */
enum { PHTL_F64 = 0, PHTL_F32C = 1, PHTL_F32CD = 2 };

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
} phtl_params;

/* Constants derived in FP64 on the host by phtl_create. */
typedef struct phtl_derived {
    double betagamma, gamma, beta;
    double eta;        /* slip factor                                              */
    double k;          /* 2 pi h / C [1/m]                                         */
    double A;          /* kick amplitude q V / (beta p0)                           */
    double etaC;       /* eta * C [m]                                              */
    double sin_phis, cos_phis;
    double K;          /* linear strength eta C A k cos(phi_s)                     */
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
 * Errors: PHTL_E_INVALID (null, non-positive C/p0/mass/gamma_t/h/beta),
 *         PHTL_E_UNSTABLE (V != 0 and not 0 < K < 4).                               */
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
 * PHTL_F32C / PHTL_F32CD -> 2n floats per coordinate ([hi | comp]).  Pointers must be
 * aligned to the element size; 16-byte alignment enables 128-bit loads.
 * integrator: PHTL_EULER_CROMER | PHTL_LEAPFROG | PHTL_RUTH4.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Updates the buffers in place.  Errors: PHTL_E_BADHANDLE, PHTL_E_INVALID,
 * PHTL_E_NODEVICE, PHTL_E_CUDA (launch failure).                                   */
int phtl_track(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
               int64_t n, int64_t turns, int integrator, int dtype, void* cuda_stream);

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

/* ---- host helpers -------------------------------------------------------------------- */

/* Cumulative counters of a handle since phtl_create (host only). */
typedef struct phtl_stats {
    int64_t launches;       /* tracking kernels enqueued by this handle          */
    int64_t particle_turns; /* sum over tracking calls of n * turns              */
    int64_t calls;          /* tracking calls that enqueued work                 */
} phtl_stats;

int phtl_get_stats(const phtl_handle* h, phtl_stats* out);

/* Moments of one monitor row: out[15] = mean z, mean d, rms z, rms d, eps_z,
 * mean x, mean x', rms x, rms x', eps_x, mean y, mean y', rms y, rms y', eps_y
 * (population rms; eps = sqrt(<u^2><u'^2> - <u u'>^2) of centred coordinates).
 * A row with n == 0 gives zeros.  Host only.                                      */
int phtl_moments_from_sums(const double* row, double* out15);

/* Diagnostic: y[i] = sine of x[i] on the device, for n device doubles, stream-ordered.
 * which = 0: the library's own FP64 sine used by the FP64 kick (Cody-Waite reduction
 * plus a fitted polynomial); which = 1: CUDA's sin(), for comparison.
 * Errors: PHTL_E_INVALID, PHTL_E_NODEVICE, PHTL_E_CUDA.                           */
int phtl_eval_sin(const double* x, double* y, int64_t n, int which, void* cuda_stream);

/* Library version string, e.g. "phtl 0.1 sm_103a".                                 */
const char* phtl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PHTL_H */
