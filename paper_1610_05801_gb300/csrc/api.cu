// Host side of the C ABI declared in include/phtl.h: argument checking, FP64
// derivation of the map constants, launch planning and the host-buffer path.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_set>

#include "internal.h"
#include "handle.h"

namespace phtl {

namespace {

// One thread: the launch runs (go = 1) unless phtl_track_cancel raised the cancel epoch to
// this call's epoch or beyond; the turns of the launches that run are counted.  The epoch
// is read with a system-scope load, so a host store is seen by the next gate.
__global__ void k_track_gate(const long long* cancel_epoch, long long epoch, int* go,
                             long long* done, int nturns, int first)
{
    long long ce;
    asm volatile("ld.relaxed.sys.global.s64 %0, [%1];" : "=l"(ce) : "l"(cancel_epoch) : "memory");
    const int g = ce < epoch ? 1 : 0;
    *go = g;
    const long long d0 = first ? 0 : *done;
    *done = d0 + (g ? nturns : 0);
}

}  // namespace

bool stream_capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return cap != cudaStreamCaptureStatusNone;
}

cudaError_t launch_gate(const long long* cancel_epoch, long long epoch, int* go, long long* done,
                        int nturns, bool first, cudaStream_t s)
{
    k_track_gate<<<1, 1, 0, s>>>(cancel_epoch, epoch, go, done, nturns, first ? 1 : 0);
    return cudaGetLastError();
}

namespace {

std::mutex g_registry_mu;
std::unordered_set<const phtl_handle*> g_registry;


// Three-shear form of the rotation by mu = 2 pi frac(Q) with beta function b:
// [[c, b s], [-s/b, c]] = [[1, p], [0, 1]] [[1, 0], [q, 1]] [[1, p], [0, 1]],
// p = b tan(mu/2), q = -s/b.  Near mu = pi, tan(mu/2) blows up: keep the matrix.
void shear_params(double Q, double b, double (&sh)[2], int32_t& use)
{
    const double mu = 2.0 * kPi * (Q - std::floor(Q));
    const double t = std::tan(0.5 * mu);
    use = std::isfinite(t) && std::fabs(t) < 1e3 ? 1 : 0;
    sh[0] = use ? b * t : 0.0;
    sh[1] = use ? -std::sin(mu) / b : 0.0;
}

void scheme_consts(const phtl_derived& d, int scheme, MapConsts& c)
{
    scheme_weights(scheme, d.A, d.etaC, c.dc, c.kw);
    for (int i = 0; i < 4; ++i) split_df(c.dc[i], c.dc_hi[i], c.dc_lo[i]);
    for (int j = 0; j < 3; ++j) split_df(c.kw[j], c.kw_hi[j], c.kw_lo[j]);
}

int derive(const phtl_params& p, phtl_derived& d, MapConsts (&mc)[4])
{
    if (!finite_pos(p.circumference_m) || !finite_pos(p.gamma_t) || !finite_pos(p.p0_eVc) ||
        !finite_pos(p.mass_eV) || !finite_pos(p.beta_x_m) || !finite_pos(p.beta_y_m) ||
        p.harmonic <= 0 || !std::isfinite(p.charge_e) || !std::isfinite(p.voltage_V) ||
        !std::isfinite(p.phi_s_rad) || !std::isfinite(p.Qx) || !std::isfinite(p.Qy) ||
        !std::isfinite(p.eta1) || !std::isfinite(p.eta2) || !std::isfinite(p.xi_x) ||
        !std::isfinite(p.xi_y) || !std::isfinite(p.voltage2_V) || !std::isfinite(p.phi2_rad))
        return PHTL_E_INVALID;
    const bool dual = p.voltage2_V != 0.0;
    if (dual && p.harmonic2 <= 0) return PHTL_E_INVALID;
    std::memset(&d, 0, sizeof(d));
    d.betagamma = p.p0_eVc / p.mass_eV;
    d.gamma = std::sqrt(1.0 + d.betagamma * d.betagamma);
    d.beta = d.betagamma / d.gamma;
    d.eta = 1.0 / (p.gamma_t * p.gamma_t) - 1.0 / (d.gamma * d.gamma);
    d.k = 2.0 * kPi * static_cast<double>(p.harmonic) / p.circumference_m;
    d.A = kick_amplitude(p, d, p.voltage_V);
    d.etaC = d.eta * p.circumference_m;
    d.sin_phis = std::sin(p.phi_s_rad);
    d.cos_phis = std::cos(p.phi_s_rad);
    // second RF system (double RF): k2 = 2 pi h2 / C, A2 = q V2 / (beta p0)
    const double k2 = dual ? 2.0 * kPi * static_cast<double>(p.harmonic2) / p.circumference_m : 0.0;
    const double A2 = dual ? kick_amplitude(p, d, p.voltage2_V) : 0.0;
    const double cos_phi2 = dual ? std::cos(p.phi2_rad) : 0.0;
    d.K = d.etaC * (d.A * d.k * d.cos_phis + A2 * k2 * cos_phi2);
    d.Qs = d.K > 0.0 ? std::sqrt(d.K) / (2.0 * kPi) : 0.0;
    d.bucket_half_length_m = kPi / d.k;
    const double r = d.A / (d.k * d.etaC);
    d.bucket_half_height = r > 0.0 ? 2.0 * std::sqrt(r) : 0.0;
    const double mux = 2.0 * kPi * (p.Qx - std::floor(p.Qx));
    const double muy = 2.0 * kPi * (p.Qy - std::floor(p.Qy));
    d.mx[0] = std::cos(mux);
    d.mx[1] = p.beta_x_m * std::sin(mux);
    d.mx[2] = -std::sin(mux) / p.beta_x_m;
    d.mx[3] = std::cos(mux);
    d.my[0] = std::cos(muy);
    d.my[1] = p.beta_y_m * std::sin(muy);
    d.my[2] = -std::sin(muy) / p.beta_y_m;
    d.my[3] = std::cos(muy);
    // the linearised motion must oscillate (0 < K < 4); with a second RF system the
    // flat-bottomed bucket K = 0 is allowed too
    if (!dual && p.voltage_V != 0.0 && !(d.K > 0.0 && d.K < 4.0)) return PHTL_E_UNSTABLE;
    if (dual && !(d.K >= 0.0 && d.K < 4.0)) return PHTL_E_UNSTABLE;

    for (int s = 0; s < 4; ++s) {
        MapConsts& c = mc[s];
        std::memset(&c, 0, sizeof(c));
        scheme_consts(d, s, c);
        c.k = d.k;
        c.k2opi = static_cast<float>(d.k * (2.0 / kPi));
        c.phis = p.phi_s_rad;
        c.sinphis = d.sin_phis;
        c.lin = d.cos_phis * d.k;
        c.linear = p.rf_linear != 0;
        c.phis_zero = p.phi_s_rad == 0.0 ? 1 : 0;
        for (int i = 0; i < 4; ++i) {
            c.mx[i] = d.mx[i];
            c.my[i] = d.my[i];
            split_df(d.mx[i], c.mx_hi[i], c.mx_lo[i]);
            split_df(d.my[i], c.my_hi[i], c.my_lo[i]);
        }
        shear_params(p.Qx, p.beta_x_m, c.shx, c.shear_x);
        shear_params(p.Qy, p.beta_y_m, c.shy, c.shear_y);
        split_df(d.k, c.k_hi, c.k_lo);
        split_df(p.phi_s_rad, c.phis_hi, c.phis_lo);
        split_df(d.sin_phis, c.sinphis_hi, c.sinphis_lo);
        split_df(c.lin, c.lin_hi, c.lin_lo);
        // widened map (eta(delta), chromaticity)
        c.eta1C = p.eta1 * p.circumference_m;
        c.eta2C = p.eta2 * p.circumference_m;
        c.qx = p.Qx - std::floor(p.Qx);
        c.qy = p.Qy - std::floor(p.Qy);
        c.xi_x = p.xi_x;
        c.xi_y = p.xi_y;
        c.bx = p.beta_x_m;
        c.by = p.beta_y_m;
        c.ibx = 1.0 / p.beta_x_m;
        c.iby = 1.0 / p.beta_y_m;
        c.chroma_x = p.xi_x != 0.0 ? 1 : 0;
        c.chroma_y = p.xi_y != 0.0 ? 1 : 0;
        // second RF system
        c.dual_rf = dual ? 1 : 0;
        if (dual) {
            double dc2[4];
            scheme_weights(s, A2, d.etaC, dc2, c.kw2);
            c.k2 = k2;
            c.phi2 = p.phi2_rad;
            c.sinphi2 = std::sin(p.phi2_rad);
            c.lin2 = cos_phi2 * k2;
        }
        for (int j = 0; j < 3; ++j) split_df(c.kw2[j], c.kw2_hi[j], c.kw2_lo[j]);
        split_df(c.k2, c.k2_hi, c.k2_lo);
        split_df(c.phi2, c.phi2_hi, c.phi2_lo);
        split_df(c.sinphi2, c.sinphi2_hi, c.sinphi2_lo);
        split_df(c.lin2, c.lin2_hi, c.lin2_lo);
        // the widened map's kernels: eta(delta), chromaticity, double RF, and RK4
        c.general = (p.eta1 != 0.0 || p.eta2 != 0.0 || c.chroma_x || c.chroma_y || dual ||
                     s == PHTL_RK4) ? 1 : 0;
        split_df(c.eta1C, c.eta1C_hi, c.eta1C_lo);
        split_df(c.eta2C, c.eta2C_hi, c.eta2C_lo);
        split_df(c.qx, c.qx_hi, c.qx_lo);
        split_df(c.qy, c.qy_hi, c.qy_lo);
        split_df(c.xi_x, c.xi_x_hi, c.xi_x_lo);
        split_df(c.xi_y, c.xi_y_hi, c.xi_y_lo);
        split_df(c.bx, c.bx_hi, c.bx_lo);
        split_df(c.by, c.by_hi, c.by_lo);
        split_df(c.ibx, c.ibx_hi, c.ibx_lo);
        split_df(c.iby, c.iby_hi, c.iby_lo);
    }
    return PHTL_OK;
}

}  // namespace

// Stage coefficients of each scheme (Sec. 1.1.2 readings, see phtl.h):
// dc[i] = w_i * eta C for the drifts, kw[j] = w_j * A for the kicks.
void scheme_weights(int scheme, double A, double etaC, double (&dc)[4], double (&kw)[3])
{
    for (int i = 0; i < 4; ++i) dc[i] = 0.0;
    for (int j = 0; j < 3; ++j) kw[j] = 0.0;
    if (scheme == PHTL_EULER_CROMER) {
        kw[0] = 1.0 * A;
        dc[0] = 1.0 * etaC;
    } else if (scheme == PHTL_LEAPFROG) {
        dc[0] = 0.5 * etaC;
        kw[0] = 1.0 * A;
        dc[1] = 0.5 * etaC;
    } else if (scheme == PHTL_RK4) {
        // classic RK4: the right-hand side uses eta C and A themselves
        dc[0] = etaC;
        kw[0] = A;
    } else {
        // Forest-Ruth: theta = 1 / (2 - 2^(1/3))
        const double th = 1.0 / (2.0 - std::cbrt(2.0));
        dc[0] = (0.5 * th) * etaC;
        kw[0] = th * A;
        dc[1] = (0.5 * (1.0 - th)) * etaC;
        kw[1] = (1.0 - 2.0 * th) * A;
        dc[2] = (0.5 * (1.0 - th)) * etaC;
        kw[2] = th * A;
        dc[3] = (0.5 * th) * etaC;
    }
}

double kick_amplitude(const phtl_params& p, const phtl_derived& d, double voltage_V)
{
    return p.charge_e * voltage_V / (d.beta * p.p0_eVc);
}

void job_weights(const phtl_handle* h, int scheme, double voltage_V, JobDesc& J)
{
    const phtl_derived& d = h->derived;
    scheme_weights(scheme, kick_amplitude(h->params, d, voltage_V), d.etaC, J.dc, J.kw);
    for (int j = 0; j < 3; ++j) J.kw2[j] = h->mc[scheme].kw2[j];
    fill_float_weights(J);
}

MapConsts batch_consts(const phtl_handle* h, bool has_rk4)
{
    MapConsts c = h->mc[0];
    if (has_rk4) c.general = 1;
    return c;
}

int voltage_check(const phtl_handle* h, double voltage_V)
{
    const phtl_derived& d = h->derived;
    const double K = d.etaC * kick_amplitude(h->params, d, voltage_V) * d.k * d.cos_phis + h->K2;
    if (h->mc[0].dual_rf) return K >= 0.0 && K < 4.0 ? PHTL_OK : PHTL_E_UNSTABLE;
    if (voltage_V != 0.0 && !(K > 0.0 && K < 4.0)) return PHTL_E_UNSTABLE;
    return PHTL_OK;
}

int handle_stream(phtl_handle* h, cudaStream_t* out)
{
    if (!h->stream) {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            h->stream = nullptr;
            return PHTL_E_CUDA;
        }
    }
    *out = h->stream;
    return PHTL_OK;
}

void release_handle_resources(phtl_handle* h)
{
    stop_server(h);
    free_programme(h);
    free_wake(h);
    if (h->stream) {
        cudaStreamSynchronize(h->stream);
        cudaStreamDestroy(h->stream);
        h->stream = nullptr;
    }
    for (cudaEvent_t& e : h->phase_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (h->ctl_host || h->gate_go) cudaDeviceSynchronize();  // no gate may still be reading them
    if (h->ctl_host) cudaFreeHost(h->ctl_host);
    if (h->gate_go) cudaFree(h->gate_go);
    h->ctl_host = nullptr;
    h->ctl_dev = nullptr;
    h->gate_go = nullptr;
    cudaGetLastError();
}

int log_level()
{
    static const int level = [] {
        const char* v = std::getenv("PHTL_LOG");
        return v ? std::atoi(v) : 0;
    }();
    return level;
}

void log_line(const char* fmt, ...)
{
    if (log_level() <= 0) return;
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
    std::fputs("phtl: ", stderr);
    va_list ap;
    va_start(ap, fmt);
    std::vfprintf(stderr, fmt, ap);
    va_end(ap);
    std::fputc('\n', stderr);
}

bool handle_valid(const phtl_handle* h)
{
    if (!h) return false;
    std::lock_guard<std::mutex> g(g_registry_mu);
    return g_registry.count(h) != 0 && h->magic == kHandleMagic;
}

int ensure_device(phtl_handle* h)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PHTL_E_NODEVICE;
    }
    if (h->dev_ready && h->device == dev) return PHTL_OK;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return PHTL_E_NODEVICE;
    }
    // the library is compiled for sm_103a only
    if (prop.major != 10 || prop.minor != 3) return PHTL_E_NODEVICE;
    // the cancellation words of persistent calls (host-mapped) and the launch gate (device)
    if (h->ctl_host) {
        cudaFreeHost(h->ctl_host);
        h->ctl_host = nullptr;
        h->ctl_dev = nullptr;
    }
    if (h->gate_go) {
        cudaFree(h->gate_go);
        h->gate_go = nullptr;
    }
    void* hp = nullptr;
    void* dp = nullptr;
    if (cudaHostAlloc(&hp, 4 * sizeof(long long), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&h->gate_go), sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (hp) cudaFreeHost(hp);
        if (h->gate_go) cudaFree(h->gate_go);
        h->gate_go = nullptr;
        return PHTL_E_NOMEM;
    }
    h->ctl_host = static_cast<long long*>(hp);
    h->ctl_dev = static_cast<long long*>(dp);
    std::memset(h->ctl_host, 0, 4 * sizeof(long long));
    h->device = dev;
    h->nsm = prop.multiProcessorCount;
    h->dev_ready = true;
    return PHTL_OK;
}

// Particle-turns per launch that keep one launch near ~50-100 ms (Sec. 2.3: bounded
// kernel duration; the turns-per-launch trade-off of Fig. turnspercall).
int64_t auto_turns_per_launch(int dtype, int scheme, int64_t n)
{
    const double budget = dtype == PHTL_F64 ? 8e8 : 8e9;
    const double w = scheme == PHTL_RUTH4 ? 3.0 : scheme == PHTL_RK4 ? 4.0 : 1.0;
    double t = budget / (w * static_cast<double>(std::max<int64_t>(n, 1)));
    t = std::min(t, 1048576.0);
    return std::max<int64_t>(1, static_cast<int64_t>(t));
}

// The per-turn variant is the persistent kernel family launched with one turn per
// launch over a grid that covers every particle once: the state makes a round trip
// through HBM each turn (Sec. 2.3's host-side turn loop).
cudaError_t launch_perturn(const LaunchDesc& L, const MapConsts& c, const MonitorArgs& m,
                           int dtype, cudaStream_t s)
{
    return dtype == PHTL_F64 ? launch_track_f64(L, c, m, s) : launch_track_f32c(L, c, m, dtype, s);
}

int occupancy_perturn(int scheme, bool trans, bool mon, int dtype, int block, int gen)
{
    return dtype == PHTL_F64 ? occupancy_f64(scheme, trans, mon, block, gen)
                             : occupancy_f32c(scheme, trans, mon, dtype, block, gen);
}

int occupancy(int dtype, int scheme, bool trans, bool mon, int block, bool perturn, int gen)
{
    if (perturn) return occupancy_perturn(scheme, trans, mon, dtype, block, gen);
    if (dtype == PHTL_F64) return occupancy_f64(scheme, trans, mon, block, gen);
    return occupancy_f32c(scheme, trans, mon, dtype, block, gen);
}

int check_track_args(const phtl_handle* h, void* const* c, int64_t n, int64_t turns,
                     int integrator, int dtype)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (integrator < PHTL_EULER_CROMER || integrator > PHTL_RK4) return PHTL_E_INVALID;
    if (dtype < PHTL_F64 || dtype > PHTL_F32CS) return PHTL_E_INVALID;
    if (n < 0 || turns < 0) return PHTL_E_INVALID;
    if (n > 0 && (!c[0] || !c[1])) return PHTL_E_INVALID;
    if ((c[2] == nullptr) != (c[3] == nullptr)) return PHTL_E_INVALID;
    if ((c[4] == nullptr) != (c[5] == nullptr)) return PHTL_E_INVALID;
    const uintptr_t es = dtype == PHTL_F64 ? 8 : 4;
    for (int i = 0; i < 6; ++i)
        if (c[i] && (reinterpret_cast<uintptr_t>(c[i]) % es) != 0) return PHTL_E_INVALID;
    return PHTL_OK;
}

// Enqueue the launches of one tracking call (persistent or per-turn family).
int enqueue_track(phtl_handle* h, void* const* c, int64_t n, int64_t turns, int integrator,
                  int dtype, cudaStream_t s, bool perturn, double* mon_rows, int64_t mon_cap,
                  int64_t mon_stride)
{
    int rc = ensure_device(h);
    if (rc != PHTL_OK) return rc;
    h->last_turns = turns;
    h->last_gated = false;
    if (mon_rows) {
        const int64_t nrows = turns / mon_stride + 1;
        if (nrows > mon_cap) return PHTL_E_INVALID;
        if (cudaMemsetAsync(mon_rows, 0, static_cast<size_t>(nrows) * PHTL_MON_FIELDS * sizeof(double),
                            s) != cudaSuccess) {
            cudaGetLastError();
            return PHTL_E_CUDA;
        }
    }
    if (n == 0) return PHTL_OK;
    if (turns == 0 && !mon_rows) return PHTL_OK;

    const bool trans = c[2] != nullptr || c[4] != nullptr;
    const bool mon = mon_rows != nullptr;
    // default block: for the FP64 persistent kernels 96 threads with a monitor (measured fastest
    // for all three schemes on 1e6 particles: 2.6 % over 128, 10 % over 256) and 32 without one
    // (EC + LF + Ruth4, transverse: 8.3 / 6.5 / 3.7 / 0.9 % over 96 at 1e5 / 3.3e5 / 1e6 / 4e6
    // particles: the last round of chunks is finer); 128 for the FP32 ones (block size made no
    // difference without a monitor), 256 for the per-turn launches
    const int block = h->block > 0 ? h->block
                                   : (perturn ? 256 : (dtype == PHTL_F64 ? (mon ? 96 : 32) : 128));
    const int es = dtype == PHTL_F64 ? 8 : 4;
    const int ppt = particles_per_thread(dtype);
    int64_t tpl = perturn ? 1 : (h->tpl > 0 ? h->tpl : auto_turns_per_launch(dtype, integrator, n));
    tpl = std::min<int64_t>(tpl, 1 << 30);

    bool vec = true;
    for (int i = 0; i < 6; ++i)
        if (c[i] && (reinterpret_cast<uintptr_t>(c[i]) % 16) != 0) vec = false;
    // FP32C buffers are [hi | comp]: the comp half is 16-byte aligned only if n % 4 == 0
    if (dtype != PHTL_F64 && (n * es) % 16 != 0) vec = false;

    const int occ = occupancy(dtype, integrator, trans, mon, block, perturn,
                              gen_level(h->mc[integrator]));
    if (occ <= 0) return PHTL_E_INVALID;
    const int64_t chunk = static_cast<int64_t>(block) * ppt;
    const int64_t nchunks = (n + chunk - 1) / chunk;
    const int64_t resident = static_cast<int64_t>(occ) * h->nsm;
    int64_t cap = resident;
    if (h->max_blocks > 0) cap = std::min<int64_t>(cap, h->max_blocks);
    const int grid = static_cast<int>(perturn ? nchunks : std::min<int64_t>(nchunks, cap));

    LaunchDesc L;
    std::memset(&L, 0, sizeof(L));
    for (int i = 0; i < 6; ++i) L.c[i] = c[i];
    L.n = n;
    L.scheme = integrator;
    L.block = block;
    L.grid = std::max(grid, 1);
    L.vec = vec ? 1 : 0;
    const MapConsts& mc = h->mc[integrator];
    // persistent calls: a cancellation gate in front of every launch (phtl_track_cancel)
    const bool gated = !perturn && h->ctl_dev && h->gate_go && !stream_capturing(s);
    const long long epoch = gated ? __atomic_add_fetch(&h->epoch, 1LL, __ATOMIC_SEQ_CST) : 0;
    h->last_gated = gated;
    L.go = gated ? h->gate_go : nullptr;

    int64_t t0 = 0;
    bool first = true;
    do {
        const int64_t nt = std::min<int64_t>(tpl, turns - t0);
        L.nturns = static_cast<int32_t>(nt);
        if (gated) {
            if (launch_gate(h->ctl_dev, epoch, h->gate_go, h->ctl_dev + 1, static_cast<int>(nt), first,
                            s) != cudaSuccess) {
                cudaGetLastError();
                return PHTL_E_CUDA;
            }
            ++h->stats.gate_launches;
        }
        MonitorArgs m;
        std::memset(&m, 0, sizeof(m));
        if (mon) {
            m.rows = mon_rows;
            m.stride = mon_stride;
            m.until = mon_stride - (t0 % mon_stride);
            m.row = t0 / mon_stride + 1;
            m.initial = first ? 1 : 0;
        }
        cudaError_t e;
        if (perturn)
            e = launch_perturn(L, mc, m, dtype, s);
        else if (dtype == PHTL_F64)
            e = launch_track_f64(L, mc, m, s);
        else
            e = launch_track_f32c(L, mc, m, dtype, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return PHTL_E_CUDA;
        }
        t0 += nt;
        first = false;
        ++h->stats.launches;
    } while (t0 < turns);
    h->stats.particle_turns += n * turns;
    ++h->stats.calls;
    if (log_level() > 0)
        log_line("%s n=%lld turns=%lld integrator=%d dtype=%d launches=%lld grid=%d block=%d "
                 "turns_per_launch=%lld monitor=%s transverse=%d", perturn ? "track_perturn" : "track",
                 static_cast<long long>(n), static_cast<long long>(turns), integrator, dtype,
                 static_cast<long long>((turns + tpl - 1) / std::max<int64_t>(tpl, 1)), L.grid,
                 block, static_cast<long long>(tpl), mon ? "on" : "off", trans ? 1 : 0);
    return PHTL_OK;
}

int track_common(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
                 int64_t n, int64_t turns, int integrator, int dtype, void* stream, bool perturn)
{
    void* c[6] = {z, dp, x, xp, y, yp};
    int rc = check_track_args(h, c, n, turns, integrator, dtype);
    if (rc != PHTL_OK) return rc;
    return enqueue_track(h, c, n, turns, integrator, dtype, static_cast<cudaStream_t>(stream),
                         perturn, h->mon_rows, h->mon_cap, h->mon_stride);
}

}  // namespace phtl

using namespace phtl;

extern "C" {

int phtl_create(const phtl_params* params, phtl_handle** out)
{
    if (!params || !out) return PHTL_E_INVALID;
    *out = nullptr;
    phtl_handle* h = new (std::nothrow) phtl_handle();
    if (!h) return PHTL_E_NOMEM;
    h->params = *params;
    int rc = derive(*params, h->derived, h->mc);
    if (rc != PHTL_OK) {
        delete h;
        return rc;
    }
    // RK4's kw2[0] is A2 itself; lin2 = cos(phi2) k2
    h->K2 = h->derived.etaC * h->mc[PHTL_RK4].kw2[0] * h->mc[PHTL_RK4].lin2;
    {
        std::lock_guard<std::mutex> g(g_registry_mu);
        g_registry.insert(h);
    }
    *out = h;
    return PHTL_OK;
}

int phtl_destroy(phtl_handle* h)
{
    {
        std::lock_guard<std::mutex> g(g_registry_mu);
        if (!h || !g_registry.count(h) || h->magic != kHandleMagic) return PHTL_E_BADHANDLE;
        g_registry.erase(h);
    }
    release_handle_resources(h);
    h->magic = 0;
    delete h;
    return PHTL_OK;
}

int phtl_get_derived(const phtl_handle* h, phtl_derived* out)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (!out) return PHTL_E_INVALID;
    *out = h->derived;
    return PHTL_OK;
}

const char* phtl_strerror(int code)
{
    switch (code) {
        case PHTL_OK: return "ok";
        case PHTL_E_INVALID: return "invalid argument";
        case PHTL_E_UNSTABLE: return "RF parameters give no stable bucket";
        case PHTL_E_NOMEM: return "out of memory or over the memory budget";
        case PHTL_E_CUDA: return "CUDA runtime error";
        case PHTL_E_TIMEOUT: return "timed out";
        case PHTL_E_CANCELLED: return "cancelled";
        case PHTL_E_BADHANDLE: return "bad handle or ticket";
        case PHTL_E_NODEVICE: return "no sm_103 CUDA device";
        case PHTL_E_TOOBIG: return "more jobs than the fixed table of the no-allocation batch run";
        case PHTL_E_CAPTURE: return "the stream is capturing a CUDA graph; this call cannot be captured";
        default: return "unknown error code";
    }
}

const char* phtl_version(void) { return "phtl 0.1 sm_103a"; }

int phtl_set_monitor(phtl_handle* h, double* rows, int64_t capacity_rows, int64_t stride)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (rows) {
        if (capacity_rows < 1 || stride < 1) return PHTL_E_INVALID;
        if (reinterpret_cast<uintptr_t>(rows) % 8 != 0) return PHTL_E_INVALID;
    }
    h->mon_rows = rows;
    h->mon_cap = rows ? capacity_rows : 0;
    h->mon_stride = rows ? stride : 1;
    return PHTL_OK;
}

int phtl_set_tuning(phtl_handle* h, int32_t block_threads, int64_t turns_per_launch,
                    int32_t max_blocks)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (block_threads != 0 && (block_threads < 32 || block_threads > 256 || block_threads % 32))
        return PHTL_E_INVALID;
    if (turns_per_launch < 0 || max_blocks < 0) return PHTL_E_INVALID;
    h->block = block_threads;
    h->tpl = turns_per_launch;
    h->max_blocks = max_blocks;
    return PHTL_OK;
}

int phtl_track(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
               int64_t n, int64_t turns, int integrator, int dtype, void* cuda_stream)
{
    return track_common(h, z, dp, x, xp, y, yp, n, turns, integrator, dtype, cuda_stream, false);
}

int phtl_track_perturn(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
                       int64_t n, int64_t turns, int integrator, int dtype, void* cuda_stream)
{
    return track_common(h, z, dp, x, xp, y, yp, n, turns, integrator, dtype, cuda_stream, true);
}

int phtl_track_host(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
                    int64_t n, int64_t turns, int integrator, int dtype, double* mon_rows,
                    int64_t mon_stride)
{
    const auto wall0 = std::chrono::steady_clock::now();
    void* hc[6] = {z, dp, x, xp, y, yp};
    int rc = check_track_args(h, hc, n, turns, integrator, dtype);
    if (rc != PHTL_OK) return rc;
    if (mon_rows && mon_stride < 1) return PHTL_E_INVALID;
    rc = ensure_device(h);
    if (rc != PHTL_OK) return rc;
    cudaStream_t s = nullptr;
    rc = handle_stream(h, &s);
    if (rc != PHTL_OK) return rc;
    for (cudaEvent_t& e : h->phase_ev) {
        if (!e && cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
            return PHTL_E_CUDA;
        }
    }
    cudaEvent_t* ev = h->phase_ev;
    const size_t per = 8u * static_cast<size_t>(n);  // n doubles or 2n floats
    const int64_t nrows = mon_rows ? turns / mon_stride + 1 : 0;
    const size_t mon_bytes = static_cast<size_t>(nrows) * PHTL_MON_FIELDS * sizeof(double);
    void* dc[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double* dmon = nullptr;
    int nplanes = 0;
    for (int i = 0; i < 6; ++i)
        if (hc[i]) ++nplanes;
    auto release = [&]() {
        for (int i = 0; i < 6; ++i)
            if (dc[i]) cudaFreeAsync(dc[i], s);
        if (dmon) cudaFreeAsync(dmon, s);
    };
    auto fail = [&](int code) {
        cudaGetLastError();
        release();
        cudaStreamSynchronize(s);
        cudaGetLastError();
        return code;
    };
    // allocate
    cudaEventRecord(ev[0], s);
    for (int i = 0; i < 6 && n > 0; ++i) {
        if (!hc[i]) continue;
        if (cudaMallocAsync(&dc[i], per, s) != cudaSuccess) return fail(PHTL_E_NOMEM);
    }
    if (mon_rows && cudaMallocAsync(reinterpret_cast<void**>(&dmon), mon_bytes, s) != cudaSuccess)
        return fail(PHTL_E_NOMEM);
    // copy in
    cudaEventRecord(ev[1], s);
    for (int i = 0; i < 6 && n > 0; ++i)
        if (hc[i] && cudaMemcpyAsync(dc[i], hc[i], per, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(PHTL_E_CUDA);
    // kernels
    cudaEventRecord(ev[2], s);
    const int64_t l0 = h->stats.launches;
    rc = enqueue_track(h, dc, n, turns, integrator, dtype, s, false, dmon, nrows,
                       mon_rows ? mon_stride : 1);
    if (rc != PHTL_OK) return fail(rc);
    // copy out
    cudaEventRecord(ev[3], s);
    for (int i = 0; i < 6 && n > 0; ++i)
        if (hc[i] && cudaMemcpyAsync(hc[i], dc[i], per, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return fail(PHTL_E_CUDA);
    if (mon_rows && cudaMemcpyAsync(mon_rows, dmon, mon_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return fail(PHTL_E_CUDA);
    // free
    cudaEventRecord(ev[4], s);
    release();
    cudaEventRecord(ev[5], s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return PHTL_E_CUDA;
    }
    phtl_phase_times& P = h->phases;
    float ms[5] = {0, 0, 0, 0, 0}, tot = 0.0f;
    for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
    cudaEventElapsedTime(&tot, ev[0], ev[5]);
    cudaGetLastError();
    P.alloc_ms = ms[0];
    P.h2d_ms = ms[1];
    P.kernel_ms = ms[2];
    P.d2h_ms = ms[3];
    P.free_ms = ms[4];
    P.total_ms = tot;
    P.h2d_bytes = n > 0 ? static_cast<int64_t>(per) * nplanes : 0;
    P.d2h_bytes = P.h2d_bytes + static_cast<int64_t>(mon_bytes);
    P.launches = h->stats.launches - l0;
    P.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    if (log_level() > 0)
        log_line("track_host alloc=%.3f h2d=%.3f kernel=%.3f d2h=%.3f free=%.3f total=%.3f wall=%.3f ms",
                 P.alloc_ms, P.h2d_ms, P.kernel_ms, P.d2h_ms, P.free_ms, P.total_ms, P.wall_ms);
    return PHTL_OK;
}

int phtl_get_phase_times(const phtl_handle* h, phtl_phase_times* out)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (!out) return PHTL_E_INVALID;
    *out = h->phases;
    return PHTL_OK;
}

int phtl_track_cancel(phtl_handle* h)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (!h->ctl_host) return PHTL_OK;  // nothing was ever enqueued
    __atomic_store_n(&h->ctl_host[0], __atomic_load_n(&h->epoch, __ATOMIC_SEQ_CST), __ATOMIC_SEQ_CST);
    return PHTL_OK;
}

int phtl_track_status(const phtl_handle* h, int64_t* turns_done)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (!turns_done) return PHTL_E_INVALID;
    if (!h->last_gated) {
        *turns_done = h->last_turns;
        return PHTL_OK;
    }
    const long long done = __atomic_load_n(&h->ctl_host[1], __ATOMIC_SEQ_CST);
    *turns_done = done;
    return done < h->last_turns ? PHTL_E_CANCELLED : PHTL_OK;
}

int phtl_get_stats(const phtl_handle* h, phtl_stats* out)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (!out) return PHTL_E_INVALID;
    *out = h->stats;
    return PHTL_OK;
}

int phtl_moments_from_sums(const double* row, double* out)
{
    if (!row || !out) return PHTL_E_INVALID;
    for (int j = 0; j < 15; ++j) out[j] = 0.0;
    const double n = row[0];
    if (!(n > 0.0)) return PHTL_OK;
    for (int plane = 0; plane < 3; ++plane) {
        const double* s = row + 1 + 5 * plane;
        double* o = out + 5 * plane;
        const double ma = s[0] / n, mb = s[1] / n;
        const double vaa = std::max(s[2] / n - ma * ma, 0.0);
        const double vbb = std::max(s[3] / n - mb * mb, 0.0);
        const double vab = s[4] / n - ma * mb;
        o[0] = ma;
        o[1] = mb;
        o[2] = std::sqrt(vaa);
        o[3] = std::sqrt(vbb);
        o[4] = std::sqrt(std::max(vaa * vbb - vab * vab, 0.0));
    }
    return PHTL_OK;
}

}  // extern "C"
