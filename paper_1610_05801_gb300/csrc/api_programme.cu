// Host side of the ramp programme (phtl_set_programme, phtl_track_programme): the
// per-turn constants in FP64 and the launches of the ramp kernels (track_ramp.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "handle.h"
#include "internal.h"

namespace phtl {

void free_programme(phtl_handle* h)
{
    if (h->ramp) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (h->ramp_device >= 0 && cur != h->ramp_device) cudaSetDevice(h->ramp_device);
        cudaDeviceSynchronize();
        cudaFree(h->ramp);
        if (cur >= 0 && cur != h->ramp_device) cudaSetDevice(cur);
        h->ramp = nullptr;
    }
    h->ramp_turns = 0;
    h->ramp_device = -1;
    cudaGetLastError();
}

// Per-turn constants of a ramp programme in FP64 (the reading stated at
// phtl_set_programme in phtl.h), with their double-float splits.
int derive_programme(const phtl_params& p, const double* V, const double* p0, int64_t nturns,
                     RampTurn* out)
{
    const double k = 2.0 * kPi * static_cast<double>(p.harmonic) / p.circumference_m;
    for (int64_t t = 0; t < nturns; ++t) {
        const double pa = p0[t], pb = p0[t + 1];
        if (!finite_pos(pa) || !finite_pos(pb) || !std::isfinite(V[t])) return PHTL_E_INVALID;
        const double bg = pa / p.mass_eV;
        const double g = std::sqrt(1.0 + bg * bg);
        const double b = bg / g;
        const double eta = 1.0 / (p.gamma_t * p.gamma_t) - 1.0 / (g * g);
        RampTurn& T = out[t];
        std::memset(&T, 0, sizeof(T));
        T.etaC = eta * p.circumference_m;
        T.A = p.charge_e * V[t] / (b * pa);
        if (V[t] == 0.0) {
            if (pb != pa) return PHTL_E_INVALID;
        } else {
            const double x = b * (pb - pa) / (p.charge_e * V[t]);
            if (!(std::fabs(x) < 1.0)) return PHTL_E_UNSTABLE;
            T.phis = eta > 0.0 ? std::asin(x) : kPi - std::asin(x);
            T.sinphis = std::sin(T.phis);
            const double K = T.etaC * T.A * k * std::cos(T.phis);
            if (!(K > 0.0 && K < 4.0)) return PHTL_E_UNSTABLE;
        }
        T.lin = std::cos(T.phis) * k;
        T.r = pa / pb;
        const struct {
            int scheme;
            double* w;
            int nd, nk;
        } sw[3] = {{PHTL_EULER_CROMER, T.w_ec, 1, 1}, {PHTL_LEAPFROG, T.w_lf, 2, 1},
                   {PHTL_RUTH4, T.w_r4, 4, 3}};
        for (const auto& e : sw) {
            for (int i = 0; i < e.nd; ++i) e.w[i] = drift_weight(e.scheme, i) * T.etaC;
            for (int j = 0; j < e.nk; ++j) e.w[e.nd + j] = kick_weight(e.scheme, j) * T.A;
        }
        split_df(T.etaC, T.etaC_h, T.etaC_l);
        split_df(T.A, T.A_h, T.A_l);
        split_df(T.phis, T.phis_h, T.phis_l);
        split_df(T.sinphis, T.sinphis_h, T.sinphis_l);
        split_df(T.lin, T.lin_h, T.lin_l);
        split_df(T.r, T.r_h, T.r_l);
    }
    return PHTL_OK;
}

}  // namespace phtl

using namespace phtl;

extern "C" {

int phtl_set_programme(phtl_handle* h, const double* voltage_V, const double* p0_eVc,
                       int64_t nturns)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (nturns < 0 || (nturns > 0 && (!voltage_V || !p0_eVc))) return PHTL_E_INVALID;
    if (nturns > (int64_t(1) << 32)) return PHTL_E_INVALID;
    if (nturns == 0) {
        free_programme(h);
        return PHTL_OK;
    }
    const phtl_params& p = h->params;
    if (p.eta1 != 0.0 || p.eta2 != 0.0 || p.xi_x != 0.0 || p.xi_y != 0.0 || p.voltage2_V != 0.0)
        return PHTL_E_INVALID;  // the programme runs the linear map only
    RampTurn* host = nullptr;
    if (cudaMallocHost(reinterpret_cast<void**>(&host), sizeof(RampTurn) * nturns) != cudaSuccess) {
        cudaGetLastError();
        // no device (or no pinned memory): validate on the heap so argument errors still
        // come first, then report the missing device
        RampTurn* tmp = new (std::nothrow) RampTurn[static_cast<size_t>(std::min<int64_t>(nturns, 1 << 20))];
        int rc = PHTL_E_NOMEM;
        if (tmp) {
            rc = PHTL_OK;
            for (int64_t t0 = 0; t0 < nturns && rc == PHTL_OK; t0 += 1 << 20) {
                const int64_t cnt = std::min<int64_t>(1 << 20, nturns - t0);
                rc = derive_programme(p, voltage_V + t0, p0_eVc + t0, cnt, tmp);
            }
            delete[] tmp;
        }
        if (rc != PHTL_OK) return rc;
        rc = ensure_device(h);
        return rc != PHTL_OK ? rc : PHTL_E_NOMEM;
    }
    int rc = derive_programme(p, voltage_V, p0_eVc, nturns, host);
    if (rc == PHTL_OK) rc = ensure_device(h);
    if (rc == PHTL_OK) {
        free_programme(h);
        if (cudaMalloc(reinterpret_cast<void**>(&h->ramp), sizeof(RampTurn) * nturns) != cudaSuccess) {
            cudaGetLastError();
            h->ramp = nullptr;
            rc = PHTL_E_NOMEM;
        } else if (cudaMemcpy(h->ramp, host, sizeof(RampTurn) * nturns, cudaMemcpyHostToDevice) !=
                   cudaSuccess) {
            cudaGetLastError();
            cudaFree(h->ramp);
            h->ramp = nullptr;
            rc = PHTL_E_CUDA;
        } else {
            h->ramp_turns = nturns;
            h->ramp_device = h->device;
        }
    }
    cudaFreeHost(host);
    return rc;
}

int phtl_track_programme(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
                         int64_t n, int64_t turn0, int64_t turns, int integrator, int dtype,
                         void* cuda_stream)
{
    void* c[6] = {z, dp, x, xp, y, yp};
    int rc = check_track_args(h, c, n, turns, integrator, dtype);
    if (rc != PHTL_OK) return rc;
    if (integrator == PHTL_RK4) return PHTL_E_INVALID;
    if (turn0 < 0 || turns > h->ramp_turns - turn0) return PHTL_E_INVALID;
    rc = ensure_device(h);
    if (rc != PHTL_OK) return rc;
    if (!h->ramp || h->ramp_device != h->device) return PHTL_E_INVALID;
    h->last_turns = turns;
    h->last_gated = false;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double* mon_rows = h->mon_rows;
    if (mon_rows) {
        const int64_t nrows = turns / h->mon_stride + 1;
        if (nrows > h->mon_cap) return PHTL_E_INVALID;
        if (cudaMemsetAsync(mon_rows, 0, static_cast<size_t>(nrows) * PHTL_MON_FIELDS * sizeof(double),
                            s) != cudaSuccess) {
            cudaGetLastError();
            return PHTL_E_CUDA;
        }
    }
    if (n == 0 || (turns == 0 && !mon_rows)) return PHTL_OK;
    // default block: 96 threads in FP64 (2 % over 128 on 1e6 x 4000 turns), 128 in FP32
    const int block = h->block > 0 ? h->block : (dtype == PHTL_F64 ? 96 : 128);
    const int ppt = particles_per_thread(dtype);
    int64_t tpl = h->tpl > 0 ? h->tpl : auto_turns_per_launch(dtype, integrator, n);
    tpl = std::min<int64_t>(tpl, 1 << 30);
    bool vec = true;
    for (int i = 0; i < 6; ++i)
        if (c[i] && (reinterpret_cast<uintptr_t>(c[i]) % 16) != 0) vec = false;
    if (dtype != PHTL_F64 && (n * 4) % 16 != 0) vec = false;
    const int occ = occupancy_ramp(integrator, dtype, block);
    if (occ <= 0) return PHTL_E_INVALID;
    const int64_t chunk = static_cast<int64_t>(block) * ppt;
    const int64_t nchunks = (n + chunk - 1) / chunk;
    int64_t cap = static_cast<int64_t>(occ) * h->nsm;
    if (h->max_blocks > 0) cap = std::min<int64_t>(cap, h->max_blocks);
    LaunchDesc L;
    std::memset(&L, 0, sizeof(L));
    for (int i = 0; i < 6; ++i) L.c[i] = c[i];
    L.n = n;
    L.scheme = integrator;
    L.block = block;
    L.grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(nchunks, cap)));
    L.vec = vec ? 1 : 0;
    // a cancellation gate in front of every launch (phtl_track_cancel), as in phtl_track
    const bool gated = h->ctl_dev && h->gate_go && !stream_capturing(s);
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
        if (mon_rows) {
            m.rows = mon_rows;
            m.stride = h->mon_stride;
            m.until = h->mon_stride - (t0 % h->mon_stride);
            m.row = t0 / h->mon_stride + 1;
            m.initial = first ? 1 : 0;
        }
        if (launch_ramp(L, h->mc[integrator], m, h->ramp, turn0 + t0, dtype, s) != cudaSuccess) {
            cudaGetLastError();
            return PHTL_E_CUDA;
        }
        t0 += nt;
        first = false;
        ++h->stats.launches;
    } while (t0 < turns);
    h->stats.particle_turns += n * turns;
    ++h->stats.calls;
    return PHTL_OK;
}

}  // extern "C"
