// Host side of the collective step (phtl_set_wake, phtl_collective_kick,
// phtl_track_collective): the library-owned slicing buffers and the per-turn launches of
// the turn and potential kernels (track_collective.cu, track_collective_f32.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "handle.h"
#include "internal.h"

namespace phtl {

void free_wake(phtl_handle* h)
{
    if (h->wake_mem) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (h->wake_device >= 0 && cur != h->wake_device) cudaSetDevice(h->wake_device);
        cudaDeviceSynchronize();
        cudaFree(h->wake_mem);
        if (h->coll_slot) cudaFree(h->coll_slot);
        if (cur >= 0 && cur != h->wake_device) cudaSetDevice(cur);
    }
    h->coll_slot = nullptr;
    h->coll_slot_cap = 0;
    h->wake_mem = nullptr;
    h->wake_w = h->wake_V = h->wake_U = nullptr;
    h->wake_U2 = nullptr;
    h->wake_counts = nullptr;
    h->wake_device = -1;
    std::memset(&h->coll, 0, sizeof(h->coll));
    cudaGetLastError();
}

}  // namespace phtl

using namespace phtl;

extern "C" {

int phtl_set_wake(phtl_handle* h, const phtl_wake* wk)
{
    if (!handle_valid(h)) return PHTL_E_BADHANDLE;
    if (!wk) {
        free_wake(h);
        return PHTL_OK;
    }
    const int ns = wk->nslices;
    if (ns < 1 || ns > PHTL_MAX_SLICES || !wk->w || !std::isfinite(wk->z_lo) ||
        !std::isfinite(wk->z_hi) || !(wk->z_hi > wk->z_lo) || !std::isfinite(wk->alpha) ||
        !std::isfinite(wk->alpha_sc))
        return PHTL_E_INVALID;
    for (int m = 0; m < ns; ++m)
        if (!std::isfinite(wk->w[m])) return PHTL_E_INVALID;
    const double inv_dz = static_cast<double>(ns) / (wk->z_hi - wk->z_lo);
    if (!std::isfinite(inv_dz)) return PHTL_E_INVALID;
    int rc = ensure_device(h);
    if (rc != PHTL_OK) return rc;
    free_wake(h);
    // w, V, U (doubles), U2 (float pairs), two counts buffers
    const size_t bytes = static_cast<size_t>(ns) * (3 * sizeof(double) + sizeof(float2) + 2 * sizeof(unsigned));
    if (cudaMalloc(&h->wake_mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        h->wake_mem = nullptr;
        return PHTL_E_NOMEM;
    }
    h->wake_w = static_cast<double*>(h->wake_mem);
    h->wake_V = h->wake_w + ns;
    h->wake_U = h->wake_V + ns;
    h->wake_U2 = reinterpret_cast<float2*>(h->wake_U + ns);
    h->wake_counts = reinterpret_cast<unsigned*>(h->wake_U2 + ns);
    if (cudaMemcpy(h->wake_w, wk->w, sizeof(double) * ns, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->wake_V, 0, bytes - sizeof(double) * ns) != cudaSuccess) {
        cudaGetLastError();
        free_wake(h);
        return PHTL_E_CUDA;
    }
    h->wake_device = h->device;
    h->coll.z_lo = wk->z_lo;
    h->coll.inv_dz = inv_dz;
    h->coll.alpha = wk->alpha;
    h->coll.alpha_sc = wk->alpha_sc;
    h->coll.nslices = ns;
    split_df(wk->z_lo, h->coll.z_lo_h, h->coll.z_lo_l);
    split_df(inv_dz, h->coll.inv_dz_h, h->coll.inv_dz_l);
    return PHTL_OK;
}

namespace {

// Launch shape of the collective kernels for n particles (grid = resident capacity).
int coll_launch(phtl_handle* h, void* const* c, int64_t n, int integrator, int dtype, LaunchDesc& L)
{
    const int block = h->block > 0 ? h->block : 128;
    const int occ = dtype == PHTL_F64 ? occupancy_coll(integrator, h->mc[integrator].general != 0, block,
                                                       h->coll.nslices)
                                      : occupancy_coll_f32(integrator, dtype, h->mc[integrator].general != 0,
                                                           block, h->coll.nslices);
    if (occ <= 0) return PHTL_E_INVALID;
    const int64_t chunk = static_cast<int64_t>(block) * particles_per_thread(dtype);
    const int64_t nchunks = (n + chunk - 1) / chunk;
    int64_t cap = static_cast<int64_t>(occ) * h->nsm;
    if (h->max_blocks > 0) cap = std::min<int64_t>(cap, h->max_blocks);
    std::memset(&L, 0, sizeof(L));
    bool vec = true;
    for (int i = 0; i < 6; ++i) {
        L.c[i] = c[i];
        if (c[i] && (reinterpret_cast<uintptr_t>(c[i]) % 16) != 0) vec = false;
    }
    // FP32C buffers are [hi | comp]: the comp half is 16-byte aligned only if n % 4 == 0
    if (dtype != PHTL_F64 && (n * 4) % 16 != 0) vec = false;
    L.n = n;
    L.scheme = integrator;
    L.block = block;
    L.grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(nchunks, cap)));
    L.vec = vec ? 1 : 0;
    L.nturns = 1;
    return PHTL_OK;
}

int coll_ready(phtl_handle* h)
{
    int rc = ensure_device(h);
    if (rc != PHTL_OK) return rc;
    if (!h->wake_mem || h->wake_device != h->device) return PHTL_E_INVALID;
    return PHTL_OK;
}

int cuda_ok(cudaError_t e)
{
    if (e == cudaSuccess) return PHTL_OK;
    cudaGetLastError();
    return PHTL_E_CUDA;
}

// The per-particle slice buffer for n particles on the wake's device (grown, never shrunk;
// the old one is freed after the work that may still use it).
int ensure_slots(phtl_handle* h, int64_t n)
{
    if (n <= h->coll_slot_cap) return PHTL_OK;
    if (h->coll_slot) {
        cudaDeviceSynchronize();
        cudaFree(h->coll_slot);
        h->coll_slot = nullptr;
        h->coll_slot_cap = 0;
    }
    const int64_t cap = (n + 4095) / 4096 * 4096;
    if (cudaMalloc(&h->coll_slot, static_cast<size_t>(cap) * sizeof(uint16_t)) != cudaSuccess) {
        cudaGetLastError();
        h->coll_slot = nullptr;
        return PHTL_E_NOMEM;
    }
    h->coll_slot_cap = cap;
    return PHTL_OK;
}

// One launch of the collective turn kernel of the arithmetic type.
int coll_turn(phtl_handle* h, const LaunchDesc& L, const MapConsts& mc, unsigned* counts,
              double* mon, int64_t rec, bool kick, bool map, int dtype, cudaStream_t s)
{
    if (dtype == PHTL_F64)
        return cuda_ok(launch_coll_turn(L, mc, h->coll, h->wake_U, counts, h->coll_slot, mon, rec,
                                        kick, map, s));
    return cuda_ok(launch_coll_turn_f32(L, mc, h->coll, h->wake_U2, counts, h->coll_slot, mon, rec,
                                        kick, map, dtype, s));
}

int coll_potential(phtl_handle* h, unsigned* counts, unsigned* clear, cudaStream_t s)
{
    return cuda_ok(launch_wake_potential(counts, h->wake_w, h->coll, h->wake_V, h->wake_U,
                                         h->wake_U2, clear, s));
}

}  // namespace

int phtl_collective_kick(phtl_handle* h, void* z, void* dp, int64_t n, int dtype,
                         uint32_t* counts_out, double* V_out, void* cuda_stream)
{
    void* c[6] = {z, dp, nullptr, nullptr, nullptr, nullptr};
    int rc = check_track_args(h, c, n, 0, PHTL_LEAPFROG, dtype);
    if (rc != PHTL_OK) return rc;
    rc = coll_ready(h);
    if (rc != PHTL_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int ns = h->coll.nslices;
    unsigned* cnt = h->wake_counts;
    rc = cuda_ok(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * ns, s));
    if (rc == PHTL_OK && n > 0) {
        LaunchDesc L;
        const MapConsts& mc = h->mc[PHTL_LEAPFROG];
        rc = ensure_slots(h, n);
        if (rc == PHTL_OK) rc = coll_launch(h, c, n, PHTL_LEAPFROG, dtype, L);
        if (rc == PHTL_OK) rc = coll_turn(h, L, mc, cnt, nullptr, -1, false, false, dtype, s);
        if (rc == PHTL_OK) rc = coll_potential(h, cnt, nullptr, s);
        if (rc == PHTL_OK) rc = coll_turn(h, L, mc, nullptr, nullptr, -1, true, false, dtype, s);
        if (rc == PHTL_OK) h->stats.launches += 3;
    } else if (rc == PHTL_OK) {
        rc = cuda_ok(cudaMemsetAsync(h->wake_V, 0, 2 * sizeof(double) * ns, s));
    }
    if (rc == PHTL_OK && counts_out)
        rc = cuda_ok(cudaMemcpyAsync(counts_out, cnt, sizeof(unsigned) * ns, cudaMemcpyDeviceToDevice, s));
    if (rc == PHTL_OK && V_out)
        rc = cuda_ok(cudaMemcpyAsync(V_out, h->wake_V, sizeof(double) * ns, cudaMemcpyDeviceToDevice, s));
    return rc;
}

int phtl_track_collective(phtl_handle* h, void* z, void* dp, void* x, void* xp, void* y, void* yp,
                          int64_t n, int64_t turns, int integrator, int dtype, void* cuda_stream)
{
    void* c[6] = {z, dp, x, xp, y, yp};
    int rc = check_track_args(h, c, n, turns, integrator, dtype);
    if (rc != PHTL_OK) return rc;
    rc = coll_ready(h);
    if (rc != PHTL_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double* mon = h->mon_rows;
    const int64_t stride = h->mon_stride;
    if (mon) {
        const int64_t nrows = turns / stride + 1;
        if (nrows > h->mon_cap) return PHTL_E_INVALID;
        rc = cuda_ok(cudaMemsetAsync(mon, 0, static_cast<size_t>(nrows) * PHTL_MON_FIELDS * sizeof(double), s));
        if (rc != PHTL_OK) return rc;
    }
    if (n == 0 || (turns == 0 && !mon)) return PHTL_OK;
    rc = ensure_slots(h, n);
    if (rc != PHTL_OK) return rc;
    LaunchDesc L;
    rc = coll_launch(h, c, n, integrator, dtype, L);
    if (rc != PHTL_OK) return rc;
    const int ns = h->coll.nslices;
    unsigned* cnt[2] = {h->wake_counts, h->wake_counts + ns};
    const MapConsts& mc = h->mc[integrator];
    rc = cuda_ok(cudaMemsetAsync(h->wake_counts, 0, 2 * sizeof(unsigned) * ns, s));
    // turn t: the previous turn's kick (t > 1), its monitor row, the map, the slicing; then
    // the potential of the new counts (clearing the other buffer for the next turn)
    for (int64_t t = 1; t <= turns && rc == PHTL_OK; ++t) {
        const int64_t rec = (mon && (t - 1) % stride == 0) ? (t - 1) / stride : -1;
        rc = coll_turn(h, L, mc, cnt[t & 1], mon, rec, t > 1, true, dtype, s);
        if (rc == PHTL_OK) rc = coll_potential(h, cnt[t & 1], cnt[(t + 1) & 1], s);
    }
    // the last turn's kick and monitor row
    if (rc == PHTL_OK) {
        const int64_t rec = (mon && turns % stride == 0) ? turns / stride : -1;
        rc = coll_turn(h, L, mc, nullptr, mon, rec, turns > 0, false, dtype, s);
    }
    if (rc != PHTL_OK) return rc;
    h->stats.launches += 2 * turns + 1;
    h->stats.particle_turns += n * turns;
    ++h->stats.calls;
    return PHTL_OK;
}

}  // extern "C"
