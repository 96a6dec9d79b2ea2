// Collective step kernels: longitudinal slicing of the bunch, the wake potential of the
// slice counts and the wake kick, interleaved with the one-turn map (FP64).
//
// The paper's conclusion names collective effects as the next workload after tracking; the
// reading is stated in phtl.h at phtl_set_wake: after each turn's map, the particles are
// counted on a uniform grid of slices, V_k = sum_{j >= k} c_j w[j - k] is formed, and each
// particle inside the grid gets delta += alpha V_k + alpha_sc D_k of its own slice, D_k the
// central difference of the counts (longitudinal space charge).
//
// The step needs the whole bunch's histogram between two turns, so the state cannot stay
// in registers across turns as in the persistent kernels: each turn is one launch of
// k_coll_turn (apply the previous turn's kick, record the monitor row, run the turn's map,
// count the new z into a block-private shared-memory histogram that is flushed to the
// global counts with one atomic per non-empty slice, and keep each particle's slice for the
// next launch's kick), then one launch of k_wake_potential
// (counts and table staged in shared memory, one warp per slice, lane-strided partial sums
// and a shuffle reduction; it also clears the other counts buffer for the next turn).  The state makes one HBM round trip per
// turn (96 bytes per particle with both transverse planes, and 4 bytes of slices), well
// under the FP64 work of the turn on GB300.  Integer counts make the histogram exact and independent of the
// order of the atomics.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "monitor.cuh"
#include "ops_f64.cuh"

namespace phtl {
namespace {

using namespace f64;

// Slice of z on the uniform grid [z_lo, z_lo + ns / inv_dz), or -1 outside: the same two
// FP64 operations (subtract, multiply) as the definition give u, and the decision
// 0 <= u < ns, k = floor(u) is taken exactly on u's bit pattern with integer instructions:
// non-negative doubles order like their bits, so u < ns (ns integral, its low word zero)
// is hi < ns_hi on the high words; -0.0 counts as 0; NaN and +Inf lie above every finite
// bound.  The compare, floor and conversion instructions would run on the FP64 pipe.
// ns_hi: the high word of (double)ns.
__device__ __forceinline__ int slice_of(double z, double z_lo, double inv_dz, int ns_hi)
{
    const double u = __dmul_rn(__dsub_rn(z, z_lo), inv_dz);
    const int hi = __double2hiint(u);
    if (hi < 0) return ((hi << 1) | __double2loint(u)) == 0 ? 0 : -1;  // -0.0, or u < 0
    if (hi >= ns_hi) return -1;
    return floor_small(hi);
}

// One turn of the collective tracking for one particle chunk per loop iteration.
//   kick:  apply delta += U[k] with the previous turn's per-slice kick U
//   rec:   monitor row to record after the kick (-1: none)
//   map:   run the turn's map and the transverse rotation
//   cnt:   counts buffer for the new z (nullptr: no slicing)
//   slot:  per-particle slices: written with the counts, read by the kick (the kick of the
//          next launch needs the slice of the same z, so it is decided once per turn)
// GEN: the widened map's code (slippage expansion, chromaticity, second RF system, RK4);
// otherwise the linear map's, which a ring without those terms gives bitwise the same result
// with fewer FP64 operations (a drift is one FMA instead of three).
// Shared memory: ns uint32 histogram bins, then the monitor's 2 * warps * 16 DF2.
template <int S, bool GEN>
__global__ void __launch_bounds__(256, 3)
    k_coll_turn(LaunchDesc L, MapConsts c, CollArgs A, const double* __restrict__ U,
                unsigned* __restrict__ counts, uint16_t* __restrict__ slot,
                double* __restrict__ mon_rows, int64_t rec_row, int kick, int map)
{
    extern __shared__ double smem_d[];
    unsigned* hist = reinterpret_cast<unsigned*>(smem_d);
    double* msm = smem_d + (A.nslices + 1) / 2;  // 8-byte aligned after the bins
    double* g[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = static_cast<double*>(L.c[i]);
    const bool hx = g[2] != nullptr, hy = g[4] != nullptr;
    const bool vec = L.vec != 0;
    if (counts)
        for (int k = threadIdx.x; k < A.nslices; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    griddep_wait();  // the previous turn's state, kick and cleared counts
    const int64_t chunk = static_cast<int64_t>(blockDim.x) * P;
    const int64_t nchunks = (L.n + chunk - 1) / chunk;
    int parity = 0;
    double g1[4], g2[4];
    if (GEN) slip_stages<S>(c, g1, g2);
    const int ns_hi = __double2hiint(static_cast<double>(A.nslices));
    for (int64_t ci = blockIdx.x; ci < nchunks; ci += gridDim.x) {
        const int64_t base = ci * chunk + static_cast<int64_t>(threadIdx.x) * P;
        double z[P], d[P], x[P], xp[P], y[P], yp[P];
        load2(g[0], base, L.n, vec, z);
        load2(g[1], base, L.n, vec, d);
#pragma unroll
        for (int p = 0; p < P; ++p) x[p] = xp[p] = y[p] = yp[p] = 0.0;
        if (hx) {
            load2(g[2], base, L.n, vec, x);
            load2(g[3], base, L.n, vec, xp);
        }
        if (hy) {
            load2(g[4], base, L.n, vec, y);
            load2(g[5], base, L.n, vec, yp);
        }
        const int64_t left = L.n - base;
        const float cnt = left >= P ? static_cast<float>(P) : (left > 0 ? static_cast<float>(left) : 0.0f);
        if (kick) {
            int k[P];
            slots_load<P>(slot, base, L.n, k);
#pragma unroll
            for (int p = 0; p < P; ++p)
                if (k[p] != static_cast<int>(kSlotOutside)) d[p] = d[p] + __ldg(U + k[p]);
        }
        if (mon_rows && rec_row >= 0) {
            record<true>(z, d, x, xp, y, yp, cnt, hx, hy, msm, parity, mon_rows, rec_row);
            parity ^= 1;
        }
        if (map) {
            if constexpr (GEN) {
                if (c.phis_zero) long_turn_nl<S, true>(z, d, c, c.dc, c.kw, c.kw2, g1, g2, c.dual_rf != 0);
                else long_turn_nl<S, false>(z, d, c, c.dc, c.kw, c.kw2, g1, g2, c.dual_rf != 0);
                transverse_gen(x, xp, y, yp, d, hx, hy, c);
            } else {
                if (c.phis_zero) long_turn<S, true>(z, d, c, c.dc, c.kw);
                else long_turn<S, false>(z, d, c, c.dc, c.kw);
                if (hx) rotate(x, xp, c.mx, c.shx, c.shear_x != 0);
                if (hy) rotate(y, yp, c.my, c.shy, c.shear_y != 0);
            }
        }
        if (counts) {
            int k[P];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                k[p] = base + p < L.n ? slice_of(z[p], A.z_lo, A.inv_dz, ns_hi) : -1;
                if (k[p] >= 0) atomicAdd(hist + k[p], 1u);
            }
            slots_store<P>(slot, base, L.n, k);
        }
        store2(g[0], base, L.n, vec, z);
        store2(g[1], base, L.n, vec, d);
        if (hx) {
            store2(g[2], base, L.n, vec, x);
            store2(g[3], base, L.n, vec, xp);
        }
        if (hy) {
            store2(g[4], base, L.n, vec, y);
            store2(g[5], base, L.n, vec, yp);
        }
    }
    // the potential kernel may launch now (it waits for this grid's completion); not earlier,
    // so that its blocks do not sit on SM slots while this grid still works
    griddep_launch_dependents();
    if (counts) {
        __syncthreads();
        for (int k = threadIdx.x; k < A.nslices; k += blockDim.x) {
            const unsigned h = hist[k];
            if (h) atomicAdd(counts + k, h);
        }
    }
}

// V_k = sum_{j >= k} c_j w[j - k] and the per-slice kick U_k = alpha V_k + alpha_sc D_k,
// D_k the central difference of the counts (one-sided at the ends); U2 holds U as float
// pairs for the FP32 paths.  Every block stages the
// counts (as doubles) and the wake table in shared memory with one coalesced pass, then
// each of its warps forms one slice at a time: lane-strided partial sums, then a butterfly
// reduction (a fixed order, so the result does not depend on the launch).  Block 0 also
// clears `clear` (the other counts buffer) for the next turn.  Shared memory: 2 ns doubles.
__global__ void __launch_bounds__(256)
    k_wake_potential(const unsigned* __restrict__ counts, const double* __restrict__ w, int ns,
                     double alpha, double alpha_sc, double* __restrict__ V, double* __restrict__ U,
                     float2* __restrict__ U2, unsigned* __restrict__ clear)
{
    extern __shared__ double sm[];
    double* c = sm;
    double* ws = sm + ns;
    griddep_wait();  // the counts of the turn kernel that precedes this launch
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
        c[k] = static_cast<double>(counts[k]);
        ws[k] = w[k];
    }
    __syncthreads();
    if (clear && blockIdx.x == 0)
        for (int k = threadIdx.x; k < ns; k += blockDim.x) clear[k] = 0u;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int k = blockIdx.x * wpb + (threadIdx.x >> 5); k < ns; k += gridDim.x * wpb) {
        double s = 0.0;
        for (int j = k + lane; j < ns; j += 32) s = fma(c[j], ws[j - k], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFullMask, s, o);
        if (lane == 0) {
            double dk = 0.0;
            if (ns > 1)
                dk = k == 0 ? c[1] - c[0] : k == ns - 1 ? c[ns - 1] - c[ns - 2] : 0.5 * (c[k + 1] - c[k - 1]);
            V[k] = s;
            const double u = fma(alpha, s, alpha_sc * dk);
            U[k] = u;
            const DF2 p = split_bits(u);  // the FP32 paths' copy
            U2[k] = make_float2(p.h, p.l);
        }
    }
    griddep_launch_dependents();
}

template <int S>
const void* coll_kernel_s(bool gen)
{
    return gen ? reinterpret_cast<const void*>(&k_coll_turn<S, true>)
               : reinterpret_cast<const void*>(&k_coll_turn<S, false>);
}

// The linear map's variant where the ring has no widened term (RK4 always takes the
// widened map's code).
const void* coll_kernel(int scheme, bool gen)
{
    if (scheme == PHTL_EULER_CROMER) return coll_kernel_s<PHTL_EULER_CROMER>(gen);
    if (scheme == PHTL_LEAPFROG) return coll_kernel_s<PHTL_LEAPFROG>(gen);
    if (scheme == PHTL_RUTH4) return coll_kernel_s<PHTL_RUTH4>(gen);
    if (scheme == PHTL_RK4) return reinterpret_cast<const void*>(&k_coll_turn<PHTL_RK4, true>);
    return nullptr;
}

size_t coll_smem(int block, int ns)
{
    return static_cast<size_t>((ns + 1) / 2) * sizeof(double) + 2u * (block / 32) * 16 * sizeof(double);
}

}  // namespace

int occupancy_coll(int scheme, bool gen, int block, int nslices)
{
    const void* k = coll_kernel(scheme, gen);
    if (!k) return 0;
    const size_t sm = coll_smem(block, nslices);
    if (sm > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, sm) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_coll_turn(const LaunchDesc& L, const MapConsts& c, const CollArgs& A,
                             const double* U, unsigned* counts, uint16_t* slot, double* mon_rows,
                             int64_t rec_row, bool kick, bool map, cudaStream_t s)
{
    const void* k = coll_kernel(L.scheme, c.general != 0);
    if (!k) return cudaErrorInvalidValue;
    LaunchDesc Lc = L;
    MapConsts cc = c;
    CollArgs aa = A;
    const double* vv = U;
    unsigned* cn = counts;
    uint16_t* sl = slot;
    double* mr = mon_rows;
    int64_t rr = rec_row;
    int kk = kick ? 1 : 0, mm = map ? 1 : 0;
    void* args[] = {&Lc, &cc, &aa, &vv, &cn, &sl, &mr, &rr, &kk, &mm};
    return launch_pdl(k, dim3(L.grid), dim3(L.block), args, coll_smem(L.block, A.nslices), s);
}

cudaError_t launch_wake_potential(const unsigned* counts, const double* w, const CollArgs& A,
                                  double* V, double* U, float2* U2, unsigned* clear, cudaStream_t s)
{
    const int ns = A.nslices;
    const int block = 256;
    // one slice per warp, at most 152 blocks: few enough that staging the table in every
    // block stays cheap, enough to spread 4096 slices
    const int grid = std::min((ns + 7) / 8, 152);
    const size_t sm = 2u * static_cast<size_t>(ns) * sizeof(double);
    // above 48 KB (more than 3072 slices; 64 KB at most) the launch must opt in, on the
    // current device
    if (sm > 48u * 1024u &&
        cudaFuncSetAttribute(k_wake_potential, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sm)) != cudaSuccess)
        return cudaGetLastError();
    const unsigned* cc = counts;
    int nn = ns;
    double al = A.alpha, as = A.alpha_sc;
    void* args[] = {&cc, const_cast<double**>(&w), &nn, &al, &as, &V, &U, &U2, &clear};
    return launch_pdl(reinterpret_cast<const void*>(&k_wake_potential), dim3(grid), dim3(block),
                      args, sm, s);
}

}  // namespace phtl
