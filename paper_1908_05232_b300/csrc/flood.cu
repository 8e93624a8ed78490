// flood.cu -- per-step kernels of the hydrodynamic update (Section 2.2): the
// flood kernel (one warp per run of 64 columns x TY rows, see flood_dev.cuh),
// its batched-ensemble form, the clock initialisation after a state change,
// the FP64 water-volume reduction and the largest hazard rating.
#include "flood_dev.cuh"

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

namespace {
using namespace fpdev;

constexpr int kFloodWarps = 8;  // warps per CTA of the flood kernels

// Batched ensemble, the members of one run-height group: a flat space of
// 64 x TY runs, member k of the group owning runs [run_off[k], run_off[k + 1]);
// one warp per run, each warp folding its own tallies into its member's clock.
template <int TY>
__global__ void __launch_bounds__(32 * kFloodWarps, 2) flood_batch_kernel(const FpSim *__restrict__ sims,
                                                                       const int *__restrict__ members,
                                                                       const int *__restrict__ run_off, int ng,
                                                                       int total_runs, int par, int slot) {
    const int r = blockIdx.x * kFloodWarps + (threadIdx.x >> 5);
    if (r >= total_runs) return;  // whole warps
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (run_off[mid] <= r) lo = mid; else hi = mid - 1;
    }
    const FpSim &S = sims[members[lo]];
    const int lr = r - run_off[lo];
    const FloodStep st = flood_step_consts(S, slot);
    if (lr == 0 && (threadIdx.x & 31) == 0) flood_clock_advance(S, slot, st);
    FloodAcc acc = flood_acc_init();
    flood_run<TY>(S, par, st, lr, acc);
    flood_acc_fold_warp(S, slot, acc);
}

// Runs of TY rows handed out one at a time from a ticket to whichever warp is
// free (at most two CTAs per SM are launched, each warp looping): a run whose
// groups stay dry costs a ticket and a flag test, a wet run a march of TY
// rows, so where only part of the grid holds water every wet run still
// starts at once, spread over all resident warps, instead of waiting behind
// a static share of dry ones.  Each warp reads the step's constants and folds
// its own tallies (no barrier: warps of a CTA finish apart); the first warp
// advances the clock.  Every warp takes exactly one ticket past the last run;
// the warp that takes the very last one resets the counter for the next
// launch (no other warp touches it after that).
template <int TY>
__global__ void __launch_bounds__(32 * kFloodWarps, 2) flood_kernel(const __grid_constant__ FpSim S, int par,
                                                                 int slot) {
    fp_pdl_wait();
    const FloodStep st = flood_step_consts(S, slot);
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) flood_clock_advance(S, slot, st);
    const unsigned nruns = (unsigned)(((S.nx + FP_TX - 1) / FP_TX) * ((S.ny + TY - 1) / TY));
    const unsigned last = nruns + gridDim.x * kFloodWarps - 1u;
    unsigned *ticket = &S.cnt->flood_ticket;
    FloodAcc acc = flood_acc_init();
    for (;;) {
        unsigned r = 0u;
        if (lane == 0) r = atomicAdd(ticket, 1u);
        r = __shfl_sync(0xffffffffu, r, 0);
        if (r >= nruns) {
            if (lane == 0 && r == last) *ticket = 0u;
            break;
        }
        flood_run<TY>(S, par, st, (int)r, acc);
    }
    flood_acc_fold_warp(S, slot, acc);
}

// U^0 wave-speed max and wet flag into clock slot `slot` (after a state change).
__global__ void init_clock_kernel(const __grid_constant__ FpSim S, int par, int slot) {
    float smax = 0.0f;
    int wet = 0;
    const long long n = (long long)S.nx * S.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % S.nx), j = (int)(c / S.nx);
        const size_t o = fp_pidx(S, i, j);
        const float h = S.h[par][o];
        if (h > FP_H_EPS_F) smax = fmaxf(smax, fp_wave_speed(S.g, h, S.hu[par][o], S.hv[par][o]));
        if (h >= FP_H_DRY_F) wet = 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        wet |= __shfl_xor_sync(0xffffffffu, wet, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (smax > 0.0f) atomicMax(&S.clock[slot].smax_bits, __float_as_uint(smax));
        if (wet) atomicOr(&S.clock[slot].wet, 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S.clock[slot].h_in = (float)fp_hydro_depth(S, S.clock[slot].t);
        S.clock[slot].q_speed = fp_discharge_speed(S, S.clock[slot].t);
    }
}

// Water volume sum h dx^2 in FP64: per-CTA partials, then the last CTA adds
// them (and the boundary inflow volumes) in index order -- deterministic.
__global__ void mass_kernel(const __grid_constant__ FpSim S, int par) {
    __shared__ double red[8];
    __shared__ bool last;
    double acc = 0.0;
    const long long n = (long long)S.nx * S.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % S.nx), j = (int)(c / S.nx);
        acc += (double)S.h[par][fp_pidx(S, i, j)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
        S.partials[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(&S.cnt->mass_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned k = 0; k < gridDim.x; ++k) s += ((volatile double *)S.partials)[k];
        const double dx = (double)S.dx;
        S.cnt->mass = s * dx * dx;
        double q = 0.0;
        for (int k = 0; k < 2 * S.nx + 2 * S.ny; ++k) q += S.bflux[k];
        S.cnt->inflow = q;
        S.cnt->mass_done = 0u;
    }
}

// Largest hazard rating HR = (max(|u|,|v|) + 0.5) h over the cells holding
// water (h > h_eps), FP32 with correctly rounded division (Section 2.4;
// Fig. 5(b) follows its time history).  Non-negative floats order as their
// bit patterns: one integer max per warp.
__global__ void hr_max_kernel(const __grid_constant__ FpSim S, int par) {
    unsigned best = 0u;
    const long long n = (long long)S.nx * S.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % S.nx), j = (int)(c / S.nx);
        const size_t o = fp_pidx(S, i, j);
        const float h = S.h[par][o];
        if (!(h > FP_H_EPS_F)) continue;
        const float V = __fdiv_rn(fmaxf(fabsf(S.hu[par][o]), fabsf(S.hv[par][o])), h);
        const float hr = __fmul_rn(__fadd_rn(V, 0.5f), h);
        best = max(best, __float_as_uint(hr));
    }
    best = __reduce_max_sync(0xffffffffu, best);
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&S.cnt->hr_max_bits, best);
}

}  // namespace

void fp_launch_hr_max(const FpSim &S, int par, cudaStream_t st) {
    cudaMemsetAsync(&S.cnt->hr_max_bits, 0, sizeof(unsigned), st);
    hr_max_kernel<<<148 * 4, 256, 0, st>>>(S, par);
}

void fp_launch_flood_batch(const FpSim *d_sims, const FpBatchGroups &fg, int par, int slot, cudaStream_t st) {
    // one launch per run-height group that has members (disjoint members)
    for (int g = 0; g < 3; ++g) {
        if (fg.n[g] == 0) continue;
        const int grid = (fg.total[g] + kFloodWarps - 1) / kFloodWarps;
        switch (kBatchFloodRows[g]) {
            case 8: flood_batch_kernel<8><<<grid, 32 * kFloodWarps, 0, st>>>(d_sims, fg.members[g], fg.off[g], fg.n[g], fg.total[g], par, slot); break;
            case 32: flood_batch_kernel<32><<<grid, 32 * kFloodWarps, 0, st>>>(d_sims, fg.members[g], fg.off[g], fg.n[g], fg.total[g], par, slot); break;
            default: flood_batch_kernel<16><<<grid, 32 * kFloodWarps, 0, st>>>(d_sims, fg.members[g], fg.off[g], fg.n[g], fg.total[g], par, slot); break;
        }
    }
}

cudaError_t fp_flood_init_attributes() { return cudaSuccess; }

// SMs of the current device, cached per device.
static int device_sms() {
    static std::mutex mu;
    static std::vector<std::pair<int, int>> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &e : cache)
        if (e.first == dev) return e.second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    cache.emplace_back(dev, sms);
    return sms;
}

// At most two CTAs per SM (the kernel's register budget), fewer for small grids.
template <int TY>
static void launch_flood_t(const FpSim &S, int par, int slot, cudaStream_t st, bool pdl) {
    const int nruns = ((S.nx + FP_TX - 1) / FP_TX) * ((S.ny + TY - 1) / TY);
    const int grid = std::min((nruns + kFloodWarps - 1) / kFloodWarps, 2 * device_sms());
    fp_launch(pdl, flood_kernel<TY>, dim3(grid), dim3(32 * kFloodWarps), 0, st, S, par, slot);
}

void fp_launch_flood(const FpSim &S, int par, int slot, int tile_rows, cudaStream_t st, bool pdl) {
    if (tile_rows == 8) launch_flood_t<8>(S, par, slot, st, pdl);
    else if (tile_rows == 32) launch_flood_t<32>(S, par, slot, st, pdl);
    else launch_flood_t<16>(S, par, slot, st, pdl);
}

void fp_launch_init_clock(const FpSim &S, int par, int slot, cudaStream_t st) {
    const long long n = (long long)S.nx * S.ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 148 * 8) blocks = 148 * 8;
    if (blocks < 1) blocks = 1;
    init_clock_kernel<<<blocks, 256, 0, st>>>(S, par, slot);
}

void fp_launch_mass(const FpSim &S, int par, cudaStream_t st) {
    const long long n = (long long)S.nx * S.ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 148 * 4) blocks = 148 * 4;
    if (blocks < 1) blocks = 1;
    mass_kernel<<<blocks, 256, 0, st>>>(S, par);
}
