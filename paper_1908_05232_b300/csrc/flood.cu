// flood.cu -- per-step kernels of the hydrodynamic update (Section 2.2): the
// flood kernel (CTAs resident on every SM, each taking a strided list of 64 x TY
// tiles, see flood_dev.cuh), its batched-ensemble form, the clock
// initialisation after a state change, and the FP64 water-volume reduction.
#include "flood_dev.cuh"

namespace {
using namespace fpdev;

// Batched ensemble: flat tile space, member s owns tiles [tile_off[s], tile_off[s+1]);
// one tile per CTA.
__global__ void __launch_bounds__(512, 2) flood_batch_kernel(const FpSim *__restrict__ sims,
                                                          const FpTmaSet *__restrict__ maps,
                                                          const int *__restrict__ tile_off, int n, int par,
                                                          int slot) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mbar[2];
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0]);
        mbar_init(&mbar[1]);
    }
    __syncthreads();
    const int t = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const FpSim &S = sims[lo];
    const int ntiles = tile_off[lo + 1] - tile_off[lo];
    unsigned phase = 0u;
    flood_tiles<16>(maps[2 * lo + par], S, par, slot, t - tile_off[lo], ntiles, ntiles, smem_raw, mbar, phase, false);
}

// One CTA per SM slot, each taking every gridDim.x-th tile.
template <int TY>
__global__ void __launch_bounds__(32 * TY, 32 / TY) flood_kernel(const __grid_constant__ FpTmaSet tm,
                                                                 const __grid_constant__ FpSim S, int par, int slot) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mbar[2];
    fp_pdl_wait();
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0]);
        mbar_init(&mbar[1]);
    }
    __syncthreads();
    const int ntiles = ((S.nx + FP_TX - 1) / FP_TX) * ((S.ny + TY - 1) / TY);
    unsigned phase = 0u;
    flood_tiles<TY>(tm, S, par, slot, blockIdx.x, gridDim.x, ntiles, smem_raw, mbar, phase, true);
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

int fp_flood_smem_bytes(int tile_rows) {
    if (tile_rows == 8) return smem_bytes<8>();
    if (tile_rows == 32) return smem_bytes<32>();
    return smem_bytes<16>();
}

void fp_launch_flood_batch(const FpSim *d_sims, const FpTmaSet *d_maps, const int *d_tile_off, int n,
                           int total_tiles, int par, int slot, cudaStream_t st) {
    flood_batch_kernel<<<total_tiles, 512, smem_bytes<16>(), st>>>(d_sims, d_maps, d_tile_off, n, par, slot);
}

// resident flood CTAs of each tile height on the whole GPU (set with the
// attributes), and the SM count
static int g_flood_ctas[3] = {0, 0, 0};
static int g_sms = 0;

template <int TY>
static cudaError_t init_flood_t(int sms) {
    cudaError_t e = cudaFuncSetAttribute(flood_kernel<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<TY>());
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, flood_kernel<TY>, 32 * TY, smem_bytes<TY>());
    g_flood_ctas[TY == 8 ? 0 : TY == 16 ? 1 : 2] = (per_sm > 0 ? per_sm : 1) * sms;
    return e;
}

cudaError_t fp_flood_init_attributes() {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_sms = sms;
    if (e == cudaSuccess) e = init_flood_t<8>(sms);
    if (e == cudaSuccess) e = init_flood_t<16>(sms);
    if (e == cudaSuccess) e = init_flood_t<32>(sms);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(flood_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<16>());
    return e;
}

template <int TY>
static void launch_flood_t(const FpSim &S, const FpTmaSet &tm, int par, int slot, cudaStream_t st, bool pdl) {
    constexpr int smem = smem_bytes<TY>();
    const int ntiles = ((S.nx + FP_TX - 1) / FP_TX) * ((S.ny + TY - 1) / TY);
    const int resident = g_flood_ctas[TY == 8 ? 0 : TY == 16 ? 1 : 2];
    int grid = resident > 0 && resident < ntiles ? resident : ntiles;
    // When every tile fits in one resident wave, at most half the resident CTAs
    // (never fewer than one per SM), each taking up to two tiles in turn: the
    // rest of each SM stays free for the pedestrian kernels that run beside
    // this one (a 512 x 512 step: 3 % faster; larger grids keep every CTA).
    if (resident > 0 && ntiles <= resident) {
        const int half = resident / 2 > g_sms ? resident / 2 : g_sms;
        if (grid > half) grid = half;
    }
    fp_launch(pdl, flood_kernel<TY>, dim3(grid), dim3(32 * TY), smem, st, tm, S, par, slot);
}

void fp_launch_flood(const FpSim &S, const void *tma_set, int par, int slot, int tile_rows, cudaStream_t st,
                     bool pdl) {
    const FpTmaSet &tm = *static_cast<const FpTmaSet *>(tma_set);
    if (tile_rows == 8) launch_flood_t<8>(S, tm, par, slot, st, pdl);
    else if (tile_rows == 32) launch_flood_t<32>(S, tm, par, slot, st, pdl);
    else launch_flood_t<16>(S, tm, par, slot, st, pdl);
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
