// persist.cu -- persistent coupled-step kernel: many steps of the whole coupled
// update in one cooperative launch (every CTA resident), the phases of a step
// separated by grid barriers with bounded waits.
//
// Launch start:  H   hash every record of B (bin, slot, evacuee counts).
// Each step:     S1  CTA 0 applies completed sandbag layers to z and snapshots
//                    the bag count; every CTA scans its contiguous chunk of
//                    bin counts (local exclusive starts), re-zeroes them and
//                    publishes the chunk total;
//                --- grid barrier ---
//                G   every CTA forms the prefix of the chunk totals in shared
//                    memory (bin start = chunk prefix + local start) and
//                    gathers its share of B into bin order A;
//                --- grid barrier ---
//                FP  flood runs (flood_dev.cuh), one warp per run, then
//                    pedestrian chunks of eight lanes per pedestrian
//                    (peds_dev.cuh) taken by whichever CTAs are free; each
//                    output record is hashed at once for the next step into
//                    the other parity's evacuee-count plane;
//                --- grid barrier ---
// The last step does not hash its output, so a launch ends with the same
// invariants as the per-step kernels (bin counts and evacuee counts zero).
#include <algorithm>
#include <mutex>
#include <vector>

#include "flood_dev.cuh"
#include "grid_sync.cuh"
#include "peds_dev.cuh"

namespace {
using namespace fpdev;

constexpr int kPT = 512;       // threads per CTA
constexpr int kPTY = 8;        // flood run height
constexpr int kPLanes = 1;     // lanes per pedestrian
constexpr int kMaxCTAs = 2048;


// exclusive scan of one value per thread over the CTA (kPT threads); returns
// the thread's prefix, total in *total
__device__ __forceinline__ int block_exclusive_scan(int v, int *total) {
    __shared__ int s_w[kPT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    int pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kPT / 32; ++w) {
        pre += w < wid ? s_w[w] : 0;
        tot += s_w[w];
    }
    __syncthreads();
    *total = tot;
    return pre + incl - v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// CTA 0 stamps the global timer after a phase (profiling only)
__device__ __forceinline__ void stamp(const FpSim &S, int idx) {
    if (S.phase_ts != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && idx < 4 * S.phase_ts_steps + 1)
        S.phase_ts[idx] = global_ns();
}

struct ChunkLookup {
    const int *local;  // chunk-local starts
    const int *base;   // shared: prefix of chunk totals
    int chunk;
    __device__ int operator()(int key) const { return base[key / chunk] + local[key]; }
};

__global__ void __launch_bounds__(kPT, 1) persistent_kernel(const __grid_constant__ FpSim S, int par0, int slot0,
                                                            int nsteps, unsigned *bar) {
    __shared__ int s_base[kMaxCTAs];
    __shared__ FloodStep s_fst;
    __shared__ StepCtl s_ctl;
    __shared__ int s_pcx;
    FpCounters *C = S.cnt;
    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
    const int nbin1 = S.nbins + 1;
    const int chunk = (nbin1 + G - 1) / G;
    const int nruns = ((S.nx + FP_TX - 1) / FP_TX) * ((S.ny + kPTY - 1) / kPTY);

    // H: hash the current records of B
    {
        const int nB = C->nB;
        for (int i = cta * kPT + tid; i < nB; i += G * kPT) {
            const uint4 pa = S.pedB[2 * i], pb = S.pedB[2 * i + 1];
            hash_record(S, i, __uint_as_float(pa.x), __uint_as_float(pa.y), pb.y, S.occ[par0]);
        }
    }
    if (!grid_sync(bar, S)) return;
    stamp(S, 0);

    for (int s = 0; s < nsteps; ++s) {
        const int par = par0 ^ (s & 1), slot = (slot0 + s) & 3;
        // S1: sandbag layers + bag snapshot; chunk-local scan of the bin counts
        if (cta == 0 && tid == 0) {
            barrier_and_snapshot(S);
            bar[2 + ((s + 1) & 1)] = 0u;  // the next step's pedestrian ticket (unused since the last barrier)
        }
        {
            const int lo = cta * chunk, hi = min(lo + chunk, nbin1);
            int running = 0;
            for (int base = lo; base < hi; base += kPT * 4) {
                int v[4], sum = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int idx = base + tid * 4 + k;
                    v[k] = idx < hi ? S.bin_count[idx] : 0;
                    sum += v[k];
                }
                int total;
                int run = running + block_exclusive_scan(sum, &total);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int idx = base + tid * 4 + k;
                    if (idx < hi) {
                        S.bin_start[idx] = run;
                        S.bin_count[idx] = 0;
                    }
                    run += v[k];
                }
                running += total;
            }
            if (tid == 0) S.scan_part[cta] = running;
        }
        if (!grid_sync(bar, S)) return;
        stamp(S, 4 * s + 1);

        // G: bin starts, gather B -> A
        {
            int total;
            for (int c0 = 0; c0 < G; c0 += kPT) {
                const int c = c0 + tid;
                const int v = c < G ? S.scan_part[c] : 0;
                const int pre = block_exclusive_scan(v, &total);
                const int carry = c0 == 0 ? 0 : s_base[c0 - 1] + S.scan_part[c0 - 1];
                if (c < G) s_base[c] = carry + pre;
                __syncthreads();
            }
        }
        const ChunkLookup lookup{S.bin_start, s_base, chunk};
        const int nA = lookup(S.nbins);
        // this kernel's scan does not read the hashing's tile counts: keep them
        // at zero for the per-step kernels' scan of a later step
        for (int t = cta * kPT + tid; t < fp_scan_tiles_dev(S.nbins); t += G * kPT) S.tile_sum[t] = 0;
        {
            const int nB = C->nB;
            for (int i = cta * kPT + tid; i < nB; i += G * kPT) {
                const int key = S.pkey[i];
                const uint4 a = S.pedB[2 * i], b = S.pedB[2 * i + 1];
                if (key == S.nbins) {
                    S.arch[2 * (size_t)b.x] = a;
                    S.arch[2 * (size_t)b.x + 1] = b;
                } else {
                    const int dst = lookup(key) + S.pslot[i];
                    if ((unsigned)dst >= (unsigned)S.cap) {  // counts out of step with the records
                        fp_set_err(S, FP_ERR_BAD_PED);
                        continue;
                    }
                    S.pedA[2 * dst] = a;
                    S.pedA[2 * dst + 1] = b;
                    S.posA[dst] = make_float2(__uint_as_float(a.x), __uint_as_float(a.y));
                    S.xiA[dst] = fp_step_draws(S, b.x, S.clock[slot].step);
                }
            }
        }
        if (!grid_sync(bar, S)) return;
        stamp(S, 4 * s + 2);
        // FP: flood runs (warp w of CTA c takes runs c * 16 + w, + 16 G, ...),
        // then pedestrian chunks taken from a ticket counter by whichever CTAs
        // are free (those whose runs were skipped as dry come first) -- both
        // read the state at step n; pedestrian outputs are hashed for the next
        // step (not after the last), into the other parity's evacuee-count plane.
        if (tid == 0) {
            load_step_ctl(S, slot, nA, s_ctl);
            const FloodStep fst = flood_step_consts(S, slot);
            s_fst = fst;
            if (cta == 0) {
                C->nA = nA;
                C->nB = nA;
                if (s_ctl.dt_ticks > 0) C->ped_updates += (unsigned long long)nA;
                flood_clock_advance(S, slot, fst);
            }
        }
        __syncthreads();
        {
            const FloodStep fst = s_fst;
            FloodAcc acc = flood_acc_init();
            for (int r = cta * (kPT / 32) + (tid >> 5); r < nruns; r += G * (kPT / 32))
                flood_run<kPTY>(S, par, fst, r, acc);
            flood_acc_fold_cta<kPT / 32>(S, slot, acc);
        }
        const StepCtl ctl = s_ctl;
        const bool hash_next = s + 1 < nsteps;
        constexpr int kPedPerCTA = kPT / kPLanes;
        unsigned *ticket = bar + 2 + (s & 1);  // zeroed during the previous step (or before the launch)
        for (;;) {
            if (tid == 0) s_pcx = (int)atomicAdd(ticket, 1u);
            __syncthreads();
            const int pcx = s_pcx;
            __syncthreads();
            if (pcx * kPedPerCTA >= nA) break;
            ped_group<kPLanes>(S, par, ctl, pcx * kPedPerCTA + tid / kPLanes, tid & (kPLanes - 1), lookup, hash_next);
        }
        if (cta == 0 && tid < 32) door_entries(S, par, ctl, hash_next);  // thread 0 set nB = nA above
        if (!grid_sync(bar, S)) return;
        stamp(S, 4 * s + 4);
    }
}

}  // namespace

// CTAs of the cooperative launch on the current device (0: no cooperative
// launch), cached per device.
int fp_persistent_ctas() {
    struct Entry {
        int dev, ctas;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry &e : cache)
        if (e.dev == dev) return e.ctas;
    int g = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel, kPT, 0) == cudaSuccess)
        g = std::min(sms * per_sm, kMaxCTAs);
    cache.push_back(Entry{dev, g});
    return g;
}

cudaError_t fp_launch_persistent(const FpSim &S, int par, int slot, int nsteps, unsigned *bar, int ctas,
                                 cudaStream_t st) {
    FpSim s = S;
    void *args[] = {(void *)&s, (void *)&par, (void *)&slot, (void *)&nsteps, (void *)&bar};
    // the barrier word and the pedestrian tickets start at zero (a barrier that
    // timed out leaves its word partly counted)
    const cudaError_t e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void *)persistent_kernel, dim3(ctas), dim3(kPT), args, 0, st);
}
