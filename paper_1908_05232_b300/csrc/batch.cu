// batch.cu -- the batched ensemble in one persistent launch: up to 256 coupled
// steps of every member per cooperative launch (every CTA resident), the
// phases of a step separated by bounded grid barriers.  Each member gets the
// work the per-step batch kernels give it, in the same order of the same
// device functions, so its bytes are those of stepping it alone.
//
// Each step:  H   every member's records of B hashed (bin, slot, tile count,
//                 evacuee count); the thread of a member's first record
//                 applies its completed sandbag layers and snapshots its bags;
//             --- grid barrier ---
//             S   the bin scan of every (member, tile) pair;
//             --- grid barrier ---
//             G   every member's records gathered into bin order A with the
//                 step's draws; the tile counts cleared;
//             --- grid barrier ---
//             FP  the flood runs of all members (one warp per run, from a
//                 ticket; the warp of a member's first run advances its
//                 clock), then pedestrian
//                 chunks of all members taken from a ticket by whichever CTAs
//                 are free (the chunk of a member's first record also admits
//                 its visitors through the doors);
//             --- grid barrier ---
// Flat spaces over all members: member m owns runs [run_off[m], run_off[m+1])
// (64 x kBatchPersistRows each) and records [rec_off[m], rec_off[m+1]), the
// latter a multiple of 256 long, so every 256 consecutive records (and every
// pedestrian chunk of 256 / kBatchPersistLanes) belong to one member.  Barrier bookkeeping (poll limit,
// error word) is member 0's.
#include <algorithm>
#include <mutex>
#include <vector>

#include "flood_dev.cuh"
#include "grid_sync.cuh"
#include "peds_dev.cuh"

namespace {
using namespace fpdev;

constexpr int kBT = 256;       // threads per CTA
constexpr int kMaxBatchCTAs = 4096;

struct DirectLookup {
    const int *start;
    __device__ int operator()(int key) const { return start[key]; }
};

__global__ void __launch_bounds__(kBT, 2) batch_persistent_kernel(const FpSim *__restrict__ sims,
                                                                  const int *__restrict__ run_off,
                                                                  const int *__restrict__ rec_off, int n,
                                                                  int total_runs, int total_rec, int max_tiles,
                                                                  int par0, int slot0, int nsteps, unsigned *bar) {
    __shared__ StepCtl s_ctl;
    __shared__ int s_pcx;
    const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const FpSim &S0 = sims[0];
    for (int s = 0; s < nsteps; ++s) {
        const int par = par0 ^ (s & 1), slot = (slot0 + s) & 3;
        // H: hash every member's records of B
        if (cta == 0 && tid == 0) {  // this step's tickets (last used two steps ago)
            bar[2 + (s & 1)] = 0u;
            bar[4 + (s & 1)] = 0u;
        }
        for (int x0 = cta * kBT; x0 < total_rec; x0 += G * kBT) {
            const int m = batch_member(rec_off, n, x0);
            const FpSim &S = sims[m];
            const int i = x0 + tid - rec_off[m];
            if (i == 0) barrier_and_snapshot(S);
            if (i < S.cnt->nB) {
                const uint4 pa = S.pedB[2 * i], pb = S.pedB[2 * i + 1];
                hash_record(S, i, __uint_as_float(pa.x), __uint_as_float(pa.y), pb.y, S.occ[par]);
            }
        }
        if (!grid_sync(bar, S0)) return;
        // S: the bin scan of every (member, tile)
        for (int it = cta; it < n * max_tiles; it += G) {
            const int m = it / max_tiles, tile = it % max_tiles;
            const FpSim &S = sims[m];
            if (tile < fp_scan_tiles_dev(S.nbins)) scan_tile(S, tile);
        }
        if (!grid_sync(bar, S0)) return;
        // G: gather into bin order, clear the tile counts
        for (int x0 = cta * kBT; x0 < total_rec; x0 += G * kBT) {
            const int m = batch_member(rec_off, n, x0);
            const FpSim &S = sims[m];
            const int i = x0 + tid - rec_off[m];
            for (int t = i; t < fp_scan_tiles_dev(S.nbins); t += rec_off[m + 1] - rec_off[m]) S.tile_sum[t] = 0;
            if (i < S.cnt->nB) gather_record(S, i, S.clock[slot].step);
        }
        if (!grid_sync(bar, S0)) return;
        // FP: flood runs, one warp per run, taken from a ticket (members' runs
        // cost very different amounts: dry groups are skipped)
        unsigned *fticket = bar + 4 + (s & 1);
        for (;;) {
            unsigned rr = 0u;
            if (lane == 0) rr = atomicAdd(fticket, 1u);
            const int r = (int)__shfl_sync(0xffffffffu, rr, 0);
            if (r >= total_runs) break;
            const int m = batch_member(run_off, n, r);
            const FpSim &S = sims[m];
            const int lr = r - run_off[m];
            const FloodStep st = flood_step_consts(S, slot);
            if (lr == 0 && lane == 0) flood_clock_advance(S, slot, st);
            FloodAcc acc = flood_acc_init();
            flood_run<kBatchPersistRows>(S, par, st, lr, acc);
            flood_acc_fold_warp(S, slot, acc);
        }
        // then pedestrian chunks (kBT / kBatchPersistLanes records each) from the ticket
        unsigned *ticket = bar + 2 + (s & 1);
        for (;;) {
            if (tid == 0) s_pcx = (int)atomicAdd(ticket, 1u);
            __syncthreads();
            const int x = s_pcx * (kBT / kBatchPersistLanes);
            if (x >= total_rec) break;  // block-uniform
            const int m = batch_member(rec_off, n, x);
            const FpSim &S = sims[m];
            const int j0 = x - rec_off[m];
            if (tid == 0) {
                FpCounters *C = S.cnt;
                load_step_ctl(S, slot, C->nA, s_ctl);
                if (j0 == 0) {
                    C->nB = s_ctl.nA;
                    if (s_ctl.dt_ticks > 0) C->ped_updates += (unsigned long long)s_ctl.nA;
                }
            }
            __syncthreads();
            const StepCtl ctl = s_ctl;
            ped_group<kBatchPersistLanes>(S, par, ctl, j0 + tid / kBatchPersistLanes, tid & (kBatchPersistLanes - 1),
                                          DirectLookup{S.bin_start}, false);
            if (j0 == 0 && tid < 32) door_entries(S, par, ctl, false);  // thread 0 set nB = nA above
            __syncthreads();  // s_ctl and s_pcx are taken again
        }
        if (!grid_sync(bar, S0)) return;
    }
}

}  // namespace

// CTAs of the batch's cooperative launch on the current device (0: no
// cooperative launch), cached per device.
int fp_batch_persistent_ctas() {
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
    if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel, kBT, 0) == cudaSuccess)
        g = std::min(sms * per_sm, kMaxBatchCTAs);
    cache.push_back(Entry{dev, g});
    return g;
}

cudaError_t fp_launch_batch_persistent(const FpSim *d_sims, const int *d_run_off, const int *d_rec_off, int n,
                                       int total_runs, int total_rec, int max_tiles, int par, int slot, int nsteps,
                                       unsigned *bar, int ctas, cudaStream_t st) {
    void *args[] = {(void *)&d_sims, (void *)&d_run_off, (void *)&d_rec_off, (void *)&n, (void *)&total_runs,
                    (void *)&total_rec, (void *)&max_tiles, (void *)&par, (void *)&slot, (void *)&nsteps,
                    (void *)&bar};
    // the barrier word and the tickets start at zero (a barrier that timed out
    // leaves its word partly counted)
    const cudaError_t e = cudaMemsetAsync(bar, 0, 8 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void *)batch_persistent_kernel, dim3(ctas), dim3(kBT), args, 0, st);
}
