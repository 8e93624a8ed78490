// peds.cu -- per-step kernels of the pedestrian side (Sections 2.3-2.4):
//   hash_count  one thread per record of B: bin, slot, evacuee count (and
//               thread 0 applies completed sandbag layers to z first);
//   step_begin  the sandbag layers and bag snapshot alone, for a step whose
//               records the previous pedestrian step already hashed (only
//               where a barrier can be built);
//   scan        exclusive scan of the bin counts: per tile of 2048 bins the
//               sum of the tile counts before it (the hashing counted the
//               records of every tile) and the tile's own scan -> bin starts
//               (no waits); re-zeroes the bin counts; the exited bin's start
//               is the new count;
//   gather      moves each record of B to its bin's range in A; exited
//               records go to the by-id archive; re-zeroes the tile counts;
//   ped_step    eight lanes per record of A (peds_dev.cuh); the first warp
//               of block 0 then admits the step's visitors through the doors.
#include "peds_dev.cuh"

namespace {
using namespace fpdev;


__global__ void hash_count_kernel(const __grid_constant__ FpSim S, int par) {
    fp_pdl_trigger();  // the scan may be scheduled now; it waits for this grid's end
    FpCounters *C = S.cnt;
    if (blockIdx.x == 0 && threadIdx.x == 0) barrier_and_snapshot(S);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.cap) return;
    const uint4 pa = S.pedB[2 * i], pb = S.pedB[2 * i + 1];  // loaded beside the count
    if (i >= C->nB) return;
    hash_record(S, i, __uint_as_float(pa.x), __uint_as_float(pa.y), pb.y, S.occ[par]);
}

// The opening of a step whose records of B the previous pedestrian step hashed
// as it wrote them: completed sandbag layers and the bag snapshot.
__global__ void step_begin_kernel(const __grid_constant__ FpSim S) {
    fp_pdl_trigger();  // the scan may be scheduled now; it waits for this grid's end
    barrier_and_snapshot(S);
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(const __grid_constant__ FpSim S) {
    fp_pdl_wait();     // the step's opening kernel (the counts)
    fp_pdl_trigger();  // the gather may be scheduled now; it waits for this grid's end
    scan_tile(S, blockIdx.x);
}

__global__ void gather_kernel(const __grid_constant__ FpSim S, int slot) {
    // The record, its key and slot, the record count and the step index come
    // from kernels that finished before the scan began: loaded, and the
    // record's draws computed, before waiting for the scan (the arrays hold
    // cap entries; the count is checked after).
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = i < S.cap;
    const int nB = S.cnt->nB;
    const long long step = S.clock[slot].step;
    int key = 0, bslot = 0;
    uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a;
    if (in) {
        key = S.pkey[i];
        bslot = S.pslot[i];
        a = S.pedB[2 * i];
        b = S.pedB[2 * i + 1];
    }
    const float2 xi = fp_step_draws(S, b.x, step);
    fp_pdl_wait();
    fp_pdl_trigger();
    // the scan has read the tile counts: clear them for the next hashing
    for (int t = i; t < fp_scan_tiles_dev(S.nbins); t += gridDim.x * blockDim.x) S.tile_sum[t] = 0;
    if (!in || i >= nB) return;
    gather_place(S, key, bslot, a, b, xi);
}

struct DirectLookup {
    const int *start;
    __device__ int operator()(int key) const { return start[key]; }
};

// hash_next: also hash the output records for the next step (bins and the
// evacuee counts of the other parity), so that step needs no hash_count pass
template <int kG>
__global__ void __launch_bounds__(256) ped_step_kernel(const __grid_constant__ FpSim S, int par, int slot,
                                                       int hash_next) {
    FpCounters *C = S.cnt;
    // the clock and the bag snapshot come from kernels that finished before
    // the scan began: read (and the time step computed) by every thread before
    // waiting for the gather -- the same addresses, so one transaction per warp
    // and no block barrier; the record count is the scan's
    StepCtl ctl;
    load_step_ctl(S, slot, 0, ctl);
    fp_pdl_wait();
    fp_pdl_trigger();  // the next step's scan may be scheduled; it waits for this grid's end
    ctl.nA = min(C->nA, S.cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        C->nB = ctl.nA;
        if (ctl.dt_ticks > 0) C->ped_updates += (unsigned long long)ctl.nA;
    }
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    ped_group<kG>(S, par, ctl, gt / kG, threadIdx.x & (kG - 1), DirectLookup{S.bin_start}, hash_next != 0);
    if (blockIdx.x == 0 && threadIdx.x < 32) door_entries(S, par, ctl, hash_next != 0);
}

// New records sit in B at [first_slot, first_slot + count): give them ids
// first_id.. in order, clear their hazard/exit bytes, check they stand in a
// walkable cell, and seed the by-id archive.
__global__ void assign_ids_kernel(const __grid_constant__ FpSim S, int first_slot, int first_id, int count) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {  // the host puts both back if a record is rejected
        S.cnt->nB = first_slot + count;
        S.cnt->n_ids = first_id + count;
    }
    if (k >= count) return;
    const int i = first_slot + k;
    const int id = first_id + k;
    uint4 a = S.pedB[2 * i], b = S.pedB[2 * i + 1];
    b.x = (unsigned)id;
    // responders: tasks 0..4; evacuees: 0, or a visitor bound for door task - 8
    const unsigned role = FP_META_ROLE(b.y) ? 1u : 0u, task = FP_META_TASK(b.y);
    const bool task_ok = role ? task <= 4u : (task == 0u || (task >= FP_TASK_VISIT0 && task < FP_TASK_VISIT0 + FP_MAX_DOORS));
    b.y = FP_META(role, task_ok ? task : 0u, 0, 0);
    if (!walkable_at(S, __uint_as_float(a.x), __uint_as_float(a.y))) atomicAdd(&S.cnt->bad_ped, 1);
    S.pedB[2 * i + 1] = b;
    S.arch[2 * (size_t)id] = a;
    S.arch[2 * (size_t)id + 1] = b;
}

__global__ void read_arch_kernel(const __grid_constant__ FpSim S, uint4 *out, int n_total) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_total) return;
    out[2 * i] = S.arch[2 * (size_t)i];
    out[2 * i + 1] = S.arch[2 * (size_t)i + 1];
}

__global__ void read_live_kernel(const __grid_constant__ FpSim S, uint4 *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.cnt->nB) return;
    const uint4 a = S.pedB[2 * i], b = S.pedB[2 * i + 1];
    out[2 * (size_t)b.x] = a;
    out[2 * (size_t)b.x + 1] = b;
}

inline int blocks_for(int n, int t) { return n <= 0 ? 1 : (n + t - 1) / t; }

// ---- batched ensemble: one launch covers every member of a batch ------------
// Flat record space: member s owns [rec_off[s], rec_off[s+1]), a multiple of 256
// records long, so every CTA belongs to one member.


__global__ void hash_count_batch_kernel(const FpSim *__restrict__ sims, const int *__restrict__ rec_off, int n,
                                        int par) {
    const int s = batch_member(rec_off, n, blockIdx.x * blockDim.x);
    const FpSim &S = sims[s];
    FpCounters *C = S.cnt;
    const int i = blockIdx.x * blockDim.x + threadIdx.x - rec_off[s];
    if (i == 0) barrier_and_snapshot(S);
    if (i >= C->nB) return;
    const uint4 pa = S.pedB[2 * i], pb = S.pedB[2 * i + 1];
    hash_record(S, i, __uint_as_float(pa.x), __uint_as_float(pa.y), pb.y, S.occ[par]);
}

__global__ void __launch_bounds__(kScanThreads) scan_batch_kernel(const FpSim *__restrict__ sims) {
    const FpSim &S = sims[blockIdx.y];
    if ((int)blockIdx.x >= (S.nbins + 1 + kScanTile - 1) / kScanTile) return;
    scan_tile(S, blockIdx.x);
}

__global__ void gather_batch_kernel(const FpSim *__restrict__ sims, const int *__restrict__ rec_off, int n,
                                    int slot) {
    const int s = batch_member(rec_off, n, blockIdx.x * blockDim.x);
    const FpSim &S = sims[s];
    const int i = blockIdx.x * blockDim.x + threadIdx.x - rec_off[s];
    for (int t = i; t < fp_scan_tiles_dev(S.nbins); t += rec_off[s + 1] - rec_off[s]) S.tile_sum[t] = 0;
    if (i < S.cnt->nB) gather_record(S, i, S.clock[slot].step);
}

// The pedestrian update of the members of one lane group: G lanes per
// pedestrian, 256 / G pedestrians per block; member k of the group owns blocks
// [blk_off[k], blk_off[k + 1]).
template <int G>
__global__ void __launch_bounds__(256) ped_step_batch_kernel(const FpSim *__restrict__ sims,
                                                             const int *__restrict__ members,
                                                             const int *__restrict__ blk_off, int ng, int par,
                                                             int slot) {
    __shared__ StepCtl s_ctl;
    constexpr int kRecPerBlock = 256 / G;
    const int k = batch_member(blk_off, ng, blockIdx.x);
    const FpSim &S = sims[members[k]];
    const int j0 = ((int)blockIdx.x - blk_off[k]) * kRecPerBlock;
    if (threadIdx.x == 0) {
        FpCounters *C = S.cnt;
        load_step_ctl(S, slot, C->nA, s_ctl);
        if (j0 == 0) {
            C->nB = s_ctl.nA;
            if (s_ctl.dt_ticks > 0) C->ped_updates += (unsigned long long)s_ctl.nA;
        }
    }
    __syncthreads();
    const StepCtl ctl = s_ctl;
    ped_group<G>(S, par, ctl, j0 + threadIdx.x / G, threadIdx.x & (G - 1), DirectLookup{S.bin_start}, false);
    if (j0 == 0 && threadIdx.x < 32) door_entries(S, par, ctl, false);
}

}  // namespace

void fp_launch_batch_peds(const FpSim *d_sims, const int *d_rec_off, int n, int total_rec, int max_scan_tiles,
                          const FpBatchGroups &pg, int par, int slot, cudaStream_t st_hash, cudaStream_t st_chain,
                          cudaEvent_t fork, bool hash_part) {
    if (hash_part) {
        hash_count_batch_kernel<<<total_rec / 256, 256, 0, st_hash>>>(d_sims, d_rec_off, n, par);
        cudaEventRecord(fork, st_hash);
        return;
    }
    scan_batch_kernel<<<dim3(max_scan_tiles, n), kScanThreads, 0, st_chain>>>(d_sims);
    gather_batch_kernel<<<total_rec / 256, 256, 0, st_chain>>>(d_sims, d_rec_off, n, slot);
    // one launch per lane group that has members (the groups touch disjoint members)
    for (int g = 0; g < 5; ++g) {
        if (pg.n[g] == 0) continue;
        const dim3 grid(pg.total[g]);
        switch (kBatchPedLanes[g]) {
            case 1: ped_step_batch_kernel<1><<<grid, 256, 0, st_chain>>>(d_sims, pg.members[g], pg.off[g], pg.n[g], par, slot); break;
            case 2: ped_step_batch_kernel<2><<<grid, 256, 0, st_chain>>>(d_sims, pg.members[g], pg.off[g], pg.n[g], par, slot); break;
            case 4: ped_step_batch_kernel<4><<<grid, 256, 0, st_chain>>>(d_sims, pg.members[g], pg.off[g], pg.n[g], par, slot); break;
            case 8: ped_step_batch_kernel<8><<<grid, 256, 0, st_chain>>>(d_sims, pg.members[g], pg.off[g], pg.n[g], par, slot); break;
            default: ped_step_batch_kernel<16><<<grid, 256, 0, st_chain>>>(d_sims, pg.members[g], pg.off[g], pg.n[g], par, slot); break;
        }
    }
}

int fp_scan_tiles(int nbins) { return (nbins + 1 + kScanTile - 1) / kScanTile; }

void fp_launch_hash_count(const FpSim &S, int par, cudaStream_t st) {
    hash_count_kernel<<<blocks_for(S.cap, 256), 256, 0, st>>>(S, par);
}
void fp_launch_scan(const FpSim &S, cudaStream_t st, bool pdl) {
    fp_launch(pdl, scan_kernel, dim3(fp_scan_tiles(S.nbins)), dim3(kScanThreads), 0, st, S);
}
void fp_launch_gather(const FpSim &S, int slot, cudaStream_t st, bool pdl) {
    fp_launch(pdl, gather_kernel, dim3(blocks_for(S.cap, 256)), dim3(256), 0, st, S, slot);
}
void fp_launch_step_begin(const FpSim &S, cudaStream_t st) { step_begin_kernel<<<1, 1, 0, st>>>(S); }
void fp_launch_ped_step(const FpSim &S, int par, int slot, int lanes, cudaStream_t st, bool pdl, bool hash_next) {
    const int hn = hash_next ? 1 : 0;
    if (lanes == 1)
        fp_launch(pdl, ped_step_kernel<1>, dim3(blocks_for(S.cap, 256)), dim3(256), 0, st, S, par, slot, hn);
    else if (lanes == 2)
        fp_launch(pdl, ped_step_kernel<2>, dim3(blocks_for(S.cap * 2, 256)), dim3(256), 0, st, S, par, slot, hn);
    else if (lanes == 4)
        fp_launch(pdl, ped_step_kernel<4>, dim3(blocks_for(S.cap * 4, 256)), dim3(256), 0, st, S, par, slot, hn);
    else if (lanes == 16)
        fp_launch(pdl, ped_step_kernel<16>, dim3(blocks_for(S.cap * 16, 256)), dim3(256), 0, st, S, par, slot, hn);
    else fp_launch(pdl, ped_step_kernel<8>, dim3(blocks_for(S.cap * 8, 256)), dim3(256), 0, st, S, par, slot, hn);
}
// Every pedestrian removed: record counts, bag and exit totals, histogram.
__global__ void clear_peds_kernel(const __grid_constant__ FpSim S) {
    FpCounters *C = S.cnt;
    C->nA = 0;
    C->nB = 0;
    C->total_bags = 0ull;
    C->bags_snap = 0ull;
    C->applied = 0ull;
    C->n_exited = 0ull;
    C->n_ids = 0;
    C->n_entered = 0ull;
    C->n_left = 0ull;
    for (int k = 0; k < 5; ++k) C->hist[k] = 0ull;
}

void fp_launch_clear_peds(const FpSim &S, cudaStream_t st) { clear_peds_kernel<<<1, 1, 0, st>>>(S); }

void fp_launch_assign_ids(const FpSim &S, int first_slot, int first_id, int count, cudaStream_t st) {
    if (count > 0) assign_ids_kernel<<<blocks_for(count, 256), 256, 0, st>>>(S, first_slot, first_id, count);
}
void fp_launch_read_peds(const FpSim &S, uint4 *out, int n_total, cudaStream_t st) {
    if (n_total <= 0) return;
    read_arch_kernel<<<blocks_for(n_total, 256), 256, 0, st>>>(S, out, n_total);
    read_live_kernel<<<blocks_for(S.cap, 256), 256, 0, st>>>(S, out);
}
