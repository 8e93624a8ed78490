// peds.cu -- pedestrian side of the coupled step (Sections 2.3-2.4).
//
// Per step (after the previous step's pedestrian output B):
//   hash_count  one thread per record of B: hash bin (hk x hk cells, bin side
//               >= the 1 m neighbour radius) or the "exited" bin, slot in the
//               bin via an integer atomic, and the evacuee count of its cell
//               (uint16 lanes of the occupancy plane, N_p of Section 2.4).
//               Thread 0 applies completed sandbag layers to z first.
//   scan        single-pass exclusive scan of the bin counts (decoupled
//               look-back, tiles in ticket order, bounded waits) -> bin starts;
//               re-zeroes the counts; the exited bin's start is the new count.
//   gather      moves each record of B to its bin's range in A; exited
//               records go to the by-id archive.
//   ped_step    one thread per record of A: Table 1 state from the cell's
//               h, u, v at step n, responder task, navigation direction,
//               repulsion from neighbours in the 3 x 3 bins (accumulated in
//               64-bit fixed point, so the sum does not depend on the order
//               records sit in a bin), velocity relaxation and cap, move with
//               wall sliding, exit; writes B.
#include "fp_common.cuh"

namespace {

__constant__ float c_speed[5] = {0.0f, 1.8f, 0.9f, 0.45f, 0.0f};  // Table 1 (index 0: own dry speed)
constexpr float kTau = 0.5f, kA = 2.0f, kB = 0.3f, kRb = 0.25f, kR = 1.0f, kSide = 0.5f;
constexpr int kTPick = 30 * 1048576, kTDrop = 30 * 1048576;
constexpr float kBagT = 0.25f;
constexpr int kScanItems = 8, kScanThreads = 256, kScanTile = kScanItems * kScanThreads;
__constant__ int c_ox[8] = {1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int c_oy[8] = {0, 1, 0, -1, 1, 1, -1, -1};

enum { G_NONE = 0, G_EXIT = 1, G_DEPOT = 2, G_BARRIER = 3, G_STRAIGHT = 4 };

__device__ __forceinline__ bool walkable_at(const FpSim &S, float x, float y) {
    const int i = fp_cell_of(x, S.dx), j = fp_cell_of(y, S.dx);
    if (i < 0 || j < 0 || i >= S.nx || j >= S.ny) return false;
    return S.walk[(size_t)j * S.nx + i] != 0;
}

__global__ void hash_count_kernel(const __grid_constant__ FpSim S) {
    FpCounters *C = S.cnt;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (S.nb > 0 && S.n_layers > 0) {
            unsigned long long done = C->total_bags / (unsigned long long)S.bpc;
            const unsigned long long cap = (unsigned long long)S.nb * (unsigned long long)S.n_layers;
            if (done > cap) done = cap;
            for (unsigned long long k = C->applied; k < done; ++k) {
                const int c = S.barrier[k % (unsigned long long)S.nb];
                S.z[fp_pidx(S, c % S.nx, c / S.nx)] += kBagT;
            }
            C->applied = done;
        }
        C->bags_snap = C->total_bags;
        for (int k = 0; k < 5; ++k) C->hist[k] = 0ull;
        C->scan_epoch += 1u;
        C->scan_ticket = 0u;
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nB = C->nB;
    if (i >= nB) return;
    const uint4 pa = S.pedB[2 * i], pb = S.pedB[2 * i + 1];
    const unsigned meta = pb.y;
    int key = S.nbins;
    if (!FP_META_EXITED(meta)) {
        const int ci = fp_cell_of(__uint_as_float(pa.x), S.dx), cj = fp_cell_of(__uint_as_float(pa.y), S.dx);
        key = (cj / S.hk) * S.nbx + ci / S.hk;
        if (FP_META_ROLE(meta) == 0) {
            const size_t o = fp_pidx(S, ci, cj);
            const unsigned shift = (unsigned)(o & 1) * 16u;
            unsigned *w = reinterpret_cast<unsigned *>(S.occ + (o & ~(size_t)1));
            const unsigned old = atomicAdd(w, 1u << shift);
            if (((old >> shift) & 0xffffu) == 0xffffu) fp_set_err(S, FP_ERR_OCC_OVERFLOW);
        }
    }
    S.pkey[i] = key;
    S.pslot[i] = atomicAdd(&S.bin_count[key], 1);
}

// status word: epoch (30 bits) << 34 | status (1 aggregate, 2 inclusive prefix) << 32 | value
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const __grid_constant__ FpSim S) {
    __shared__ int s_tile, s_prefix;
    __shared__ int s_warp[kScanThreads / 32];
    const int tid = threadIdx.x;
    FpCounters *C = S.cnt;
    if (tid == 0) s_tile = (int)atomicAdd(&C->scan_ticket, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int n = S.nbins + 1;
    const unsigned long long epoch = (unsigned long long)(C->scan_epoch & 0x3fffffffu);
    const int base = tile * kScanTile + tid * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int idx = base + k;
        v[k] = idx < n ? S.bin_count[idx] : 0;
        sum += v[k];
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) S.bin_count[base + k] = 0;
    // block exclusive scan of the per-thread sums
    const int lane = tid & 31, wid = tid >> 5;
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    int wpre = 0, total = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < wid) wpre += s_warp[w];
        total += s_warp[w];
    }
    // warp-parallel decoupled look-back: lane l inspects predecessor tile - 1 - l
    // (and the window moves back by 32 while none of them has its inclusive prefix)
    if (wid == 0) {
        volatile unsigned long long *flags = S.scan_flags;
        int excl = 0;
        if (tile == 0) {
            if (lane == 0) flags[0] = (epoch << 34) | (2ull << 32) | (unsigned)total;
        } else {
            if (lane == 0) {
                flags[tile] = (epoch << 34) | (1ull << 32) | (unsigned)total;
                __threadfence();
            }
            __syncwarp();
            int t = tile - 1 - lane;
            bool timed_out = false;
            while (true) {
                unsigned long long w = 0;
                unsigned st = 2u;  // tiles before 0: an inclusive prefix of 0
                if (t >= 0) {
                    int it = 0;
                    for (; it < (1 << 22); ++it) {
                        w = flags[t];
                        st = (unsigned)(w >> 32) & 3u;
                        if ((w >> 34) == epoch && st != 0u) break;
                    }
                    if (it == (1 << 22)) { timed_out = true; w = 0; st = 2u; }
                }
                const int val = t >= 0 ? (int)(unsigned)(w & 0xffffffffull) : 0;
                const unsigned pmask = __ballot_sync(0xffffffffu, st == 2u);
                const int last = pmask ? __ffs(pmask) - 1 : 31;  // nearest predecessor with a prefix
                int part = lane <= last ? val : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                excl += part;
                if (pmask) break;
                t -= 32;
            }
            if (__any_sync(0xffffffffu, timed_out) && lane == 0) fp_set_err(S, FP_ERR_TIMEOUT);
            if (lane == 0) {
                __threadfence();
                flags[tile] = (epoch << 34) | (2ull << 32) | (unsigned)(excl + total);
            }
        }
        if (lane == 0) s_prefix = excl;
    }
    __syncthreads();
    int run = s_prefix + wpre + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int idx = base + k;
        if (idx < n) {
            S.bin_start[idx] = run;
            if (idx == n - 1) {
                S.bin_start[n] = run + v[k];
                C->nA = run;  // records before the exited bin
            }
        }
        run += v[k];
    }
}

__global__ void gather_kernel(const __grid_constant__ FpSim S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.cnt->nB) return;
    const int key = S.pkey[i];
    const uint4 a = S.pedB[2 * i], b = S.pedB[2 * i + 1];
    if (key == S.nbins) {
        S.arch[2 * (size_t)b.x] = a;
        S.arch[2 * (size_t)b.x + 1] = b;
    } else {
        const int dst = S.bin_start[key] + S.pslot[i];
        S.pedA[2 * dst] = a;
        S.pedA[2 * dst + 1] = b;
    }
}

__global__ void __launch_bounds__(256) ped_step_kernel(const __grid_constant__ FpSim S, int par, int slot) {
    __shared__ long long s_dt, s_step;
    __shared__ int s_wet;
    __shared__ unsigned long long s_bags;
    __shared__ int s_nA;
    FpCounters *C = S.cnt;
    if (threadIdx.x == 0) {
        const FpClock c = S.clock[slot];
        const float hin = (float)fp_hydro_depth(S, c.t);
        s_dt = fp_dt_ticks(S, c, hin);
        s_step = c.step;
        s_wet = c.wet;
        s_bags = C->bags_snap;
        s_nA = C->nA;
        if (blockIdx.x == 0) {
            C->nB = s_nA;
            if (s_dt > 0) C->ped_updates += (unsigned long long)s_nA;
        }
    }
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = j < s_nA;
    const long long dt_ticks = s_dt;
    int hr = 0;
    if (valid) {
        const uint4 pa = S.pedA[2 * j], pb = S.pedA[2 * j + 1];
        if (dt_ticks == 0) {
            S.pedB[2 * j] = pa;
            S.pedB[2 * j + 1] = pb;
        } else {
            const float dx = S.dx;
            const float dt = (float)dt_ticks * (1.0f / FP_TICKS_F);
            const float x = __uint_as_float(pa.x), y = __uint_as_float(pa.y);
            float vx = __uint_as_float(pa.z), vy = __uint_as_float(pa.w);
            const unsigned id = pb.x, meta = pb.y;
            int timer = (int)pb.z;
            const float v0 = __uint_as_float(pb.w);
            const int role = FP_META_ROLE(meta);
            int task = FP_META_TASK(meta);
            const int ci = fp_cell_of(x, dx), cj = fp_cell_of(y, dx);
            const int c = cj * S.nx + ci;
            const size_t pc = fp_pidx(S, ci, cj);
            hr = fp_hr_state(S.h[par][pc], S.hu[par][pc], S.hv[par][pc]);
            float speed = hr == 0 ? v0 : c_speed[hr];
            int goal = G_NONE, target = -1;
            if (role == 0) {
                goal = (S.evac_trigger == 0 || s_wet) ? G_EXIT : G_NONE;
            } else {
                const unsigned long long cap =
                    (unsigned long long)S.nb * (unsigned long long)S.n_layers * (unsigned long long)S.bpc;
                if (task != 4 && s_bags >= cap) task = 4;
                switch (task) {
                    case 4: goal = G_EXIT; break;
                    case 0:
                        if (S.nav[1][c] == FP_AT_GOAL) { task = 1; timer = kTPick; }
                        else goal = G_DEPOT;
                        break;
                    case 1:
                        timer = (int)(timer - dt_ticks);
                        if (timer <= 0) { task = 2; timer = 0; }
                        break;
                    case 2:
                        target = S.barrier[(s_bags / (unsigned long long)S.bpc) % (unsigned long long)S.nb];
                        if (c == target) { task = 3; timer = kTDrop; }
                        else if (S.nav[2][c] == FP_AT_GOAL) goal = G_STRAIGHT;
                        else goal = G_BARRIER;
                        break;
                    case 3:
                        timer = (int)(timer - dt_ticks);
                        if (timer <= 0) { atomicAdd(&C->total_bags, 1ull); task = 0; timer = 0; }
                        break;
                    default: break;
                }
                if (task == 1 || task == 3) speed = 0.0f;
            }
            // desired velocity
            float ex = 0.0f, ey = 0.0f, sdes = speed;
            if (goal != G_NONE) {
                float tx = 0.0f, ty = 0.0f;
                bool have = false, arriving = false;
                if (goal == G_STRAIGHT) {
                    tx = ((float)(target % S.nx) + 0.5f) * dx;
                    ty = ((float)(target / S.nx) + 0.5f) * dx;
                    have = arriving = true;
                } else {
                    const unsigned char *nav = S.nav[goal == G_EXIT ? 0 : goal == G_DEPOT ? 1 : 2];
                    const int code = nav[c];
                    if (code < 8) {
                        const int ti = ci + c_ox[code], tj = cj + c_oy[code];
                        tx = ((float)ti + 0.5f) * dx;
                        ty = ((float)tj + 0.5f) * dx;
                        have = true;
                        arriving = nav[tj * S.nx + ti] == FP_AT_GOAL;
                    }
                }
                if (have) {
                    const float ddx = tx - x, ddy = ty - y;
                    const float len = sqrtf(ddx * ddx + ddy * ddy);
                    if (len > 0.0f) { ex = ddx / len; ey = ddy / len; }
                    if (arriving && len / dt < sdes) sdes = len / dt;
                }
            }
            float vdx = 0.0f, vdy = 0.0f;
            if (goal != G_NONE && speed > 0.0f) {
                unsigned long long ctr[4] = {(unsigned long long)id, (unsigned long long)s_step, 0ull, 0ull};
                fp_philox4x64(ctr, S.seed, 0ull);
                const float xi1 = (float)(ctr[0] >> 40) * (1.0f / 16777216.0f);
                const float xi2 = (float)(ctr[1] >> 40) * (1.0f / 16777216.0f);
                vdx = sdes * ex + S.ped_noise * (xi1 - 0.5f);
                vdy = sdes * ey + S.ped_noise * (xi2 - 0.5f);
            }
            // repulsion from neighbours in the 3 x 3 bins, fixed-point accumulation
            const float vdn = sqrtf(vdx * vdx + vdy * vdy);
            const float fcut = expf((2.0f * kRb - kR) / kB);
            long long Fx = 0, Fy = 0;
            const int bx = ci / S.hk, by = cj / S.hk;
            const int bx0 = bx > 0 ? bx - 1 : 0, bx1 = bx + 1 < S.nbx ? bx + 1 : S.nbx - 1;
            const int by0 = by > 0 ? by - 1 : 0, by1 = by + 1 < S.nby ? by + 1 : S.nby - 1;
            for (int yy = by0; yy <= by1; ++yy) {
                const int k0 = S.bin_start[yy * S.nbx + bx0], k1 = S.bin_start[yy * S.nbx + bx1 + 1];
                for (int k = k0; k < k1; ++k) {
                    if (k == j) continue;
                    const float4 q = *reinterpret_cast<const float4 *>(&S.pedA[2 * k]);
                    const float rx = x - q.x, ry = y - q.y;
                    if (fabsf(rx) >= kR || fabsf(ry) >= kR) continue;
                    const float d2 = rx * rx + ry * ry;
                    if (d2 >= kR * kR || d2 <= 0.0f) continue;
                    const float d = sqrtf(d2);
                    const float fm = kA * (expf((2.0f * kRb - d) / kB) - fcut);
                    float fx = fm * rx / d, fy = fm * ry / d;
                    if (vdn > 0.0f) {
                        const float w = -(vdx * rx + vdy * ry) / (vdn * d);
                        if (w > 0.0f) {
                            fx += kSide * w * fm * (-ry / d);
                            fy += kSide * w * fm * (rx / d);
                        }
                    }
                    Fx += __float2ll_rn(fx * 4294967296.0f);
                    Fy += __float2ll_rn(fy * 4294967296.0f);
                }
            }
            const float fxs = (float)Fx * (1.0f / 4294967296.0f), fys = (float)Fy * (1.0f / 4294967296.0f);
            // relaxation toward the desired velocity, capped at the state's speed
            const float a = fminf(1.0f, dt / kTau);
            vx = vx + a * (vdx - vx) + dt * fxs;
            vy = vy + a * (vdy - vy) + dt * fys;
            if (speed <= 0.0f) {
                vx = 0.0f; vy = 0.0f;
            } else {
                const float sp = sqrtf(vx * vx + vy * vy);
                if (sp > speed) { vx = vx * (speed / sp); vy = vy * (speed / sp); }
            }
            float xn = x + dt * vx, yn = y + dt * vy;
            if (walkable_at(S, xn, yn)) {
            } else if (walkable_at(S, xn, y)) { yn = y; vy = 0.0f; }
            else if (walkable_at(S, x, yn)) { xn = x; vx = 0.0f; }
            else { xn = x; yn = y; vx = 0.0f; vy = 0.0f; }
            int exited = 0;
            if (goal == G_EXIT) {
                const int ii = fp_cell_of(xn, dx), jj = fp_cell_of(yn, dx);
                if (S.exitm[(size_t)jj * S.nx + ii]) exited = 1;
            }
            if (exited) atomicAdd(&C->n_exited, 1ull);
            S.pedB[2 * j] = make_uint4(__float_as_uint(xn), __float_as_uint(yn), __float_as_uint(vx), __float_as_uint(vy));
            S.pedB[2 * j + 1] = make_uint4(id, FP_META(role, task, hr, exited), (unsigned)timer, pb.w);
        }
    }
    // state histogram, aggregated per warp
    if (dt_ticks > 0) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const unsigned m = __ballot_sync(0xffffffffu, valid && hr == s);
            if (lane == 0 && m) atomicAdd(&C->hist[s], (unsigned long long)__popc(m));
        }
    }
}

// New records sit in B at [first_slot, first_slot + count): give them ids
// first_id.. in order, clear their hazard/exit bytes, check they stand in a
// walkable cell, and seed the by-id archive.
__global__ void assign_ids_kernel(const __grid_constant__ FpSim S, int first_slot, int first_id, int count) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int i = first_slot + k;
    const int id = first_id + k;
    uint4 a = S.pedB[2 * i], b = S.pedB[2 * i + 1];
    b.x = (unsigned)id;
    b.y = FP_META(FP_META_ROLE(b.y) ? 1 : 0, FP_META_TASK(b.y) <= 4 ? FP_META_TASK(b.y) : 0, 0, 0);
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

}  // namespace

int fp_scan_tiles(int nbins) { return (nbins + 1 + kScanTile - 1) / kScanTile; }

void fp_launch_hash_count(const FpSim &S, cudaStream_t st) {
    hash_count_kernel<<<blocks_for(S.cap, 256), 256, 0, st>>>(S);
}
void fp_launch_scan(const FpSim &S, cudaStream_t st) {
    scan_kernel<<<fp_scan_tiles(S.nbins), kScanThreads, 0, st>>>(S);
}
void fp_launch_gather(const FpSim &S, cudaStream_t st) { gather_kernel<<<blocks_for(S.cap, 256), 256, 0, st>>>(S); }
void fp_launch_ped_step(const FpSim &S, int par, int slot, cudaStream_t st) {
    ped_step_kernel<<<blocks_for(S.cap, 256), 256, 0, st>>>(S, par, slot);
}
void fp_launch_assign_ids(const FpSim &S, int first_slot, int first_id, int count, cudaStream_t st) {
    if (count > 0) assign_ids_kernel<<<blocks_for(count, 256), 256, 0, st>>>(S, first_slot, first_id, count);
}
void fp_launch_read_peds(const FpSim &S, uint4 *out, int n_total, cudaStream_t st) {
    if (n_total <= 0) return;
    read_arch_kernel<<<blocks_for(n_total, 256), 256, 0, st>>>(S, out, n_total);
    read_live_kernel<<<blocks_for(S.cap, 256), 256, 0, st>>>(S, out);
}
