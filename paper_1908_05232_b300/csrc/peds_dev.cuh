// peds_dev.cuh -- device code of the pedestrian side of the coupled step
// (Sections 2.3-2.4), shared by the per-step kernels and the persistent
// coupled-step kernel.
//
//   hash_record   a record's hash bin (hk x hk cells, bin side >= the 1 m
//                 neighbour radius) or the "exited" bin, its slot in the bin
//                 (integer atomic), its scan tile's record count and the
//                 evacuee count of its cell (uint16 lanes of the occupancy
//                 plane, N_p of Section 2.4);
//   barrier_and_snapshot   completed sandbag layers raise z;
//   ped_group     eight lanes per pedestrian: Table 1 state from the cell's
//                 h, u, v at step n, responder task, navigation direction,
//                 repulsion from neighbours in the 3 x 3 bins split over the
//                 lanes (integer fixed point, so the sum does not depend on the
//                 order records sit in a bin), velocity relaxation and cap, move
//                 with wall sliding, exit (through the emergency exit, or a
//                 visitor through the door it is bound for);
//   door_entries  visitors admitted through the doors during the step.
#pragma once
#include "fp_common.cuh"

namespace fpdev {


__constant__ float c_speed[5] = {0.0f, 1.8f, 0.9f, 0.45f, 0.0f};  // Table 1 (index 0: own dry speed)

// single-instruction reciprocal square root and base-2 exponential (relative
// error ~1e-7) for the pair forces, whose rounding enters positions far below
// parity tolerances
__device__ __forceinline__ float rsqrt_approx(float v) {
    float r;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float exp2_approx(float v) {
    float r;
    asm("ex2.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Paired FP32 arithmetic (two correctly rounded operations per instruction).
// The code generator merges a paired multiply into a following paired add even
// with the rounding spelled out, so products and sums are written as fused
// multiply-adds with a run-time 1 and -0 (P2): a b - 0 and a 1 + b round once,
// the same bits as the plain product and sum.
struct P2 {
    float2 one, nz;
};
__device__ __forceinline__ float2 p2_fma(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{ .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
        " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd; }"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 p2_mul(const P2 &k, float2 a, float2 b) { return p2_fma(a, b, k.nz); }
__device__ __forceinline__ float2 p2_add(const P2 &k, float2 a, float2 b) { return p2_fma(a, k.one, b); }
__device__ __forceinline__ float2 p2_sub(const P2 &k, float2 a, float2 b) {
    return p2_fma(make_float2(-b.x, -b.y), k.one, a);
}
constexpr float kTau = 0.5f, kA = 2.0f, kB = 0.3f, kRb = 0.25f, kR = 1.0f, kSide = 0.5f;
constexpr int kTPick = 30 * 1048576, kTDrop = 30 * 1048576;
constexpr float kBagT = 0.25f;
__constant__ int c_ox[8] = {1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int c_oy[8] = {0, 1, 0, -1, 1, 1, -1, -1};

enum { G_NONE = 0, G_EXIT = 1, G_DEPOT = 2, G_BARRIER = 3, G_STRAIGHT = 4, G_DOOR = 5 };

// cell flags at a position: bit 0 walkable, bit 1 exit (0 outside the domain)
__device__ __forceinline__ unsigned cell_flags_at(const FpSim &S, float x, float y) {
    const int i = fp_cell_of(x, S.dx), j = fp_cell_of(y, S.dx);
    if (i < 0 || j < 0 || i >= S.nx || j >= S.ny) return 0u;
    return S.walk[(size_t)j * S.nx + i];
}

__device__ __forceinline__ bool walkable_at(const FpSim &S, float x, float y) {
    return (cell_flags_at(S, x, y) & 1u) != 0u;
}



// Values every thread of a step reads once (filled by one thread per CTA).
struct StepCtl {
    long long t, dt_ticks, step;
    unsigned long long bags;
    int wet, nA;
};

__device__ __forceinline__ void load_step_ctl(const FpSim &S, int slot, int nA, StepCtl &ctl) {
    const FpClock c = S.clock[slot];
    ctl.t = c.t;
    ctl.dt_ticks = fp_dt_ticks(S, c, c.h_in);
    ctl.step = c.step;
    ctl.wet = c.wet;
    ctl.bags = S.cnt->bags_snap;
    ctl.nA = min(nA, S.cap);  // the records of A never exceed the capacity
}

// Hash one record of B (index i) for the next step: its bin (or the exited bin),
// its slot in the bin and, for a present evacuee, +1 on its cell's count.
// Of the active lanes, those in the same run of equal values (runs over the
// active lanes in lane order) form one group: *first = the run's lowest lane,
// *n = its size, return = this lane's rank in it.
__device__ __forceinline__ int lane_run(unsigned act, unsigned long long v, int *first, int *n) {
    const int lane = threadIdx.x & 31;
    const unsigned me = 1u << lane, lt = me - 1u;
    const unsigned below = act & lt;
    const int src = below ? 31 - __clz(below) : lane;  // the next active lane below
    const unsigned long long vb = __shfl_sync(act, v, src);
    const unsigned heads = __ballot_sync(act, !below || vb != v);
    const int h = 31 - __clz(heads & (lt | me));
    const unsigned above = heads & ~(lt | me);
    const unsigned upto = above ? (1u << (__ffs(above) - 1)) - 1u : 0xffffffffu;
    const unsigned run = act & upto & ~((1u << h) - 1u);
    *first = h;
    *n = __popc(run);
    return __popc(run & lt);
}

__device__ __forceinline__ void hash_record(const FpSim &S, int i, float x, float y, unsigned meta,
                                            unsigned short *occ) {
    // Records arrive in bin order, so neighbouring lanes mostly share a bin
    // (dense crowds put hundreds in one): each run of lanes with the same bin
    // (same cell) takes its slots (adds its count) with one atomic.
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    int key = S.nbins;
    size_t o = 0;
    bool evac = false;
    if (!FP_META_EXITED(meta)) {
        const int ci = fp_cell_of(x, S.dx), cj = fp_cell_of(y, S.dx);
        key = (cj / S.hk) * S.nbx + ci / S.hk;
        evac = FP_META_ROLE(meta) == 0;
        if (evac) o = fp_pidx(S, ci, cj);
    }
    // bin slots: a run of one bin takes consecutive slots
    int first, n;
    const int rank = lane_run(act, (unsigned long long)key, &first, &n);
    const int bfirst = first;
    int base = 0;
    if (lane == first) base = atomicAdd(&S.bin_count[key], n);
    // the scan's tile sums: a run of lanes in one tile adds its records with one atomic
    lane_run(act, (unsigned long long)(key / FP_SCAN_TILE), &first, &n);
    if (lane == first) atomicAdd(&S.tile_sum[key / FP_SCAN_TILE], n);
    // evacuee counts: runs of evacuees on one cell (other lanes are runs of one);
    // both atomics are in flight before either result is used
    lane_run(act, evac ? (unsigned long long)o : ~0ull - (unsigned long long)lane, &first, &n);
    const unsigned shift = (unsigned)(o & 1) * 16u;
    unsigned old = 0u;
    if (evac && lane == first) old = atomicAdd(reinterpret_cast<unsigned *>(occ + (o & ~(size_t)1)), (unsigned)n << shift);
    base = __shfl_sync(act, base, bfirst);
    S.pkey[i] = key;
    S.pslot[i] = base + rank;
    if (evac && lane == first && ((old >> shift) & 0xffffu) + (unsigned)n > 0xffffu) fp_set_err(S, FP_ERR_OCC_OVERFLOW);
}

// Completed sandbag cell-layers raise the bed (one thread, before the flood
// update of the step reads z); snapshot of the bag count for the step.
__device__ __forceinline__ void barrier_and_snapshot(const FpSim &S) {
    FpCounters *C = S.cnt;
    // both counters loaded before any store (nothing else writes them now)
    const unsigned long long total = C->total_bags, applied = C->applied;
    if (S.nb > 0 && S.n_layers > 0) {
        unsigned long long done = total / (unsigned long long)S.bpc;
        const unsigned long long cap = (unsigned long long)S.nb * (unsigned long long)S.n_layers;
        if (done > cap) done = cap;
        if (done > applied) {
            for (unsigned long long k = applied; k < done; ++k) {
                const int c = S.barrier[k % (unsigned long long)S.nb];
                S.z[fp_pidx(S, c % S.nx, c / S.nx)] += kBagT;
            }
            C->applied = done;
        }
    }
    C->bags_snap = total;
    for (int k = 0; k < 5; ++k) C->hist[k] = 0ull;
}

// One pedestrian (record j of A) by a group of kG lanes (sub = lane in the
// group; kG = 1, 2, 4, 8 or 16).  lookup(key) gives the first record of hash bin key in A.  With
// hash_next the group's first lane also hashes its output record for the next
// step.  Every lane of the warp must call this (shuffles over the full warp).
template <int kG, class Lookup>
__device__ __forceinline__ void ped_group(const FpSim &S, int par, const StepCtl &ctl, int j, int sub,
                                          const Lookup &lookup, bool hash_next) {
    FpCounters *C = S.cnt;
    const bool leader = sub == 0;
    const bool valid = j < ctl.nA;
    const long long dt_ticks = ctl.dt_ticks;
    const bool live = valid && dt_ticks > 0;
    const float dx = S.dx;
    const float dt = (float)dt_ticks * (1.0f / FP_TICKS_F);
    int hr = 0, role = 0, task = 0, timer = 0, goal = G_NONE, target = -1, ci = 0, cj = 0, door = 0;
    unsigned nbr = 0u;  // walk flags of the 3 x 3 cells around the pedestrian
    float x = 0.f, y = 0.f, vx = 0.f, vy = 0.f, speed = 0.f, vdx = 0.f, vdy = 0.f;
    unsigned id = 0, v0bits = 0;
    bool drop = false;
    int rk0[3] = {0, 0, 0}, rk1[3] = {0, 0, 0};  // record ranges of the three bin rows
    if (valid) {
        const uint4 pa = S.pedA[2 * j], pb = S.pedA[2 * j + 1];
        if (dt_ticks == 0) {
            if (leader) {
                S.pedB[2 * j] = pa;
                S.pedB[2 * j + 1] = pb;
                if (hash_next) hash_record(S, j, __uint_as_float(pa.x), __uint_as_float(pa.y), pb.y, S.occ[par ^ 1]);
            }
        } else {
            x = __uint_as_float(pa.x); y = __uint_as_float(pa.y);
            vx = __uint_as_float(pa.z); vy = __uint_as_float(pa.w);
            id = pb.x;
            const unsigned meta = pb.y;
            timer = (int)pb.z;
            v0bits = pb.w;
            role = FP_META_ROLE(meta);
            task = FP_META_TASK(meta);
            ci = fp_cell_of(x, dx);
            cj = fp_cell_of(y, dx);
            const int c = cj * S.nx + ci;
            const size_t pc = fp_pidx(S, ci, cj);
            // independent loads issued together: the cell's water, the step's
            // two uniform draws (fp_step_draws on id and step, computed by the
            // gather that placed the record), the 3 x 3 bin ranges
            const float hc = S.h[par][pc], huc = S.hu[par][pc], hvc = S.hv[par][pc];
            nbr = S.nbr[c];
            const float2 xi = S.xiA[j];
            const float xi1 = xi.x, xi2 = xi.y;
            {
                const int bx = ci / S.hk, by = cj / S.hk;
                const int bx0 = bx > 0 ? bx - 1 : 0, bx1 = bx + 1 < S.nbx ? bx + 1 : S.nbx - 1;
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const int yy = by - 1 + r;
                    if (yy < 0 || yy >= S.nby) { rk0[r] = 0; rk1[r] = 0; continue; }
                    rk0[r] = lookup(yy * S.nbx + bx0);
                    rk1[r] = min(lookup(yy * S.nbx + bx1 + 1), ctl.nA);  // never read past the records of A
                }
            }
            hr = fp_hr_state(hc, huc, hvc);
            speed = hr == 0 ? __uint_as_float(v0bits) : c_speed[hr];
            if (role == 0) {
                // before the trigger a visitor walks to its door; once water is
                // seen (or with no trigger) every evacuee heads for the exit
                if (S.evac_trigger == 0 || ctl.wet) {
                    goal = G_EXIT;
                    task = 0;
                } else if (task >= FP_TASK_VISIT0 && task - FP_TASK_VISIT0 < S.n_doors) {
                    goal = G_DOOR;
                    door = task - FP_TASK_VISIT0;
                }
            } else {
                const unsigned long long cap =
                    (unsigned long long)S.nb * (unsigned long long)S.n_layers * (unsigned long long)S.bpc;
                if (task != 4 && ctl.bags >= cap) task = 4;
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
                        target = S.barrier[(ctl.bags / (unsigned long long)S.bpc) % (unsigned long long)S.nb];
                        if (c == target) { task = 3; timer = kTDrop; }
                        else if (S.nav[2][c] == FP_AT_GOAL) goal = G_STRAIGHT;
                        else goal = G_BARRIER;
                        break;
                    case 3:
                        timer = (int)(timer - dt_ticks);
                        if (timer <= 0) { drop = true; task = 0; timer = 0; }
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
                    int code, bit;
                    unsigned arr;
                    if (goal == G_DOOR) {
                        code = S.door_nav[(size_t)door * ((size_t)S.nx * S.ny) + c];
                        arr = S.door_arrive[c];  // loaded beside the code
                        bit = door;
                    } else {
                        bit = goal == G_EXIT ? 0 : goal == G_DEPOT ? 1 : 2;
                        code = S.nav[bit][c];
                        arr = S.arrive[c];
                    }
                    if (code < 8) {
                        const int ti = ci + c_ox[code], tj = cj + c_oy[code];
                        tx = ((float)ti + 0.5f) * dx;
                        ty = ((float)tj + 0.5f) * dx;
                        have = true;
                        arriving = ((arr >> bit) & 1u) != 0u;
                    }
                }
                if (have) {
                    const float ddx = tx - x, ddy = ty - y;
                    const float len = sqrtf(__fmaf_rn(ddx, ddx, ddy * ddy));
                    if (len > 0.0f) { ex = ddx / len; ey = ddy / len; }
                    if (arriving && len / dt < sdes) sdes = len / dt;
                }
            }
            if (goal != G_NONE && speed > 0.0f) {
                vdx = __fmaf_rn(S.ped_noise, xi1 - 0.5f, sdes * ex);
                vdy = __fmaf_rn(S.ped_noise, xi2 - 0.5f, sdes * ey);
            }
        }
    }
    // repulsion from neighbours in the 3 x 3 bins, split over the group.  Each
    // pair term (|term| < 16 m/s^2) is rounded to an int32 count of 2^-18 m/s^2
    // and summed in 64-bit integers, so the total does not depend on order.
    long long Fx = 0, Fy = 0;
    if (live) {
        const float vdn = sqrtf(__fmaf_rn(vdx, vdx, vdy * vdy));
        const float inv_vdn = vdn > 0.0f ? __frcp_rn(vdn) : 0.0f;
        // exp((2 Rb - d) / B) = 2^(log2(e) (2 Rb - d) / B) = 2^(kC - d kL)
        constexpr float kL = 1.44269504f / kB, kC = 2.0f * kRb * (1.44269504f / kB);
        const float fcut = exp2_approx(__fmaf_rn(-kR, kL, kC));
        // the three bin rows' record ranges as one list, split over the lanes;
        // the next candidate's record is loaded before the current one is used
        const int n0 = rk1[0] - rk0[0], n01 = n0 + (rk1[1] - rk0[1]);
        const int ntot = n01 + (rk1[2] - rk0[2]);
        auto rec_of = [&](int t) { return t < n0 ? rk0[0] + t : t < n01 ? rk0[1] + t - n0 : rk0[2] + t - n01; };
        float2 qn = sub < ntot ? S.posA[rec_of(sub)] : make_float2(0.f, 0.f);
        // The force is carried in units of 2^-18 m/s^2 from the start (kA
        // times a power of two: every product below is the unscaled one times
        // 2^18, exactly).  A term (|v| < 2^22) is rounded to the nearest
        // integer, ties to even, by adding 1.5 * 2^23 in FP32: the sum lies in
        // [2^23, 2^24), where the spacing is 1, and its bits are 0x4B400000 +
        // rint(v).  A lane sums at most 256 terms modulo 2^32 (the true sum is
        // below 2^30 in magnitude) before adding them to its int64 total.
        // With vdn = 0, inv_vdn = 0 makes w = 0: no side-step term, as the
        // model says.
        constexpr float kAs = kA * 262144.0f;
        // Two candidates per lane and iteration (t and t + kG) on the paired
        // FP32 instructions: the same correctly rounded operations as one at a
        // time, products and sums written as fused multiply-adds with a
        // run-time 1 and -0 so that none is merged into another.
        const float one = __fdiv_rn(S.dx, S.dx), nzero = -__fmul_rn(0.0f, S.dx);
        const P2 K{make_float2(one, one), make_float2(nzero, nzero)};
        const float2 xx = make_float2(x, x), yy = make_float2(y, y);
        const float2 vdx2 = make_float2(vdx, vdx), vdy2 = make_float2(vdy, vdy), ivd2 = make_float2(inv_vdn, inv_vdn);
        const float2 fcut2 = make_float2(-fcut, -fcut), kRnd = make_float2(12582912.0f, 12582912.0f);
        float2 qa = qn, qb = sub + kG < ntot ? S.posA[rec_of(sub + kG)] : make_float2(0.f, 0.f);
#pragma unroll 1
        for (int t0 = sub; t0 < ntot; t0 += 256 * kG) {
            const int tend = min(ntot, t0 + 256 * kG);
            unsigned ax = 0u, ay = 0u;
#pragma unroll 1
            for (int t = t0; t < tend; t += 2 * kG) {
                const float2 pa = qa, pb = qb;
                const bool hb = t + kG < tend;
                if (t + 2 * kG < ntot) qa = S.posA[rec_of(t + 2 * kG)];
                if (t + 3 * kG < ntot) qb = S.posA[rec_of(t + 3 * kG)];
                // the pedestrian itself (the same position bits) gives d2 = 0 and
                // is skipped with any other pedestrian at zero distance; |rx| or
                // |ry| >= kR = 1 gives d2 >= 1 after rounding
                const float2 rx = p2_sub(K, xx, make_float2(pa.x, pb.x)), ry = p2_sub(K, yy, make_float2(pa.y, pb.y));
                const float2 d2 = p2_fma(rx, rx, p2_mul(K, ry, ry));
                const bool ua = d2.x < kR * kR && d2.x > 0.0f, ub = hb && d2.y < kR * kR && d2.y > 0.0f;
                if (!ua && !ub) continue;
                const float2 invd = make_float2(rsqrt_approx(d2.x), rsqrt_approx(d2.y));
                const float2 d = p2_mul(K, d2, invd);
                const float2 ea = p2_fma(make_float2(-d.x, -d.y), make_float2(kL, kL), make_float2(kC, kC));
                const float2 fm = p2_mul(K, make_float2(kAs, kAs),
                                         p2_add(K, make_float2(exp2_approx(ea.x), exp2_approx(ea.y)), fcut2));
                const float2 nx_ = p2_mul(K, rx, invd), ny_ = p2_mul(K, ry, invd);
                float2 fx = p2_mul(K, fm, nx_), fy = p2_mul(K, fm, ny_);
                const float2 wm = p2_fma(vdx2, nx_, p2_mul(K, vdy2, ny_));
                const float2 w = p2_mul(K, make_float2(-wm.x, -wm.y), ivd2);
                float2 sw = p2_mul(K, p2_mul(K, make_float2(kSide, kSide), w), fm);
                // no side step for w <= 0: a zero product leaves the term's
                // integer value unchanged
                if (!(w.x > 0.0f)) sw.x = 0.0f;
                if (!(w.y > 0.0f)) sw.y = 0.0f;
                fx = p2_add(K, p2_fma(sw, make_float2(-ny_.x, -ny_.y), fx), kRnd);
                fy = p2_add(K, p2_fma(sw, nx_, fy), kRnd);
                if (ua) { ax += __float_as_uint(fx.x) - 0x4B400000u; ay += __float_as_uint(fy.x) - 0x4B400000u; }
                if (ub) { ax += __float_as_uint(fx.y) - 0x4B400000u; ay += __float_as_uint(fy.y) - 0x4B400000u; }
            }
            Fx += (int)ax;
            Fy += (int)ay;
        }
    }
#pragma unroll
    for (int o = kG / 2; o > 0; o >>= 1) {
        Fx += __shfl_xor_sync(0xffffffffu, Fx, o, kG);
        Fy += __shfl_xor_sync(0xffffffffu, Fy, o, kG);
    }
    if (live && leader) {
        const float fxs = __ll2float_rn(Fx) * (1.0f / 262144.0f), fys = __ll2float_rn(Fy) * (1.0f / 262144.0f);
        // relaxation toward the desired velocity, capped at the state's speed
        const float a = fminf(1.0f, dt / kTau);
        vx = __fmaf_rn(dt, fxs, __fmaf_rn(a, vdx - vx, vx));
        vy = __fmaf_rn(dt, fys, __fmaf_rn(a, vdy - vy, vy));
        if (speed <= 0.0f) {
            vx = 0.0f; vy = 0.0f;
        } else {
            const float sp = sqrtf(__fmaf_rn(vx, vx, vy * vy));
            if (sp > speed) { vx = vx * (speed / sp); vy = vy * (speed / sp); }
        }
        float xn = __fmaf_rn(dt, vx, x), yn = __fmaf_rn(dt, vy, y);
        // the flags of a cell next to the pedestrian's come from its
        // neighbourhood word; a move past the neighbouring cells loads them
        auto flags = [&](float px, float py) -> unsigned {
            const int ddx = fp_cell_of(px, dx) - ci, ddy = fp_cell_of(py, dx) - cj;
            if (ddx >= -1 && ddx <= 1 && ddy >= -1 && ddy <= 1) return (nbr >> (2 * ((ddy + 1) * 3 + ddx + 1))) & 3u;
            return cell_flags_at(S, px, py);
        };
        unsigned fl = flags(xn, yn);  // the exit bit of the usual move too
        if (fl & 1u) {
        } else if (flags(xn, y) & 1u) { yn = y; vy = 0.0f; fl = flags(xn, yn); }
        else if (flags(x, yn) & 1u) { xn = x; vx = 0.0f; fl = flags(xn, yn); }
        else { xn = x; yn = y; vx = 0.0f; vy = 0.0f; fl = flags(xn, yn); }
        // gone: through the emergency exit (1), or a visitor now in a cell of
        // its door (2); the new position is in a walkable cell of the domain
        int exited = goal == G_EXIT && (fl & 2u) ? 1 : 0;
        if (goal == G_DOOR) {
            const size_t cn = (size_t)fp_cell_of(yn, dx) * S.nx + fp_cell_of(xn, dx);
            if (S.door_nav[(size_t)door * ((size_t)S.nx * S.ny) + cn] == FP_AT_GOAL) exited = 2;
        }
        if (exited == 1) atomicAdd(&C->n_exited, 1ull);
        if (exited == 2) atomicAdd(&C->n_left, 1ull);
        if (drop) atomicAdd(&C->total_bags, 1ull);
        const unsigned meta_out = FP_META(role, task, hr, exited);
        S.pedB[2 * j] = make_uint4(__float_as_uint(xn), __float_as_uint(yn), __float_as_uint(vx), __float_as_uint(vy));
        S.pedB[2 * j + 1] = make_uint4(id, meta_out, (unsigned)timer, v0bits);
        if (hash_next) hash_record(S, j, xn, yn, meta_out, S.occ[par ^ 1]);
    }
    // state histogram, aggregated per warp over the group leaders
    if (dt_ticks > 0) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const unsigned m = __ballot_sync(0xffffffffu, live && leader && hr == s);
            if (lane == 0 && m) atomicAdd(&C->hist[s], (unsigned long long)__popc(m));
        }
    }
}


// Visitors entering through the doors during the step (t, t + dt] (Sections 3
// and 3.2): while no water has been seen (evac_trigger 1), door d admits one
// visitor at each whole multiple of the entry period in the interval (t >= 0).
// The step's visitors take the next ids and the slots of B after the nA
// records the pedestrian step writes, door by door; ids past the capacity are
// refused (error bit).  A visitor's draws come from the generator's block at
// counter (id, 0, 1, 0): its position in the door's entry cell (a quarter to
// three quarters of a cell along each axis), its destination door (equal
// probabilities) and its dry walking speed.  It stands at rest, and with
// hash_next it is hashed for the next step like the step's other outputs.
// Called by one full warp of the block whose thread 0 set nB = nA for the step
// (that thread, lane 0 here, moves nB on).
__device__ __forceinline__ void door_entries(const FpSim &S, int par, const StepCtl &ctl, bool hash_next) {
    if (S.n_doors == 0 || S.evac_trigger == 0 || ctl.wet || ctl.dt_ticks <= 0) return;
    const int lane = threadIdx.x & 31;
    FpCounters *C = S.cnt;
    const long long T = S.entry_period;
    const int k = lane < S.n_doors ? (int)((ctl.t + ctl.dt_ticks) / T - ctl.t / T) : 0;
    int incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    const int pre = incl - k;
    const int id0 = C->n_ids;
    const int admitted = max(0, min(total, S.cap - id0));
    __syncwarp();
    if (lane == 0) {
        if (admitted < total) fp_set_err(S, FP_ERR_CAPACITY);
        C->nB = ctl.nA + admitted;
        C->n_ids = id0 + admitted;
        C->n_entered += (unsigned long long)admitted;
    }
    for (int e0 = 0; e0 < admitted; e0 += 32) {
        const int e = e0 + lane;
        int door = 0;  // the last door (with admissions) whose first visitor is <= e
        for (int d = 0; d < S.n_doors; ++d) {
            const int pd = __shfl_sync(0xffffffffu, pre, d), kd = __shfl_sync(0xffffffffu, k, d);
            if (kd > 0 && e >= pd) door = d;
        }
        if (e < admitted) {
            const int id = id0 + e, slot = ctl.nA + e;
            unsigned long long r[4] = {(unsigned long long)id, 0ull, 1ull, 0ull};
            fp_philox4x64(r, S.seed, 0ull);
            const float ox = __fmaf_rn(0.5f, (float)(unsigned)(r[0] >> 42) * (1.0f / 4194304.0f), 0.25f);
            const float oy = __fmaf_rn(0.5f, (float)(unsigned)(r[1] >> 42) * (1.0f / 4194304.0f), 0.25f);
            const int dest = (int)((((r[2] >> 40) * (unsigned long long)S.n_doors)) >> 24);
            const float v0 = __fmaf_rn((float)(unsigned)(r[3] >> 40) * (1.0f / 16777216.0f), S.entry_vspan, S.entry_vlo);
            const int c = S.door_entry[door];
            const float x = __fmul_rn(__fadd_rn((float)(c % S.nx), ox), S.dx);
            const float y = __fmul_rn(__fadd_rn((float)(c / S.nx), oy), S.dx);
            const unsigned meta = FP_META(0, FP_TASK_VISIT0 + dest, 0, 0);
            const uint4 a = make_uint4(__float_as_uint(x), __float_as_uint(y), 0u, 0u);
            const uint4 b = make_uint4((unsigned)id, meta, 0u, __float_as_uint(v0));
            S.pedB[2 * slot] = a;
            S.pedB[2 * slot + 1] = b;
            S.arch[2 * (size_t)id] = a;
            S.arch[2 * (size_t)id + 1] = b;
            if (hash_next) hash_record(S, slot, x, y, meta, S.occ[par ^ 1]);
        }
    }
}

// ---- the bin scan, the gather and the batch's member lookup (shared by the
// per-step, batch and persistent kernels) ------------------------------------
constexpr int kScanItems = 8, kScanThreads = 256, kScanTile = kScanItems * kScanThreads;
static_assert(kScanTile == FP_SCAN_TILE, "the hashing counts records per scan tile");
static_assert(kScanItems == 8, "scan_load and scan_tile move a thread's bins as two int4");

// The counts of this thread's kScanItems consecutive bins of tile `tile`
// (0 past the last bin), two 16-byte loads where the tile is whole.
__device__ __forceinline__ void scan_load(const FpSim &S, int base, int n, int v[kScanItems]) {
    if (base + kScanItems <= n) {
        const int4 a = *reinterpret_cast<const int4 *>(S.bin_count + base);
        const int4 b = *reinterpret_cast<const int4 *>(S.bin_count + base + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = base + k < n ? S.bin_count[base + k] : 0;
    }
}

// Block sum of one int per thread (every thread gets it).
__device__ __forceinline__ int block_sum(int x) {
    __shared__ int s_red[kScanThreads / 32];
    __shared__ int s_tot;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += s_red[w];
        s_tot = t;
    }
    __syncthreads();
    return s_tot;
}

// The tile's exclusive prefix is the sum of the records the hashing counted
// in the tiles before it; then the tile's own exclusive scan.
__device__ __forceinline__ void scan_tile(const FpSim &S, int tile) {
    __shared__ int s_warp[kScanThreads / 32];
    const int tid = threadIdx.x;
    FpCounters *C = S.cnt;
    if (tile == 0 && tid < 5) C->hist[tid] = 0ull;  // the step's state histogram (the pedestrian kernel fills it)
    const int n = S.nbins + 1;
    const int base = tile * kScanTile + tid * kScanItems;
    int part = 0;
    for (int t = tid; t < tile; t += kScanThreads) part += S.tile_sum[t];
    int v[kScanItems];
    scan_load(S, base, n, v);
    const int prefix = block_sum(part);
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sum += v[k];
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
    int wpre = 0;
    for (int w = 0; w < wid; ++w) wpre += s_warp[w];
    int run = prefix + wpre + incl - sum;
    int out[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        out[k] = run;
        run += v[k];
    }
    if (base + kScanItems <= n) {
        const int4 z = make_int4(0, 0, 0, 0);
        *reinterpret_cast<int4 *>(S.bin_count + base) = z;
        *reinterpret_cast<int4 *>(S.bin_count + base + 4) = z;
        *reinterpret_cast<int4 *>(S.bin_start + base) = make_int4(out[0], out[1], out[2], out[3]);
        *reinterpret_cast<int4 *>(S.bin_start + base + 4) = make_int4(out[4], out[5], out[6], out[7]);
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k)
            if (base + k < n) {
                S.bin_count[base + k] = 0;
                S.bin_start[base + k] = out[k];
            }
    }
    // the exited bin (the last) starts where the records still present end
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k == n - 1) {
            S.bin_start[n] = out[k] + v[k];
            C->nA = out[k];
        }
}

// Record i of B to its place in A (or, gone, to the by-id archive), with the
// step's two uniform draws the pedestrian kernel reads beside it.
__device__ __forceinline__ void gather_place(const FpSim &S, int key, int bslot, const uint4 &a, const uint4 &b,
                                             float2 xi) {
    if (key == S.nbins) {
        S.arch[2 * (size_t)b.x] = a;
        S.arch[2 * (size_t)b.x + 1] = b;
    } else {
        const int dst = S.bin_start[key] + bslot;
        if ((unsigned)dst >= (unsigned)S.cap) {  // counts out of step with the records: never write past A
            fp_set_err(S, FP_ERR_BAD_PED);
            return;
        }
        S.pedA[2 * dst] = a;
        S.pedA[2 * dst + 1] = b;
        S.posA[dst] = make_float2(__uint_as_float(a.x), __uint_as_float(a.y));
        S.xiA[dst] = xi;
    }
}

__device__ __forceinline__ void gather_record(const FpSim &S, int i, long long step) {
    const int key = S.pkey[i];
    const uint4 a = S.pedB[2 * i], b = S.pedB[2 * i + 1];
    gather_place(S, key, S.pslot[i], a, b, fp_step_draws(S, b.x, step));
}

// The member owning flat index x: the largest s with off[s] <= x.
__device__ __forceinline__ int batch_member(const int *off, int n, int x) {
    int lo = 0, hi = n - 1;  // largest s with off[s] <= x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}


}  // namespace fpdev
