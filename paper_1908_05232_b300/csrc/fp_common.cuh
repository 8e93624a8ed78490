// fp_common.cuh -- device data layout and shared device helpers of the coupled
// flood-pedestrian step (Shirvani, Kesserwani & Richmond, arXiv 1908.05232).
//
// HBM layout (one simulation):
//   - water planes h, hu, hv (two copies, ping-pong by step parity), bed z and
//     base Manning n0: float, padded pitch `px` floats (a multiple of 8, at
//     least nx + 8), cell (i, j) stored at (j + 1) * px + i + FP_PADX.  The
//     4-float guard columns keep every TMA box start 16-byte aligned and every
//     4-cell group a 16-byte vector; guard rows j = -1 and j = ny are zero and
//     never read as cells.
//   - occ: uint16 evacuees per cell with the same padding, incremented by the
//     hash kernel (Section 2.4 N_p) and cleared by the flood kernel that uses it.
//   - blk_wet: per 64 x 8-cell block and plane parity, 0 if the block holds no
//     water in that plane (written by the flood update that produced it).
//   - walkable / exit / navigation codes: uint8[ny * nx], unpadded.
//   - pedestrians: arrays of 32-byte fp_ped records (float4 x,y,vx,vy + uint4
//     id,meta,timer,v0), "A" sorted by spatial-hash bin, "B" the step output.
//   - a 4-slot clock ring: slot s holds the time, step index, max wave speed
//     and wet flag of the step that reads it.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <utility>

#define FP_PADX 4
#define FP_TX 64                 // flood tile width (cells)
#define FP_TICKS_F 1048576.0f    // ticks per second (2^20)
#define FP_DT_MAX_TICKS 1048576LL
#define FP_H_EPS_F 1e-6f         // depth with no velocity (m)
#define FP_H_DRY_F 1e-3f         // dry pedestrian below 1 mm (m)
#define FP_NP_CAP 20             // evacuees counted per cell (Section 2.4)
#define FP_MAX_HYDRO 64
#define FP_BARRIER_POLLS_DEFAULT (1 << 22)

// error bits
#define FP_ERR_TIMEOUT 1u
#define FP_ERR_OCC_OVERFLOW 2u
#define FP_ERR_NAN 4u
#define FP_ERR_BAD_PED 8u
#define FP_ERR_CAPACITY 16u   // a door admission past the pedestrian capacity was refused

#define FP_SCAN_TILE 2048      // bins per tile of the bin-count scan
#define FP_MAX_DOORS 8
#define FP_TASK_VISIT0 8      // evacuee task 8 + d: a visitor bound for door d

// pedestrian meta word: role | task << 8 | hr << 16 | exited << 24 (byte lanes of fp_ped)
#define FP_META_ROLE(m) ((m) & 0xffu)
#define FP_META_TASK(m) (((m) >> 8) & 0xffu)
#define FP_META_HR(m) (((m) >> 16) & 0xffu)
#define FP_META_EXITED(m) (((m) >> 24) & 0xffu)
#define FP_META(role, task, hr, ex) ((uint32_t)(role) | ((uint32_t)(task) << 8) | ((uint32_t)(hr) << 16) | ((uint32_t)(ex) << 24))

#define FP_AT_GOAL 8
#define FP_UNREACHABLE 255

struct __align__(16) FpClock {
    long long t;            // ticks
    long long step;         // step index (random counter)
    unsigned int smax_bits; // max over wet cells of max(|u|,|v|) + sqrt(g h), float bits
    int wet;                // sticky: some cell held >= 1 mm
    float h_in;             // inflow hydrograph depth at t, rounded to FP32 (evaluated once per step)
    float q_speed;          // wave speed of the water entering through the discharge breach at t (0: none)
};

struct FpCounters {
    int nA;                           // records in A (sorted, input of the pedestrian step)
    int nB;                           // records in B (output of the pedestrian step)
    unsigned long long total_bags;    // bags dropped so far
    unsigned long long bags_snap;     // total at the start of the step
    unsigned long long applied;       // barrier cell-layers applied to z
    unsigned long long n_exited;
    unsigned long long neg_depth;
    unsigned int err;
    int bad_ped;
    unsigned long long hist[5];
    double mass;                      // last mass reduction (m^3)
    double inflow;                    // net boundary inflow volume (m^3)
    unsigned int mass_done;           // blocks finished in the mass reduction
    unsigned int cfl_over;            // fixed-dt steps whose CFL number exceeded the limit
    unsigned long long ped_updates;   // sum over steps with dt > 0 of pedestrians advanced
    unsigned int hr_max_bits;         // largest hazard rating of the last FP_FIELD_HR_MAX read, float bits
    int n_ids;                        // pedestrian ids issued (added or admitted through a door)
    unsigned long long n_entered;     // visitors admitted through the doors
    unsigned long long n_left;        // visitors gone through the door they were bound for
    unsigned int flood_ticket;        // next run of the flood kernel in flight (0 between launches)
};

struct FpSim {
    int nx, ny, px;            // cells, padded pitch (floats)
    int nbx, nby, hk, nbins;   // hash bins (hk x hk cells each), nbins = nbx * nby
    float dx, g, cfl, ped_noise;
    long long t_end;           // ticks
    unsigned long long seed;
    int coupling, evac_trigger, has_inflow, n_hydro;
    int cap;                   // pedestrian capacity
    int nb, n_layers, bpc;     // barrier cells, layers, bags per cell-layer
    float *h[2], *hu[2], *hv[2];
    float *z, *n0;
    unsigned short *occ[2];    // evacuees per cell, by the parity of the step that uses them
    const unsigned char *bc[4];
    const unsigned char *walk;    // per cell: bit 0 walkable, bit 1 exit
    const unsigned *nbr;          // per cell: the walk flags of the 3 x 3 cells centred on it, 2 bits each,
                                  // row by row from the south-west (0 outside the domain)
    const unsigned char *nav[3];  // per goal (exit, depot, barrier): direction code 0..7, FP_AT_GOAL, 255
    const unsigned char *arrive;  // per cell: bit g set if the cell nav[g] points to is a goal cell of g
    const int *barrier;
    const double *hydro_t, *hydro_h;
    FpClock *clock;
    FpCounters *cnt;
    uint4 *pedA, *pedB;        // 2 x uint4 per record
    float2 *posA;              // positions of the records of A (the neighbour scans read these)
    float2 *xiA;               // the step's two uniform draws of each record of A (written by the gather)
    uint4 *arch;               // records by id (exited ones)
    int *bin_count;            // nbins + 1 (last = exited)
    int *bin_start;            // nbins + 2
    int *pkey, *pslot;         // per record of B
    int *tile_sum;             // per scan tile of FP_SCAN_TILE bins: the records hashed into it (zeroed by the gather)
    double *bflux;             // 2 nx + 2 ny inflow volume per boundary face (S, N, W, E)
    double *partials;          // mass reduction partial sums
    int *scan_part;            // persistent kernel: bin-count total of each CTA's chunk
    unsigned long long *phase_ts;  // optional: global timer at each persistent-kernel phase end
    int phase_ts_steps;            // steps recorded in phase_ts (4 stamps per step + 1)
    long long dt_fixed;            // fixed time step in ticks (0: CFL step)
    int barrier_polls;             // polls of a persistent-kernel grid barrier before it gives up
    int riemann;                   // interface flux: 0 HLL, 1 HLLC
    int order;                     // 1: first order (the paper's); 2: MUSCL + two-stage Runge-Kutta
    float *mh, *mhu, *mhv;         // second order: the first stage's state (padded planes)
    // second order: per tile of 32 x 8 cells (row-major over the tile grid), 0
    // if h = hu = hv = 0 in all its cells: [0], [1] the state planes by parity,
    // [2] the first stage's state (written by the stage that produced the
    // plane); nullptr when the first-order update is used
    unsigned char *mflag[3];
    // discharge breach (Section 3.1): boundary cells coded FP_BC_DISCHARGE take
    // the hydrograph Q(t) (points q_t, q_Q) spread over their width q_width
    int has_discharge, n_q;
    const double *q_t, *q_Q;
    double q_width;                // breach width B (m): discharge cells x dx
    double h_qin;                  // depth of the inflowing water (m), an FP32 value
    long long q_end_ticks;         // Q = 0 from this time on (the breach is a wall)
    // entrance doors (Sections 3, 3.2): door d admits a visitor every
    // entry_period ticks at its entry cell door_entry[d] while no water has been
    // seen; door_nav[d * nx * ny + c] the direction code toward door d,
    // door_arrive[c] bit d: the cell that code points to is a cell of door d
    int n_doors;
    int door_entry[FP_MAX_DOORS];
    long long entry_period;
    float entry_vlo, entry_vspan;  // visitors' dry walking speed: lo + u span
    const unsigned char *door_nav;
    const unsigned char *door_arrive;
    const unsigned char *tile_mask;  // per flood tile: 0 = skip (nullptr: every tile runs)
    // Water flags of 64 x 8-cell blocks, by the parity of the state plane they
    // describe: 0 = the block holds h = hu = hv = 0 there (written by the flood
    // update that produced the plane); 1 = maybe water.  nullptr: not used.
    unsigned char *blk_wet[2];
    unsigned *blk_runs;  // profiling only: flood updates computed per block (nullptr: not counted)
};

#define FP_BLK_ROWS 8

__device__ __forceinline__ size_t fp_pidx(const FpSim &S, int i, int j) {
    return (size_t)(j + 1) * (size_t)S.px + (size_t)(i + FP_PADX);
}

// Piecewise-linear inflow depth at time t (ticks), evaluated in FP64 with
// explicit round-to-nearest operations (no contraction) in the same order as
// any other evaluation of the same table.
__device__ __forceinline__ double fp_hydro_depth(const FpSim &S, long long t_ticks) {
    const int n = S.n_hydro;
    if (n <= 0) return 0.0;
    const double t = __ddiv_rn((double)t_ticks, 1048576.0);
    if (t <= S.hydro_t[0]) return S.hydro_h[0];
    if (t >= S.hydro_t[n - 1]) return S.hydro_h[n - 1];
    for (int k = 0; k + 1 < n; ++k) {
        const double t1 = S.hydro_t[k + 1];
        if (t < t1) {
            const double t0 = S.hydro_t[k];
            const double a = __ddiv_rn(__dsub_rn(t, t0), __dsub_rn(t1, t0));
            return __dadd_rn(S.hydro_h[k], __dmul_rn(__dsub_rn(S.hydro_h[k + 1], S.hydro_h[k]), a));
        }
    }
    return S.hydro_h[n - 1];
}

// Discharge hydrograph Q(t) (m^3/s, t in s): piecewise linear between its
// points, constant outside; FP64 with explicit round-to-nearest operations.
__device__ __forceinline__ double fp_discharge(const FpSim &S, double t) {
    const int n = S.n_q;
    if (n <= 0) return 0.0;
    if (t <= S.q_t[0]) return S.q_Q[0];
    if (t >= S.q_t[n - 1]) return S.q_Q[n - 1];
    for (int k = 0; k + 1 < n; ++k) {
        const double t1 = S.q_t[k + 1];
        if (t < t1) {
            const double t0 = S.q_t[k];
            const double a = __ddiv_rn(__dsub_rn(t, t0), __dsub_rn(t1, t0));
            return __dadd_rn(S.q_Q[k], __dmul_rn(__dsub_rn(S.q_Q[k + 1], S.q_Q[k]), a));
        }
    }
    return S.q_Q[n - 1];
}

// Volume released by the hydrograph from t = 0 to t (m^3): the integral of the
// piecewise-linear Q, one trapezoid per piece between its breakpoints.
__device__ __forceinline__ double fp_discharge_volume(const FpSim &S, double t) {
    if (S.n_q <= 0 || !(t > 0.0)) return 0.0;
    double v = 0.0, a = 0.0;
    for (int k = 0; k <= S.n_q; ++k) {
        double b = k < S.n_q ? S.q_t[k] : t;
        if (b > t) b = t;
        if (b > a) {
            const double qa = fp_discharge(S, a), qb = fp_discharge(S, b);
            v = __dadd_rn(v, __dmul_rn(__dmul_rn(0.5, __dadd_rn(qa, qb)), __dsub_rn(b, a)));
            a = b;
        }
    }
    return v;
}

// Wave speed of the inflowing water at t (ticks): depth h_qin moving at
// Q(t) / (B h_qin), so Q / (B h_qin) + sqrt(g h_qin) in FP32; 0 when Q(t) = 0.
__device__ __forceinline__ float fp_discharge_speed(const FpSim &S, long long t_ticks) {
    if (!S.has_discharge) return 0.0f;
    const double Q = fp_discharge(S, __ddiv_rn((double)t_ticks, 1048576.0));
    if (!(Q > 0.0)) return 0.0f;
    const float u = (float)__ddiv_rn(Q, __dmul_rn(S.q_width, S.h_qin));
    return __fadd_rn(u, __fsqrt_rn(__fmul_rn(S.g, (float)S.h_qin)));
}

// The step's dt in ticks: min(1 s, CFL dx / max wave speed, t_end - t), the
// max over wet cells of the state it reads, the inflow ghost state and the
// water entering through a discharge breach.
// Taken in FP32 with correctly rounded division and square root.
__device__ __forceinline__ long long fp_dt_ticks(const FpSim &S, const FpClock &c, float h_in) {
    if (S.dt_fixed > 0) {
        long long left = S.t_end - c.t;
        if (left < 0) left = 0;
        return S.dt_fixed < left ? S.dt_fixed : left;
    }
    float smax = __uint_as_float(c.smax_bits);
    if (S.has_inflow && h_in > FP_H_EPS_F) {
        const float s = __fsqrt_rn(__fmul_rn(S.g, h_in));
        smax = fmaxf(smax, s);
    }
    if (c.q_speed > 0.0f) smax = fmaxf(smax, c.q_speed);
    long long ticks = FP_DT_MAX_TICKS;
    if (smax > 0.0f) {
        const float dtf = __fdiv_rn(__fmul_rn(S.cfl, S.dx), smax);
        const float tk = __fmul_rn(dtf, FP_TICKS_F);
        ticks = tk >= FP_TICKS_F ? FP_DT_MAX_TICKS : (long long)tk;
    }
    long long left = S.t_end - c.t;
    if (left < 0) left = 0;
    return ticks < left ? ticks : left;
}

// Wave speed of one cell for the CFL bound: max(|u|,|v|) + sqrt(g h).  The max of
// the two correctly rounded quotients equals the quotient of the larger
// magnitude, so one division suffices.
__device__ __forceinline__ float fp_wave_speed(float g, float h, float hu, float hv) {
    const float a = __fdiv_rn(fmaxf(fabsf(hu), fabsf(hv)), h);
    return __fadd_rn(a, __fsqrt_rn(__fmul_rn(g, h)));
}

// Table 1 flood-risk state from HR = (V + 0.5) h, V = max(|u|, |v|), FP32.
__device__ __forceinline__ int fp_hr_state(float h, float hu, float hv) {
    if (!(h >= FP_H_DRY_F)) return 0;
    const float V = __fdiv_rn(fmaxf(fabsf(hu), fabsf(hv)), h);
    const float hr = __fmul_rn(__fadd_rn(V, 0.5f), h);
    if (hr < 0.75f) return 1;
    if (hr < 1.5f) return 2;
    if (hr < 2.5f) return 3;
    return 4;
}

__device__ __forceinline__ int fp_cell_of(float x, float dx) { return (int)floorf(__fdiv_rn(x, dx)); }

// Philox4x64-10 (Salmon et al., SC'11) from its published round function.
__device__ __forceinline__ void fp_philox4x64(unsigned long long c[4], unsigned long long k0, unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0; k1 += W1;
    }
}

// A pedestrian's two uniform draws of a step (the random term of its desired
// velocity): the top 24 bits of the first two words of the generator's block
// at counter (id, step, 0, 0), exact in FP32.
__device__ __forceinline__ float2 fp_step_draws(const FpSim &S, unsigned id, long long step) {
    unsigned long long ctr[4] = {(unsigned long long)id, (unsigned long long)step, 0ull, 0ull};
    fp_philox4x64(ctr, S.seed, 0ull);
    return make_float2((float)(unsigned)(ctr[0] >> 40) * (1.0f / 16777216.0f),
                       (float)(unsigned)(ctr[1] >> 40) * (1.0f / 16777216.0f));
}

__device__ __forceinline__ void fp_set_err(const FpSim &S, unsigned int bit) { atomicOr(&S.cnt->err, bit); }

// tiles of the bin-count scan (the bins and the exited bin)
__device__ __forceinline__ int fp_scan_tiles_dev(int nbins) { return (nbins + 1 + FP_SCAN_TILE - 1) / FP_SCAN_TILE; }

// launchers (defined in flood.cu / peds.cu)
void fp_launch_flood(const FpSim &S, int par, int slot, int tile_rows, cudaStream_t st, bool pdl = false);
void fp_launch_init_clock(const FpSim &S, int par, int slot, cudaStream_t st);
void fp_launch_muscl(const FpSim &S, int par, int slot, cudaStream_t st);
void fp_launch_mass(const FpSim &S, int par, cudaStream_t st);
void fp_launch_hr_max(const FpSim &S, int par, cudaStream_t st);
cudaError_t fp_flood_init_attributes();
void fp_launch_hash_count(const FpSim &S, int par, cudaStream_t st);
void fp_launch_scan(const FpSim &S, cudaStream_t st, bool pdl = false);
void fp_launch_gather(const FpSim &S, int slot, cudaStream_t st, bool pdl = false);
void fp_launch_ped_step(const FpSim &S, int par, int slot, int lanes, cudaStream_t st, bool pdl = false,
                        bool hash_next = false);
void fp_launch_step_begin(const FpSim &S, cudaStream_t st);
void fp_launch_assign_ids(const FpSim &S, int first_slot, int first_id, int count, cudaStream_t st);
void fp_launch_clear_peds(const FpSim &S, cudaStream_t st);
void fp_launch_read_peds(const FpSim &S, uint4 *out, int n_total, cudaStream_t st);
int fp_scan_tiles(int nbins);
void fp_note_error(const char *msg);  // message for fp_last_error(NULL)
int fp_persistent_ctas();
// launch shape of the batch's persistent kernel: flood run height and lanes
// per pedestrian
constexpr int kBatchPersistRows = 8;
constexpr int kBatchPersistLanes = 1;
int fp_batch_persistent_ctas();
cudaError_t fp_launch_batch_persistent(const FpSim *d_sims, const int *d_run_off, const int *d_rec_off, int n,
                                       int total_runs, int total_rec, int max_tiles, int par, int slot, int nsteps,
                                       unsigned *bar, int ctas, cudaStream_t st);
// Members of a batch grouped by launch shape (their own fp_set_tuning): group
// g holds n[g] members (device indices members[g][k]) whose work items --
// flood runs of the group's height, or pedestrian blocks of 256 threads at
// the group's lanes per pedestrian -- are [off[g][k], off[g][k + 1]) of the
// group's flat space of total[g] items.  Flood groups: 8, 16, 32 rows;
// pedestrian groups: 1, 2, 4, 8, 16 lanes.
struct FpBatchGroups {
    static constexpr int kMax = 5;
    const int *members[kMax];
    const int *off[kMax];
    int n[kMax];
    int total[kMax];
};
constexpr int kBatchFloodRows[3] = {8, 16, 32};
constexpr int kBatchPedLanes[5] = {1, 2, 4, 8, 16};

void fp_launch_batch_peds(const FpSim *d_sims, const int *d_rec_off, int n, int total_rec, int max_scan_tiles,
                          const FpBatchGroups &ped_groups, int par, int slot, cudaStream_t st_hash,
                          cudaStream_t st_chain, cudaEvent_t fork, bool hash_part);
void fp_launch_flood_batch(const FpSim *d_sims, const FpBatchGroups &flood_groups, int par, int slot,
                           cudaStream_t st);
cudaError_t fp_launch_persistent(const FpSim &S, int par, int slot, int nsteps, unsigned *bar, int ctas,
                                 cudaStream_t st);

// Programmatic dependent launch: the kernel may be scheduled while the previous
// kernel of its stream is finishing; it must execute fp_pdl_wait() before it
// reads anything that kernel wrote (a no-op when launched normally).
__device__ __forceinline__ void fp_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void fp_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t fp_launch(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// surrogate window (window.cu, surrogate.cu)
struct fp_surrogate;

// Net activations are BF16 images stored by channel groups of 8 (k-cores):
// element (image b, row y, column x, channel c) of an H x W image with C
// channels sits at (((b H + y) (C / 8) + c / 8) P + x) 8 + c % 8 with the row
// pitch P = W rounded up to 32 pixels, so that a row of one group is one
// contiguous run of 512-byte blocks (what the tensor-core operand is staged
// from); pixels x >= W of a row are padding.
// One pixel of the net's input has 16 channels: (a, b, c, d) rounded, then
// their rounded remainders (group 0), then 8 zeros (group 1).
__host__ __device__ constexpr int fp_sur_pitch(int w) { return (w + 31) & ~31; }
__device__ __forceinline__ void fp_sur_pack_pixel(float a, float b, float c, float d, void *group0, void *group1) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(a, b), h1 = __floats2bfloat162_rn(c, d);
    const __nv_bfloat162 l0 = __floats2bfloat162_rn(a - __low2float(h0), b - __high2float(h0));
    const __nv_bfloat162 l1 = __floats2bfloat162_rn(c - __low2float(h1), d - __high2float(h1));
    uint4 w0;
    w0.x = *reinterpret_cast<const unsigned *>(&h0);
    w0.y = *reinterpret_cast<const unsigned *>(&h1);
    w0.z = *reinterpret_cast<const unsigned *>(&l0);
    w0.w = *reinterpret_cast<const unsigned *>(&l1);
    *static_cast<uint4 *>(group0) = w0;
    *static_cast<uint4 *>(group1) = make_uint4(0u, 0u, 0u, 0u);
}
cudaError_t fp_sur_forward_packed(fp_surrogate *sur, const void *x16, int B, int H, int W, float *y, cudaStream_t st);
unsigned fp_sur_error_bits(fp_surrogate *sur);
void fp_launch_clock_advance(const FpSim &S, int slot, cudaStream_t st);
void fp_launch_sur_classify(const FpSim &S, int par, const FpClock *c0, int tiles_x, int tiles_y, unsigned char *wet,
                            cudaStream_t st);
void fp_launch_sur_compact(const unsigned char *flags, int n, int *list, int *batch_of, int *count, cudaStream_t st);
void fp_launch_sur_input(const FpSim &S, const float *h, const float *hu, const float *hv, const int *list, int count,
                         int tiles_x, void *x16, cudaStream_t st);
void fp_launch_sur_apply(const FpSim &S, int par, const float *h0, const float *hu0, const float *hv0,
                         const float *dU, const int *list, const int *batch_of, int count, int tiles_x,
                         const FpClock *c0, float mass_tol, float fix_tol, unsigned char *fail, float *resid, int *n_fail,
                         cudaStream_t st);
void fp_launch_sur_occupancy(const FpSim &S, unsigned short *occ, cudaStream_t st);
void fp_launch_sur_diff(const FpSim &S, const float *a, const float *b, const unsigned char *keep, int tiles_x,
                        unsigned *max_bits, cudaStream_t st);
void fp_launch_sur_merge(const FpSim &S, int par, const float *h, const float *hu, const float *hv,
                         const unsigned char *flags, int tiles_x, int tiles_y, cudaStream_t st);
