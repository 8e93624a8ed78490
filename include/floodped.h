/*
 * floodped.h -- C ABI of the B300 coupled flood-pedestrian simulation library
 * (libfloodped.so).
 *
 * One simulation step advances, on one GPU and from the same state at step n,
 *   (a) every hydrodynamic cell by the first-order finite-volume shallow-water
 *       update of Eq. (2) of the paper (Section 2.2) with the global CFL time
 *       step of Section 3,
 *   (b) every pedestrian by the rules of Sections 2.3-2.4 (Table 1 hazard
 *       states, navigation toward the emergency exit / sandbag storage /
 *       barrier, repulsion from neighbours, responders' sandbag cycle),
 *   (c) the two-way coupling of Section 2.4: evacuees per cell raise the
 *       Manning n of the next flood update (n_M + N_p n_M, N_p <= 20) and
 *       completed sandbag layers raise the barrier cells' bed.
 *
 * Conventions (all entry points):
 *   - Grids are row-major, index c = j * nx + i; i runs west->east along x,
 *     j south->north along y; cell (i, j) covers [i dx, (i+1) dx) x [j dx, (j+1) dx).
 *   - Array arguments may be host or device pointers (unified addressing
 *     decides); the library copies them, never keeps a caller pointer, and the
 *     set-up calls return only once the copy is complete.
 *   - Every call returns FP_OK (0) or a negative FP_E* code; fp_last_error()
 *     gives a message.  No C++ exception crosses the ABI.  A handle is not
 *     thread-safe; distinct handles are independent.
 *   - Time is kept as int64 ticks of 2^-20 s (the step's dt is quantised down
 *     to whole ticks).
 */
#ifndef FLOODPED_H
#define FLOODPED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define FP_OK 0
#define FP_EINVAL (-1)    /* bad argument or size */
#define FP_ENOMEM (-2)    /* device allocation failed */
#define FP_ECUDA (-3)     /* a CUDA call failed */
#define FP_ETIMEOUT (-4)  /* a bounded device-side wait gave up */
#define FP_ENAN (-5)      /* non-finite state detected */
#define FP_EOVERFLOW (-6) /* a per-cell counter or capacity overflowed */

/* boundary condition codes, one per boundary cell (Section 3.1) */
#define FP_BC_WALL 0         /* reflective wall */
#define FP_BC_TRANSMISSIVE 1 /* zero-gradient ("slip" outflow) */
#define FP_BC_INFLOW 2       /* ghost at rest with the hydrograph depth */
#define FP_BC_DISCHARGE 3    /* breach: a wall through which the discharge hydrograph enters */

#define FP_EDGE_SOUTH 0 /* row j = 0, nx codes */
#define FP_EDGE_NORTH 1 /* row j = ny-1, nx codes */
#define FP_EDGE_WEST 2  /* column i = 0, ny codes */
#define FP_EDGE_EAST 3  /* column i = nx-1, ny codes */

/* pedestrian roles (Section 2.4) and states */
#define FP_ROLE_EVACUEE 0
#define FP_ROLE_RESPONDER 1
#define FP_HR_DRY 0      /* depth below 1 mm */
#define FP_HR_LOW 1      /* Table 1: HR in [0, 0.75), 1.8 m/s */
#define FP_HR_MEDIUM 2   /* [0.75, 1.5), 0.9 m/s */
#define FP_HR_HIGH 3     /* [1.5, 2.5), 0.45 m/s */
#define FP_HR_HIGHEST 4  /* >= 2.5, 0 m/s */
#define FP_TASK_TO_DEPOT 0
#define FP_TASK_PICKUP 1
#define FP_TASK_TO_BARRIER 2
#define FP_TASK_DROP 3
#define FP_TASK_DONE 4

/* fields for fp_read_state */
#define FP_FIELD_H 0        /* float[ny*nx] depth h (m) */
#define FP_FIELD_HU 1       /* float[ny*nx] unit discharge hu (m^2/s) */
#define FP_FIELD_HV 2       /* float[ny*nx] unit discharge hv (m^2/s) */
#define FP_FIELD_Z 3        /* float[ny*nx] bed elevation z (m), barrier raises included */
#define FP_FIELD_PEDS 4     /* fp_ped[n_peds_total], indexed by pedestrian id */
#define FP_FIELD_COUNTERS 5 /* one fp_counters */
#define FP_FIELD_NAV 6      /* uint8[3*ny*nx]: exit, storage, barrier direction codes */
#define FP_FIELD_MASS 7     /* double[2]: water volume sum h dx^2 (m^3), net boundary inflow volume (m^3) */
#define FP_FIELD_PROFILE 8  /* double[7]: profiled steps, then total ms of: the hashing/scan part,
                               the flood update, the gather + pedestrian part, whole steps;
                               then the cell updates the flood kernel computed (cells of
                               tiles not skipped as dry, see fp_step); then total ms of
                               the pedestrian kernel alone (0 in FP_MODE_PERSISTENT)
                               (see fp_set_profiling) */
#define FP_FIELD_HR_MAX 9   /* float[1]: largest hazard rating HR = (max(|u|,|v|) + 0.5) h over
                               the cells holding water (Section 2.4; sampled over time it is the
                               maximum-HR history of Fig. 5(b)) */

/* Simulation set-up.  Sizes: nx, ny >= 1; max_peds >= 0. */
typedef struct fp_config {
    int32_t nx, ny;     /* cells along x and y */
    float dx;           /* cell side (m); cells are square */
    float g;            /* gravity (m/s^2) */
    float cfl;          /* Courant number (Section 3) */
    float ped_noise;    /* amplitude of the random term of the desired velocity (m/s) */
    double t_end;       /* simulated end time (s); steps past it do nothing */
    uint64_t seed;      /* key of the counter-based random generator */
    int32_t max_peds;   /* pedestrian capacity */
    int32_t coupling;   /* 1: evacuees raise Manning n (Section 2.4), 0: off */
    int32_t evac_trigger; /* 0: evacuees head for the exit from t = 0;
                             1: only once some cell holds water (Section 2.4) */
    int32_t tile_rows;  /* flood run height: 8, 16 or 32 (0 = 16) */
    int32_t riemann;    /* interface flux: FP_RIEMANN_HLL (0, the paper's first-order
                           scheme) or FP_RIEMANN_HLLC (1: the cited scheme's three-wave
                           solver, which also resolves the contact wave of the
                           tangential momentum); else FP_EINVAL */
    int32_t order;      /* 0 or 1: the paper's first-order update (Eq. 2); 2: the cited
                           scheme at full order -- MUSCL minmod reconstruction of the
                           surface, the depth and the velocities (first order on the
                           domain edge and next to dry cells), the hydrostatic
                           reconstruction with the centred bed-slope term (a lake at
                           rest stays at rest), two-stage Runge-Kutta; every cell is
                           computed every step; FP_MODE_KERNELS only (no persistent
                           mode, batch or surrogate window); else FP_EINVAL */
    int32_t reserved[2];
} fp_config;

#define FP_RIEMANN_HLL 0
#define FP_RIEMANN_HLLC 1

/* One pedestrian record (32 bytes).  On input, id is ignored: ids are given
 * in order of addition starting at 0.  timer_ticks is the remaining wait of a
 * responder picking up or dropping a sandbag. */
typedef struct fp_ped {
    float x, y;      /* position (m) */
    float vx, vy;    /* velocity (m/s) */
    uint32_t id;
    uint8_t role;    /* FP_ROLE_* */
    uint8_t task;    /* FP_TASK_* (responders); evacuees: 0, or FP_TASK_VISIT0 + d
                        for a visitor bound for door d (fp_set_doors) */
    uint8_t hr;      /* FP_HR_* of the last step */
    uint8_t exited;  /* 1 once through the emergency exit, 2 once a visitor has
                        left through the door it was bound for */
    int32_t timer_ticks;
    float v0;        /* walking speed on dry ground (m/s) */
} fp_ped;

typedef struct fp_counters {
    int64_t t_ticks;        /* simulated time */
    int64_t step;           /* steps taken with dt > 0 */
    int64_t n_active;       /* pedestrians still in the domain */
    int64_t n_exited;
    int64_t total_bags;     /* sandbags dropped so far */
    int64_t applied_layers; /* barrier cell-layers completed and applied to z */
    int64_t neg_depth;      /* negative depths clamped to 0 (expected 0) */
    int64_t hist[5];        /* pedestrians per FP_HR_* state in the last step */
    int32_t wet;            /* 1 once any cell held >= 1 mm of water */
    uint32_t error_flags;   /* device-side error bits (0 = none) */
    int64_t ped_updates;    /* pedestrians advanced, summed over steps */
    int64_t cfl_exceeded;   /* fixed-dt steps whose Courant number exceeded cfg.cfl
                               (see fp_set_fixed_dt; 0 in CFL mode) */
    int64_t n_ids;          /* pedestrian ids issued: added, or admitted through a door
                               (FP_FIELD_PEDS returns this many records) */
    int64_t n_entered;      /* visitors admitted through the doors (fp_set_doors) */
    int64_t n_left;         /* visitors gone through the door they were bound for */
} fp_counters;

typedef struct fp_sim fp_sim; /* opaque handle, owned by the library */

/* Create a simulation: validates *cfg, allocates device memory on the current
 * CUDA device.  Terrain defaults to flat, dry, walkable, n = 0.01, all walls. */
int fp_sim_create(const fp_config *cfg, fp_sim **out);

/* Run subsequent work on a caller CUDA stream (cudaStream_t, may be NULL for the
 * library's own stream).  The caller keeps ownership of the stream. */
int fp_set_stream(fp_sim *sim, void *cuda_stream);

/* Terrain (Section 2.1 flood agent z, n_M; navigation map walkable cells and
 * emergency exit cells).  z, n0: float[ny*nx]; walkable, exit_mask: uint8[ny*nx]
 * (non-zero = yes).  Rebuilds the navigation fields. */
int fp_set_terrain(fp_sim *sim, const float *z, const float *n0, const uint8_t *walkable,
                   const uint8_t *exit_mask);

/* Bed elevation only (Section 2.1 flood agent z), float[ny*nx]: replaces z,
 * barrier raises included, leaving walkability and the navigation fields as
 * they are (e.g. to restore a run taken mid-deployment together with
 * fp_set_barrier_progress).  The next two steps compute every flood tile. */
int fp_set_bed(fp_sim *sim, const float *z);

/* Boundary codes of one edge (FP_EDGE_*): uint8[nx] for south/north, uint8[ny]
 * for west/east, each FP_BC_*. */
int fp_set_boundary(fp_sim *sim, int32_t edge, const uint8_t *codes);

/* Inflow depth hydrograph (Section 3.1, depth form): n >= 1 points (t_k, h_k),
 * t increasing (s), h >= 0 (m); linear between points, constant outside. */
int fp_set_hydrograph(fp_sim *sim, const double *t, const double *h, int32_t n);

/* Discharge hydrograph (Section 3.1, the paper's form): n >= 1 points (t_k,
 * Q_k), t increasing (s), Q >= 0 (m^3/s); linear between points, constant
 * outside (a triangle (0, 0), (t_inflow / 2, Q_peak), (t_inflow, 0) is the
 * paper's).  The water enters through the boundary cells coded
 * FP_BC_DISCHARGE, spread evenly over their total width B = count x dx, at
 * depth h_inflow (m, > 0; the paper's 1 m): over a step [t, t + dt] each
 * breach face carries the mass flux q = (V(t + dt) - V(t)) / (dt B), V the
 * exact volume the hydrograph has released since t = 0, and the momentum
 * q^2 / h_inflow, added to the flux of a wall (so the domain gains exactly
 * V(t + dt) - V(t); with Q = 0 the breach is a wall).  The CFL step includes
 * the inflowing water's speed Q(t) / (B h_inflow) + sqrt(g h_inflow).
 * FP_EINVAL for bad points or depth.  Not taken by fp_surrogate_advance. */
int fp_set_discharge(fp_sim *sim, const double *t, const double *q, int32_t n, double h_inflow);

/* Sandbag storage cells and the ordered barrier cells (Section 2.4, Fig. 3-right),
 * flat cell indices; n_layers = N_L layers of one bag thickness (0.25 m). */
int fp_set_goals(fp_sim *sim, const int32_t *depot_cells, int32_t n_depot,
                 const int32_t *barrier_cells, int32_t n_barrier, int32_t n_layers);

/* Entrance doors and the entry/exit flow before the flood (Sections 2.4, 3 and
 * 3.2: pedestrians enter and leave through the doors, each door used with
 * equal probability; once water is seen nobody enters any more and everyone
 * present evacuates).  Door d (0 <= d < n_doors <= FP_MAX_DOORS) is the walkable
 * cells cells[k] with door[k] == d (flat indices, n_cells entries); visitors
 * enter in its first listed cell.  With cfg.evac_trigger = 1 and while no cell
 * has held water, every door admits one visitor at each whole multiple of
 * entry_period_s (>= 2^-10 s, rounded to the tick) within a step's interval
 * (t, t + dt] (t >= 0): an evacuee record (role 0) with the next id, at rest at
 * a random point of the middle half of the entry cell (each axis), dry walking
 * speed uniform in [v0_min, v0_max] (0 <= v0_min <= v0_max <= 10 m/s), task
 * FP_TASK_VISIT0 + its destination door, drawn with probability 1/n_doors.
 * The draws come from the random generator's block at counter (id, 0, 1, 0).
 * Before the trigger a visitor walks toward its destination door on that
 * door's navigation field and leaves (exited = 2, fp_counters.n_left) after
 * the move that puts it in one of the door's cells; once water is seen it is
 * an evacuee bound for the emergency exit (task 0).  An admission past the
 * capacity (cfg.max_peds ids) is refused and fp_synchronize reports
 * FP_EOVERFLOW.  Records added with fp_add_pedestrians may carry a visitor task
 * too.  n_doors = 0 removes the doors; fp_set_terrain removes them as well (set
 * them after the terrain).  FP_EINVAL for cells outside the domain or not
 * walkable, a door with no cell, or values out of range. */
#define FP_MAX_DOORS 8
#define FP_TASK_VISIT0 8
int fp_set_doors(fp_sim *sim, const int32_t *cells, const int32_t *door, int32_t n_cells, int32_t n_doors,
                 double entry_period_s, double v0_min, double v0_max);

/* Water state U = [h, hu, hv] (Eq. 1), float[ny*nx] each; h >= 0. */
int fp_set_state(fp_sim *sim, const float *h, const float *hu, const float *hv);

/* Set simulated time (ticks) and step index (the random generator's counter). */
int fp_set_time(fp_sim *sim, int64_t t_ticks, int64_t step);

/* Sandbags already dropped and barrier cell-layers already built into z (for a
 * run resumed mid-deployment); total_bags >= 0, 0 <= applied_layers. */
int fp_set_barrier_progress(fp_sim *sim, int64_t total_bags, int64_t applied_layers);

/* Append count pedestrians; each must stand in a walkable cell inside the domain. */
int fp_add_pedestrians(fp_sim *sim, const fp_ped *peds, int32_t count);

/* Remove all pedestrians and reset the exit and sandbag counters. */
int fp_clear_pedestrians(fp_sim *sim);

/* Enqueue n_steps coupled steps on the simulation's stream (asynchronous).
 * Flood tiles whose cells and one-cell halo held no water after the previous
 * step, whose output already holds the zero state and that have no active
 * inflow ghost are skipped (the update would write zeros: every flux is zero);
 * the first two steps after fp_set_state, fp_set_time, fp_set_hydrograph or a
 * surrogate window compute every tile. */
int fp_step(fp_sim *sim, int32_t n_steps);

/* How fp_step runs a step (both give bit-identical results):
 * FP_MODE_KERNELS (default): four or five kernels per step on two streams (the flood
 *   update overlaps the pedestrian chain), 64-step CUDA graphs;
 * FP_MODE_PERSISTENT (devices with cooperative launch): up to 256 steps per
 *   launch of one persistent kernel whose phases are separated by grid
 *   barriers with bounded waits (FP_ETIMEOUT if one gives up). */
/* Launch shape of the per-step kernels (results do not depend on it): flood
 * tile height tile_rows (8, 16, 32 cells; 64 wide) and lanes per pedestrian in
 * the pedestrian step (1, 2, 4, 8, 16).  Chosen by the package's autotuner. */
int fp_set_tuning(fp_sim *sim, int32_t tile_rows, int32_t ped_lanes);

/* Hash-ahead in FP_MODE_KERNELS (results do not depend on it): with on = 1
 * (the default) the pedestrian kernel also hashes the records it writes into
 * the bins of the next step, whose hashing pass then shrinks to a one-thread
 * kernel (sandbag layers, bag snapshot) where a barrier can be built and to
 * nothing elsewhere; with on = 0 every step opens with a hashing pass of one
 * thread per record.  The first saves a launch's worth of
 * latency per step; the second is faster where the pedestrian kernel runs in
 * many waves, each block then ending with an atomic round trip.  Chosen by the
 * package's autotuner.  FP_EINVAL for on other than 0 or 1. */
int fp_set_hash_ahead(fp_sim *sim, int32_t on);

#define FP_MODE_KERNELS 0
#define FP_MODE_PERSISTENT 1
int fp_set_step_mode(fp_sim *sim, int32_t mode);

/* Fixed time step (build-added; the paper's step is the CFL step of Section 3):
 * dt_seconds > 0 makes every later step dt_seconds long (rounded to the
 * 2^-20 s tick, at least one tick, at most 1 s; the last step before t_end is
 * shortened to end on it).  Steps whose Courant number max(|u|,|v|)+sqrt(g h)
 * times dt / dx exceeds cfg.cfl are counted in fp_counters.cfl_exceeded; the
 * step is taken all the same.  dt_seconds = 0 returns to the CFL step.  The
 * learned surrogate runs on a fixed step. */
int fp_set_fixed_dt(fp_sim *sim, double dt_seconds);

/* Profiling mode (on != 0): fp_step synchronises at its end and accumulates
 * the time of the parts of each step -- per-step kernels: the call's steps
 * captured into one CUDA graph with CUDA events around the kernel groups
 * (without programmatic dependent launches, which the events would split) and
 * replayed once; persistent kernel: global-timer stamps at every phase
 * boundary.  FP_FIELD_PROFILE
 * returns the totals.  Turning it on resets them. */
int fp_set_profiling(fp_sim *sim, int32_t on);

/* ---- batched ensemble --------------------------------------------------------
 * Many independent scenarios (different grids, crowds, barriers, hydrographs)
 * stepped together: each step is one set of kernels over all members (flat
 * tile / record / pedestrian work lists), 64-step CUDA graphs.  Every member
 * keeps its own time step, clock and counters, so a member's results are
 * bit-identical to stepping it alone.  This is the ensemble use of the
 * simulator (Section 3.3 runs 36 scenarios of responder group size x barrier
 * height); the paper runs them one by one.
 *
 * fp_batch_create: sims[0..n) are simulations created and loaded through the
 *   calls above, on the current device, at the same step parity (e.g. all
 *   fresh, or all stepped the same number of times); they must outlive the
 *   batch and must not be stepped on their own while batched.  The batch
 *   re-reads their configuration at every fp_batch_step.  Launch shapes: in
 *   the per-step-kernel mode each member runs with the flood run height and
 *   lanes per pedestrian set on it by fp_set_tuning when the batch is created
 *   (one flood and one pedestrian launch per distinct value; results never
 *   depend on the shape); the persistent mode runs 8-row runs and 1 lane.
 * fp_batch_step: n_steps coupled steps of every member (asynchronous on the
 *   batch's stream).  fp_batch_synchronize waits for it and reports device
 *   error bits of any member; read members with fp_read_state afterwards. */
typedef struct fp_batch fp_batch;
int fp_batch_create(fp_sim *const *sims, int32_t n, fp_batch **out);
int fp_batch_step(fp_batch *batch, int32_t n_steps);
/* How fp_batch_step runs (both give every member the bytes of stepping it alone):
 * FP_MODE_KERNELS (default): per step one set of batch kernels, 64-step CUDA
 *   graphs; FP_MODE_PERSISTENT (devices with cooperative launch): up to 256
 *   steps of every member per launch of one persistent kernel (every CTA
 *   resident), the phases of a step separated by grid barriers with bounded
 *   waits (member 0's fp_set_barrier_wait_limit; a wait that gives up is
 *   reported by fp_batch_synchronize as FP_ETIMEOUT).  FP_EINVAL for another
 *   mode or no cooperative launch. */
int fp_batch_set_step_mode(fp_batch *batch, int32_t mode);
int fp_batch_synchronize(fp_batch *batch);
int fp_batch_destroy(fp_batch *batch);

/* ---- learned surrogate -------------------------------------------------------
 * Build-added (the paper has no surrogate): a 5-layer 3x3 convolutional net
 * 8 -> 32 -> 32 -> 32 -> 32 -> 3 channels, ReLU between layers, mapping
 * (h, hu, hv, z) over an 11 x 11 neighbourhood to the change of (h, hu, hv) of
 * the centre cell over FP_SUR_WINDOW fixed time steps.  Forward on the tensor
 * cores (tcgen05, BF16 operands, FP32 accumulation); the 8 input channels are
 * the four inputs rounded to BF16 and the BF16-rounded remainders of that
 * rounding (so the first layer sees them to about 16 bits); FP32 master parameters,
 * layer by layer w[ky][kx][ci][co] then b[co]. */
#define FP_SUR_WINDOW 8
#define FP_SUR_HALO 5
/* The last layer's output times this is the predicted change: changes of
 * 1e-4 .. 1e-2 over a window are then order-1 outputs of the net. */
#define FP_SUR_OUT_SCALE (1.0f / 1024.0f)
typedef struct fp_surrogate fp_surrogate;
int fp_surrogate_num_params(void);
int fp_surrogate_create(uint64_t seed, fp_surrogate **out);
int fp_surrogate_destroy(fp_surrogate *sur);
int fp_surrogate_get_params(fp_surrogate *sur, float *dst, size_t n);
int fp_surrogate_set_params(fp_surrogate *sur, const float *src, size_t n);
/* x: device FP32 [B][H][W][4] = (h, hu, hv, z); y: device FP32
 * [B][H-10][W-10][3] = predicted change of (h, hu, hv); H, W >= 11. */
int fp_surrogate_forward(fp_surrogate *sur, const float *x, int32_t B, int32_t H, int32_t W, float *y);
/* Loss = mean squared error of the forward output against target (device FP32
 * [B][H-10][W-10][3]) and its gradient with respect to every parameter
 * (grads: host or device, fp_surrogate_num_params floats; may be NULL).  The
 * backward runs on the tensor cores as well: each layer's output gradient is
 * carried as its BF16 rounding plus the BF16 rounding of the remainder (about
 * FP32 precision), per-CTA partial sums are added in a fixed order, so the
 * result does not change from call to call. */
int fp_surrogate_gradients(fp_surrogate *sur, const float *x, const float *target, int32_t B, int32_t H, int32_t W,
                           float *grads, double *loss);
/* One Adam step (beta1 0.9, beta2 0.999) of learning rate lr on that loss. */
int fp_surrogate_train_step(fp_surrogate *sur, const float *x, const float *target, int32_t B, int32_t H, int32_t W,
                            float lr, double *loss);
/* At most ctas CTAs for each of the net's kernels (0: as many as the GPU
 * holds), e.g. to leave SMs to a simulation stepping beside it.  Results are
 * the same up to the order of the weight-gradient partial sums.  Returns
 * FP_EINVAL for ctas < 0. */
int fp_surrogate_set_max_ctas(fp_surrogate *sur, int32_t ctas);

/* Advance a simulation by n_windows windows of FP_SUR_WINDOW fixed steps with
 * the surrogate standing in for the flood update (requires fp_set_fixed_dt;
 * kernel step mode is used whatever fp_set_step_mode says).  One window:
 *   1. tiles of FP_SUR_TILE x FP_SUR_TILE cells whose region grown by
 *      FP_SUR_WINDOW cells holds no water (h = 0, no inflow over the window)
 *      are dry: the plain update leaves them unchanged, so they are skipped;
 *   2. every other tile, with a FP_SUR_HALO-cell halo (a 256 x 256 input;
 *      cells past the domain edge repeat the edge cell), goes through the
 *      net: U' = U + dU, h' >= 0, no momentum where h' < 1 mm;
 *   3. the pedestrians take the window's steps on the state at its start
 *      (coupled steps whose flood update moves no water), sandbag layers
 *      raising the bed as they complete;
 *   4. guard per tile: |change of tile water volume - inflow through the tile
 *      edges| / max(tile volume, 1 cm x tile area) <= guard->mass_tol, where
 *      the inflow is the window length times the mean of the HLL mass fluxes
 *      of the start and end states; U' finite; Courant number of U' <= cfg.cfl;
 *      with guard->fix_tol > 0 the mass bound is fix_tol instead and every
 *      accepted tile's h, hu, hv are scaled by one factor so that its volume
 *      change equals that inflow (mass balance closed exactly per tile);
 *   5. a failed tile is recomputed by the plain update from the window's start
 *      state over the tile grown by FP_SUR_WINDOW cells (cells outside held at
 *      their start values), with the evacuee roughness of the window's end;
 *   6. every guard->check_every windows (0: never) the whole grid is recomputed
 *      by the plain update and the largest depth difference over the net
 *      tiles the guard accepted is recorded (rejected tiles take the plain
 *      result anyway); when it exceeds guard->check_tol (m), the next
 *      guard->suspend_windows windows run the plain update on every tile.
 * Stops before a window that would cross t_end.  *stats accumulates (zero it
 * before the first call).  Synchronises the stream. */
#define FP_SUR_TILE 246  /* output cells per tile side: the net's input tile, halo included, is 256 x 256 */
typedef struct fp_surrogate_guard {
    float mass_tol;           /* 1e-4 */
    float check_tol;          /* 0.01 m */
    int32_t check_every;      /* 8 windows = 64 steps */
    int32_t suspend_windows;  /* 8 */
    float fix_tol;            /* 0: off (the mass bound is mass_tol, no correction) */
} fp_surrogate_guard;
typedef struct fp_surrogate_stats {
    int64_t windows;          /* windows advanced */
    int64_t tiles;            /* tile-windows in total */
    int64_t tiles_net;        /* tile-windows given to the net */
    int64_t tiles_fallback;   /* net tiles the guard sent to the plain update, of which */
    int64_t fail_mass;        /*   over the mass bound, */
    int64_t fail_courant;     /*   over the Courant limit, */
    int64_t fail_nonfinite;   /*   with a non-finite value (a tile may count under several) */
    int64_t tiles_plain;      /* tile-windows of check and suspended windows */
    int64_t checks;           /* plain checks */
    int64_t checks_failed;    /* checks over check_tol */
    double max_residual;      /* largest guard mass residual of a net tile */
    double max_check_error;   /* largest depth difference of accepted net tiles at a check (m) */
} fp_surrogate_stats;
int fp_surrogate_advance(fp_sim *sim, fp_surrogate *sur, int32_t n_windows, const fp_surrogate_guard *guard,
                         fp_surrogate_stats *stats);

/* Wait for enqueued work; returns FP_ETIMEOUT / FP_EOVERFLOW / FP_ENAN when the
 * device raised the corresponding error bit (a non-finite depth or discharge
 * written by the flood update: FP_ENAN; a grid-barrier wait that gave up:
 * FP_ETIMEOUT).  An error is reported once: the call then clears the device
 * error word and the per-step hash and evacuee counts, so the handle stays
 * usable, but the water and pedestrian state reached by the failed steps is
 * undefined -- set it again (fp_set_state, fp_clear_pedestrians +
 * fp_add_pedestrians, fp_set_time) before stepping on. */
int fp_synchronize(fp_sim *sim);

/* Bound of every grid-barrier wait of the persistent step kernel
 * (FP_MODE_PERSISTENT), in polls of the barrier word (default 4,194,304, a
 * few seconds).  A CTA whose wait runs out sets the timeout error bit and
 * leaves the kernel (no copy of it is in flight at a barrier); the others
 * follow at their next barrier, and fp_synchronize returns FP_ETIMEOUT.  A
 * small limit makes a wait run out on purpose (failure-detection tests);
 * polls >= 0, else FP_EINVAL. */
int fp_set_barrier_wait_limit(fp_sim *sim, int32_t polls);

/* Copy one FP_FIELD_* into dst (host or device), bytes >= the field's size.
 * Synchronises the stream. */
int fp_read_state(fp_sim *sim, int32_t which, void *dst, size_t bytes);

/* Free the handle and its device memory. */
int fp_destroy(fp_sim *sim);

/* Last error message of the handle (or, with sim NULL, of the last failed
 * fp_sim_create or fp_water_volume_noalloc). */
const char *fp_last_error(const fp_sim *sim);

/* ---- allocation-free entry point --------------------------------------------
 * The paper has no counterpart: this is a service of the library.
 *
 * Water volume sum(h) * dx^2 (m^3, FP64) of a depth grid the caller owns, for
 * callers that may not allocate device memory through this library: code whose
 * device memory is all owned by a host framework's pool (a cudaMalloc/cudaFree
 * from here would bypass the pool, and cudaFree synchronises the whole device),
 * tools that size their device memory once at start-up and must not grow it,
 * and hot loops where an allocation per call would cost more than the sum.
 * It allocates nothing: its scratch is one fixed device array of
 * FP_NOALLOC_MAX_ROWS + 32 doubles (~512 KB) that every GPU loading the
 * library holds until the process exits.
 *
 * h: device pointer to ny rows of nx floats, row r at h + r * row_pitch
 * (row_pitch >= nx, in elements); out: device-accessible pointer to one double,
 * written when the kernel finishes; cuda_stream: cudaStream_t or NULL.  The
 * call is asynchronous on that stream.  Returns FP_EINVAL (with a message in
 * fp_last_error(NULL)) for null pointers, nx or ny < 1, row_pitch < nx, dx <= 0,
 * or ny > FP_NOALLOC_MAX_ROWS; FP_ECUDA if the set-up or launch fails.
 *
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture begins.  Every call shares the one scratch array and the
 * kernel re-arms its completion counter for the next call, so calls must not
 * overlap on the GPU: two calls in flight at once (other streams, other host
 * threads) race on the array. */
#define FP_NOALLOC_MAX_ROWS 65536
int fp_water_volume_noalloc(const float *h, int32_t nx, int32_t ny, int64_t row_pitch, float dx,
                            double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FLOODPED_H */
