/*
 * floodped_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, single-threaded FP64 CPU oracle of one coupled
 * flood-pedestrian simulation step of Shirvani, Kesserwani & Richmond,
 * "Agent-based simulator of dynamic flood-people interactions"
 * (arXiv 1908.05232).  Loops run over cells and agents in plain index order.
 * Only the tests, the package smoke check and the benchmark's CPU-baseline leg
 * may load this library; the CUDA path never links or calls it, and it shares
 * no code with it.
 *
 * What it follows (paper sections / equations):
 *   - Eq. (1): 2D shallow-water equations, U = [h, hu, hv], bed slope and
 *     Manning friction sources (Section 2.2).
 *   - Eq. (2): explicit first-order finite-volume update with east/west and
 *     north/south interface fluxes; "Wang et al. 2011 reduced to first order"
 *     is read as a Godunov-type scheme with non-negative hydrostatic
 *     reconstruction of the face depths and the HLL Riemann solver (HLLC,
 *     which also resolves the contact wave, as an option: the cited scheme's
 *     three-wave solver).  The cited scheme at full order, as an option: MUSCL
 *     reconstruction of the surface, the depth and the velocities (minmod
 *     slopes, first order next to dry cells and on the domain edge), the
 *     hydrostatic reconstruction at the faces with the centred bed-slope term
 *     that keeps a lake at rest, and two-stage Runge-Kutta time stepping.
 *   - Section 3 (CFL-adaptive time step when wet, 1.0 s pedestrian step when
 *     dry); Section 3.1 inflow: a depth hydrograph (ghost state) or the
 *     paper's triangular discharge hydrograph Q(t) entering through a breach
 *     of width B with depth h_inflow (boundary mass flux, exact volume).
 *   - Section 2.4 + Table 1: HR = (V + 0.5) h with V = max(|u|, |v|), the
 *     four flood-risk states and walking speeds; evacuee roughness coupling
 *     n_M = n_M + N_p n_M with N_p <= 20; responders' sandbag cycle (storage
 *     -> 30 s pick-up -> barrier -> 30 s drop), the barrier cell raising its
 *     bed by one bag thickness per completed layer, N_L layers.
 *   - Section 2.3: pedestrians steered by navigation information toward their
 *     destination, avoiding each other (a social-force repulsion).
 *   - Sections 2.4, 3 and 3.2: the entry/exit flow before the flood -- visitors
 *     enter through the entrance doors at a constant rate per door, each bound
 *     for a door drawn with equal probability, and leave through it; once any
 *     cell holds water nobody enters and everyone present evacuates.
 *
 * Where floating point decides an integer (the CFL time step in ticks, the
 * hazard state, the cell a position falls in, the wet flag), the decision is
 * taken in FP32 from the FP32-rounded state, the precision of the GPU path.
 *
 * Parity unpinned: the pedestrian-pedestrian repulsion constants (the paper
 * only cites a social-force model) are pinned only by invariants and by
 * brute-force sums on tiny inputs, not by a value the paper prints; the paper's
 * 3484-bag count for its barrier is not derivable and is not reproduced.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_H_EPS 1e-6            /* depth below which a cell has no velocity (m) */
#define OR_H_DRY_F 1e-3f         /* depth below which a pedestrian is "dry" (m) */
#define OR_TICKS 1048576.0       /* ticks per second, 2^20 */
#define OR_DT_MAX_TICKS 1048576  /* 1.0 s pedestrian step */
#define OR_NP_CAP 20             /* at most 20 evacuees counted per cell */

/* boundary codes */
#define OR_BC_WALL 0
#define OR_BC_TRANS 1
#define OR_BC_INFLOW 2
#define OR_BC_DISCHARGE 3
/* pedestrian roles, hazard states, responder task states */
#define OR_EVAC 0
#define OR_RESP 1
#define OR_DRY 0
#define OR_LOW 1
#define OR_MED 2
#define OR_HIGH 3
#define OR_HIGHEST 4
#define OR_TO_DEPOT 0
#define OR_PICKUP 1
#define OR_TO_BARRIER 2
#define OR_DROP 3
#define OR_DONE 4
#define OR_VISIT0 8              /* evacuee task 8 + d: a visitor bound for door d */
#define OR_MAX_DOORS 8
/* navigation codes: 0..7 = direction to the next cell, 8 = at goal, 255 = unreachable */
#define OR_AT_GOAL 8
#define OR_UNREACHABLE 255

/* pedestrian model constants (reading of the cited social-force model) */
static const double OR_TAU = 0.5;     /* relaxation time (s) */
static const double OR_A = 2.0;       /* repulsion strength (m/s^2) */
static const double OR_B = 0.3;       /* repulsion range (m) */
static const double OR_RB = 0.25;     /* body radius (m) */
static const double OR_R = 1.0;       /* neighbour radius (m) */
static const double OR_SIDE = 0.5;    /* share of the repulsion turned sideways when approaching */
static const double OR_SPEED[5] = {0.0, 1.8, 0.9, 0.45, 0.0};  /* Table 1; [0] unused (dry: own v0) */
static const int32_t OR_T_PICK = 30 * 1048576;   /* 30 s pick-up wait */
static const int32_t OR_T_DROP = 30 * 1048576;   /* 30 s drop wait */
static const double OR_BAG_L = 0.40, OR_BAG_W = 0.30, OR_BAG_T = 0.25;  /* Section 3, sandbag (m) */

/* direction table: E, N, W, S, NE, NW, SW, SE */
static const int OR_OX[8] = {1, 0, -1, 0, 1, -1, -1, 1};
static const int OR_OY[8] = {0, 1, 0, -1, 1, 1, -1, -1};

typedef struct {
    int32_t nx, ny;
    double dx, g, cfl;
    int64_t t_end_ticks;
    int32_t n_hydro;
    const double *hydro_t, *hydro_h;
    const uint8_t *bc_s, *bc_n, *bc_w, *bc_e;
    const double *n0;
    const uint8_t *walkable, *exit_mask;
    int32_t n_depot;
    const int32_t *depot_cells;
    int32_t n_barrier;
    const int32_t *barrier_cells;
    int32_t n_layers;
    int32_t coupling, evac_trigger;
    uint64_t seed;
    double ped_noise;
    int64_t dt_fixed_ticks;   /* > 0: fixed step (a build-added mode), else the CFL step */
    int32_t n_q;              /* discharge hydrograph points (0: none) */
    const double *q_t, *q_Q;  /* times (s) and discharges Q (m^3/s) */
    double h_qin;             /* depth of the inflowing water at the breach (m) */
    int32_t riemann;          /* 0: HLL, 1: HLLC (the contact wave resolved) */
    int32_t n_doors;          /* entrance doors (0: no entry/exit flow) */
    int32_t n_door_cells;
    const int32_t *door_cells;   /* flat cell indices; a door's first listed cell is its entry cell */
    const int32_t *door_of;      /* the door of each listed cell */
    int64_t entry_period_ticks;  /* each door admits one visitor every this many ticks */
    double entry_v0_lo, entry_v0_hi;  /* visitors' dry walking speeds (FP32 values, m/s) */
    int32_t order;            /* 2: the second-order (MUSCL, two-stage) scheme; else first order */
} or_params;

typedef struct {
    double *h, *hu, *hv, *z;          /* [ny*nx] */
    double *bflux;                    /* [2*nx+2*ny] inflow volume per boundary face: S, N, W, E */
    int64_t t_ticks, step;
    int32_t wet;
    int32_t pad0;
    int64_t total_bags, applied_layers, neg_depth, n_exited;
    int64_t hist[5];
    int32_t np;
    int32_t pad1;
    double *px, *py, *pvx, *pvy, *pv0;
    int32_t *pid, *ptimer;
    uint8_t *prole, *pfsm, *phr, *pexit;
    uint8_t *nav_exit, *nav_depot, *nav_barrier;  /* [ny*nx] */
    int64_t last_dt_ticks;
    int32_t cap;              /* capacity of the pedestrian arrays (ids 0 .. cap-1) */
    int32_t pad2;
    int64_t n_entered, n_left, entry_refused;
    uint8_t *nav_door;        /* [n_doors][ny*nx] */
} or_state;

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11), written from its     */
/* published definition: 10 rounds of two 64x64->128 multiplies with the   */
/* round and key-schedule (Weyl) constants of the paper.                    */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    __uint128_t p = (__uint128_t)a * (__uint128_t)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void or_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in [0, 1) from the top 24 bits: exact in FP32 and FP64 */
static double or_uniform24(uint64_t r) { return (double)(r >> 40) * (1.0 / 16777216.0); }

/* A visitor's draws (Section 3: doors used with equal probability), from the
 * generator's block at counter (id, 0, 1, 0) -- the per-step draws use
 * (id, step, 0, 0), so the streams never meet:
 *   off[0], off[1]  its entry position inside the entry cell, in cells:
 *                   1/4 + u/2 with u the top 22 bits (exact in FP32);
 *   off[2]          its dry walking speed lo + u (hi - lo), u the top 24 bits,
 *                   one FP32 fused multiply-add after the FP32 difference;
 *   *dest           its destination door floor(u n_doors), u the top 24 bits
 *                   (an integer product: exact). */
void or_visitor_draw(uint64_t seed, uint64_t id, int32_t n_doors, float v0_lo, float v0_hi, float off[3],
                     int32_t *dest) {
    uint64_t ctr[4] = {id, 0, 1, 0}, key[2] = {seed, 0}, r[4];
    or_philox4x64(ctr, key, r);
    off[0] = 0.25f + 0.5f * ((float)(r[0] >> 42) * (1.0f / 4194304.0f));
    off[1] = 0.25f + 0.5f * ((float)(r[1] >> 42) * (1.0f / 4194304.0f));
    const float span = v0_hi - v0_lo;
    off[2] = fmaf((float)(r[3] >> 40) * (1.0f / 16777216.0f), span, v0_lo);
    *dest = (int32_t)(((r[2] >> 40) * (uint64_t)n_doors) >> 24);
}

/* ------------------------------------------------------------------------ */
/* Navigation map (Section 2.1/2.3): a 4-connected BFS distance over        */
/* walkable cells from the goal set; each cell points at the 8-neighbour    */
/* with the smallest distance (ties: E, N, W, S, NE, NW, SW, SE; diagonals  */
/* only when both side cells are walkable).                                 */
/* ------------------------------------------------------------------------ */
void or_nav_field(int32_t nx, int32_t ny, const uint8_t *walkable, const uint8_t *goal,
                  uint8_t *dir_out, int32_t *dist) {
    int64_t n = (int64_t)nx * ny;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t head = 0, tail = 0;
    for (int64_t c = 0; c < n; ++c) {
        dist[c] = -1;
        if (goal[c]) { dist[c] = 0; queue[tail++] = (int32_t)c; }
    }
    while (head < tail) {
        int32_t c = queue[head++];
        int32_t i = c % nx, j = c / nx;
        for (int k = 0; k < 4; ++k) {
            int32_t ii = i + OR_OX[k], jj = j + OR_OY[k];
            if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
            int32_t d = jj * nx + ii;
            if (!walkable[d] || dist[d] >= 0) continue;
            dist[d] = dist[c] + 1;
            queue[tail++] = d;
        }
    }
    for (int32_t j = 0; j < ny; ++j) {
        for (int32_t i = 0; i < nx; ++i) {
            int32_t c = j * nx + i;
            if (goal[c]) { dir_out[c] = OR_AT_GOAL; continue; }
            if (dist[c] < 0) { dir_out[c] = OR_UNREACHABLE; continue; }
            int best = -1;
            int32_t bestd = dist[c];
            for (int k = 0; k < 8; ++k) {
                int32_t ii = i + OR_OX[k], jj = j + OR_OY[k];
                if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
                int32_t d = jj * nx + ii;
                if (dist[d] < 0) continue;
                if (k >= 4) {
                    if (!walkable[j * nx + ii] || !walkable[jj * nx + i]) continue;
                }
                if (dist[d] < bestd) { bestd = dist[d]; best = k; }
            }
            dir_out[c] = best < 0 ? OR_UNREACHABLE : (uint8_t)best;
        }
    }
    free(queue);
}

/* ------------------------------------------------------------------------ */
/* Boundary inflow depth hydrograph (Section 3.1, depth form): piecewise     */
/* linear in time, constant outside the table.                              */
/* ------------------------------------------------------------------------ */
double or_hydro_depth(const or_params *P, int64_t t_ticks) {
    double t = (double)t_ticks / OR_TICKS;
    int n = P->n_hydro;
    if (n <= 0) return 0.0;
    if (t <= P->hydro_t[0]) return P->hydro_h[0];
    if (t >= P->hydro_t[n - 1]) return P->hydro_h[n - 1];
    for (int k = 0; k + 1 < n; ++k) {
        if (t < P->hydro_t[k + 1]) {
            double a = (t - P->hydro_t[k]) / (P->hydro_t[k + 1] - P->hydro_t[k]);
            return P->hydro_h[k] + (P->hydro_h[k + 1] - P->hydro_h[k]) * a;
        }
    }
    return P->hydro_h[n - 1];
}

/* ------------------------------------------------------------------------ */
/* Discharge hydrograph (Section 3.1): Q(t) piecewise linear between its     */
/* points, constant outside; the inflow volume V(t) = integral of Q from 0   */
/* to t, exact for that shape (a trapezoid per piece).                       */
/* ------------------------------------------------------------------------ */
double or_discharge(const or_params *P, double t) {
    int n = P->n_q;
    if (n <= 0) return 0.0;
    if (t <= P->q_t[0]) return P->q_Q[0];
    if (t >= P->q_t[n - 1]) return P->q_Q[n - 1];
    for (int k = 0; k + 1 < n; ++k) {
        if (t < P->q_t[k + 1]) {
            double a = (t - P->q_t[k]) / (P->q_t[k + 1] - P->q_t[k]);
            return P->q_Q[k] + (P->q_Q[k + 1] - P->q_Q[k]) * a;
        }
    }
    return P->q_Q[n - 1];
}

double or_discharge_volume(const or_params *P, double t) {
    if (P->n_q <= 0 || t <= 0.0) return 0.0;
    /* the breakpoints of Q in (0, t): Q is linear between consecutive ones */
    double v = 0.0, a = 0.0;
    for (int k = 0; k <= P->n_q; ++k) {
        double b = k < P->n_q ? P->q_t[k] : t;
        if (b > t) b = t;
        if (b > a) {
            v += 0.5 * (or_discharge(P, a) + or_discharge(P, b)) * (b - a);
            a = b;
        }
    }
    return v;
}

/* width (m) of the breach: the boundary cells coded discharge */
double or_discharge_width(const or_params *P) {
    int32_t cnt = 0;
    for (int i = 0; i < P->nx; ++i) cnt += (P->bc_s[i] == OR_BC_DISCHARGE) + (P->bc_n[i] == OR_BC_DISCHARGE);
    for (int j = 0; j < P->ny; ++j) cnt += (P->bc_w[j] == OR_BC_DISCHARGE) + (P->bc_e[j] == OR_BC_DISCHARGE);
    return (double)cnt * P->dx;
}

static int or_has_inflow(const or_params *P) {
    for (int i = 0; i < P->nx; ++i) if (P->bc_s[i] == OR_BC_INFLOW || P->bc_n[i] == OR_BC_INFLOW) return 1;
    for (int j = 0; j < P->ny; ++j) if (P->bc_w[j] == OR_BC_INFLOW || P->bc_e[j] == OR_BC_INFLOW) return 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* CFL time step (Section 3): dt = min(1 s, CFL * dx / max wave speed,      */
/* t_end - t) over wet cells and inflow ghost states, in ticks of 2^-20 s.  */
/* Decision taken in FP32.                                                  */
/* ------------------------------------------------------------------------ */
int64_t or_dt_ticks(const or_params *P, const double *h, const double *hu, const double *hv,
                    int64_t t_ticks) {
    if (P->dt_fixed_ticks > 0) {
        int64_t left = P->t_end_ticks - t_ticks;
        if (left < 0) left = 0;
        return P->dt_fixed_ticks < left ? P->dt_fixed_ticks : left;
    }
    const float g = (float)P->g;
    const float heps = (float)OR_H_EPS;
    float smax = 0.0f;
    int64_t n = (int64_t)P->nx * P->ny;
    for (int64_t c = 0; c < n; ++c) {
        float hf = (float)h[c];
        if (hf > heps) {
            float u = (float)hu[c] / hf, v = (float)hv[c] / hf;
            float a = fmaxf(fabsf(u), fabsf(v));
            float s = a + sqrtf(g * hf);
            if (s > smax) smax = s;
        }
    }
    if (or_has_inflow(P)) {
        float hin = (float)or_hydro_depth(P, t_ticks);
        if (hin > heps) {
            float s = sqrtf(g * hin);
            if (s > smax) smax = s;
        }
    }
    /* the inflowing water at the breach: depth h_qin at velocity Q(t) / (B h_qin) */
    const double B = or_discharge_width(P);
    if (B > 0.0) {
        double Q = or_discharge(P, (double)t_ticks / OR_TICKS);
        if (Q > 0.0) {
            float u = (float)(Q / (B * P->h_qin));
            float s = u + sqrtf(g * (float)P->h_qin);
            if (s > smax) smax = s;
        }
    }
    int64_t ticks = OR_DT_MAX_TICKS;
    if (smax > 0.0f) {
        float dtf = ((float)P->cfl * (float)P->dx) / smax;
        float tk = dtf * 1048576.0f;
        ticks = tk >= 1048576.0f ? OR_DT_MAX_TICKS : (int64_t)tk;
    }
    int64_t left = P->t_end_ticks - t_ticks;
    if (left < 0) left = 0;
    return ticks < left ? ticks : left;
}

/* ------------------------------------------------------------------------ */
/* Hazard rating and flood-risk state (Section 2.4, Table 1), in FP32.      */
/* Bands are lower-inclusive; below 1 mm of water the pedestrian is dry.    */
/* ------------------------------------------------------------------------ */
int or_hr_state(float h, float hu, float hv) {
    if (!(h >= OR_H_DRY_F)) return OR_DRY;
    float u = hu / h, v = hv / h;
    float V = fmaxf(fabsf(u), fabsf(v));
    float hr = (V + 0.5f) * h;
    if (hr < 0.75f) return OR_LOW;
    if (hr < 1.5f) return OR_MED;
    if (hr < 2.5f) return OR_HIGH;
    return OR_HIGHEST;
}

static int32_t or_cell_index(double x, float dxf) { return (int32_t)floorf((float)x / dxf); }

/* ------------------------------------------------------------------------ */
/* HLL flux across one face (normal velocity un, tangential ut), given the  */
/* reconstructed depths.  out = (mass, normal momentum, tangential          */
/* momentum) fluxes, with the face pressure 1/2 g h^2 included.             */
/* ------------------------------------------------------------------------ */
static double or_press(double g, double h) { return 0.5 * g * h * h; }

void or_hll(double g, double hL, double unL, double utL, double hR, double unR, double utR,
            double out[3]) {
    if (hL <= OR_H_EPS && hR <= OR_H_EPS) { out[0] = out[1] = out[2] = 0.0; return; }
    double qL = hL * unL, qR = hR * unR;
    double FL[3] = {qL, qL * unL + or_press(g, hL), qL * utL};
    double FR[3] = {qR, qR * unR + or_press(g, hR), qR * utR};
    if (hL == hR && unL == unR && utL == utR) {
        out[0] = FL[0]; out[1] = FL[1]; out[2] = FL[2];
        return;
    }
    double cL = sqrt(g * hL), cR = sqrt(g * hR), sL, sR;
    if (hL <= OR_H_EPS) {
        sL = unR - 2.0 * cR;
        sR = unR + cR;
    } else if (hR <= OR_H_EPS) {
        sL = unL - cL;
        sR = unL + 2.0 * cL;
    } else {
        double us = 0.5 * (unL + unR) + (cL - cR);
        double cs = 0.5 * (cL + cR) + 0.25 * (unL - unR);
        double a = unL - cL, b = us - cs;
        sL = a < b ? a : b;
        double c = unR + cR, d = us + cs;
        sR = c > d ? c : d;
    }
    if (sL >= 0.0) { out[0] = FL[0]; out[1] = FL[1]; out[2] = FL[2]; return; }
    if (sR <= 0.0) { out[0] = FR[0]; out[1] = FR[1]; out[2] = FR[2]; return; }
    double UL[3] = {hL, qL, hL * utL};
    double UR[3] = {hR, qR, hR * utR};
    for (int k = 0; k < 3; ++k)
        out[k] = (sR * FL[k] - sL * FR[k] + sL * sR * (UR[k] - UL[k])) / (sR - sL);
}

/* HLLC (Toro's three-wave solver for the shallow-water equations): the mass
 * and normal momentum fluxes are HLL's; the tangential momentum is carried by
 * the mass flux with the tangential velocity of the side the contact wave
 * S* = (sL hR (uR - sR) - sR hL (uL - sL)) / (hR (uR - sR) - hL (uL - sL))
 * leaves behind (left for S* > 0, right for S* < 0, their mean at S* = 0). */
void or_hllc(double g, double hL, double unL, double utL, double hR, double unR, double utR, double out[3]) {
    or_hll(g, hL, unL, utL, hR, unR, utR, out);
    if (hL <= OR_H_EPS && hR <= OR_H_EPS) return;
    if (hL == hR && unL == unR && utL == utR) return;
    double cL = sqrt(g * hL), cR = sqrt(g * hR), sL, sR;
    if (hL <= OR_H_EPS) { sL = unR - 2.0 * cR; sR = unR + cR; }
    else if (hR <= OR_H_EPS) { sL = unL - cL; sR = unL + 2.0 * cL; }
    else {
        double us = 0.5 * (unL + unR) + (cL - cR);
        double cs = 0.5 * (cL + cR) + 0.25 * (unL - unR);
        double a = unL - cL, b = us - cs;
        sL = a < b ? a : b;
        double c = unR + cR, d = us + cs;
        sR = c > d ? c : d;
    }
    if (sL >= 0.0 || sR <= 0.0) return;  /* one-sided: the physical flux already carries the right ut */
    double ss = (sL * hR * (unR - sR) - sR * hL * (unL - sL)) / (hR * (unR - sR) - hL * (unL - sL));
    double ut = ss > 0.0 ? utL : (ss < 0.0 ? utR : 0.5 * (utL + utR));
    out[2] = out[0] * ut;
}

static void or_flux(const or_params *P, double g, double hL, double unL, double utL, double hR, double unR,
                    double utR, double out[3]) {
    if (P->riemann == 1) or_hllc(g, hL, unL, utL, hR, unR, utR, out);
    else or_hll(g, hL, unL, utL, hR, unR, utR, out);
}

/* one side of a face: depth, velocities, bed */
typedef struct { double h, u, v, z; } or_side;

static or_side or_cell_side(const or_state *S, int64_t c) {
    or_side s;
    s.h = S->h[c];
    s.z = S->z[c];
    if (s.h > OR_H_EPS) { s.u = S->hu[c] / s.h; s.v = S->hv[c] / s.h; }
    else { s.u = 0.0; s.v = 0.0; }
    return s;
}

/* ghost state outside an edge cell; normal_x selects which velocity is normal */
static or_side or_ghost(uint8_t code, or_side in, int normal_x, double h_in) {
    or_side g = in;
    if (code == OR_BC_WALL || code == OR_BC_DISCHARGE) {
        if (normal_x) g.u = -in.u; else g.v = -in.v;
    } else if (code == OR_BC_INFLOW) {
        g.h = h_in; g.u = 0.0; g.v = 0.0;
    }
    return g;
}

/* ------------------------------------------------------------------------ */
/* Eq. (2): U^{n+1} = U^n - dt/dx (F_E - F_W) - dt/dy (G_N - G_S) + S.      */
/* Bed slope enters through the hydrostatic reconstruction: at each face    */
/* z_f = max(z_L, z_R), h*_{L,R} = max(0, eta_{L,R} - z_f), and each cell   */
/* takes the face flux minus the pressure 1/2 g h*^2 of its own side.       */
/* Manning friction (Eq. 1, S_f) is applied point-implicitly afterwards.    */
/* ------------------------------------------------------------------------ */
void or_flood_step(const or_params *P, or_state *S, int64_t dt_ticks, const double *n_eff) {
    const int32_t nx = P->nx, ny = P->ny;
    const int64_t n = (int64_t)nx * ny;
    const double dt = (double)dt_ticks / OR_TICKS;
    const double dx = P->dx, g = P->g;
    const double h_in = or_hydro_depth(P, S->t_ticks);
    /* discharge breach (Section 3.1): over this step the mean unit discharge
     * qb = (V(t + dt) - V(t)) / (dt B) enters through the faces coded
     * discharge (walls otherwise), carrying momentum qb * u_in, u_in = qb / h_qin */
    double qb = 0.0, u_in = 0.0;
    {
        const double B = or_discharge_width(P);
        const double t0 = (double)S->t_ticks / OR_TICKS, t1 = (double)(S->t_ticks + dt_ticks) / OR_TICKS;
        if (B > 0.0 && dt > 0.0) {
            qb = (or_discharge_volume(P, t1) - or_discharge_volume(P, t0)) / (dt * B);
            u_in = qb / P->h_qin;
        }
    }
    double *FE = (double *)calloc((size_t)n * 3, sizeof(double));
    double *FW = (double *)calloc((size_t)n * 3, sizeof(double));
    double *GN = (double *)calloc((size_t)n * 3, sizeof(double));
    double *GS = (double *)calloc((size_t)n * 3, sizeof(double));
    double f[3];
    /* x faces: face i lies between cell i-1 and cell i */
    for (int32_t j = 0; j < ny; ++j) {
        for (int32_t i = 0; i <= nx; ++i) {
            or_side L, R;
            if (i == 0) { R = or_cell_side(S, (int64_t)j * nx); L = or_ghost(P->bc_w[j], R, 1, h_in); }
            else L = or_cell_side(S, (int64_t)j * nx + i - 1);
            if (i == nx) R = or_ghost(P->bc_e[j], L, 1, h_in);
            else if (i > 0) R = or_cell_side(S, (int64_t)j * nx + i);
            double zf = L.z > R.z ? L.z : R.z;
            double hLs = L.h + L.z - zf; if (hLs < 0.0) hLs = 0.0;
            double hRs = R.h + R.z - zf; if (hRs < 0.0) hRs = 0.0;
            or_flux(P, g, hLs, L.u, L.v, hRs, R.u, R.v, f);
            if (i == 0 && P->bc_w[j] == OR_BC_DISCHARGE) { f[0] += qb; f[1] += qb * u_in; }
            if (i == nx && P->bc_e[j] == OR_BC_DISCHARGE) { f[0] -= qb; f[1] += qb * u_in; }
            if (i > 0) {
                int64_t c = (int64_t)j * nx + i - 1;
                FE[3 * c] = f[0]; FE[3 * c + 1] = f[1] - or_press(g, hLs); FE[3 * c + 2] = f[2];
            }
            if (i < nx) {
                int64_t c = (int64_t)j * nx + i;
                FW[3 * c] = f[0]; FW[3 * c + 1] = f[1] - or_press(g, hRs); FW[3 * c + 2] = f[2];
            }
            if (i == 0) S->bflux[2 * nx + j] += f[0] * dt * dx;
            if (i == nx) S->bflux[2 * nx + ny + j] -= f[0] * dt * dx;
        }
    }
    /* y faces: face j lies between cell row j-1 and row j; normal velocity v */
    for (int32_t j = 0; j <= ny; ++j) {
        for (int32_t i = 0; i < nx; ++i) {
            or_side L, R;
            if (j == 0) { R = or_cell_side(S, i); L = or_ghost(P->bc_s[i], R, 0, h_in); }
            else L = or_cell_side(S, (int64_t)(j - 1) * nx + i);
            if (j == ny) R = or_ghost(P->bc_n[i], L, 0, h_in);
            else if (j > 0) R = or_cell_side(S, (int64_t)j * nx + i);
            double zf = L.z > R.z ? L.z : R.z;
            double hLs = L.h + L.z - zf; if (hLs < 0.0) hLs = 0.0;
            double hRs = R.h + R.z - zf; if (hRs < 0.0) hRs = 0.0;
            or_flux(P, g, hLs, L.v, L.u, hRs, R.v, R.u, f);   /* f = (mass, hv-flux, hu-flux) */
            if (j == 0 && P->bc_s[i] == OR_BC_DISCHARGE) { f[0] += qb; f[1] += qb * u_in; }
            if (j == ny && P->bc_n[i] == OR_BC_DISCHARGE) { f[0] -= qb; f[1] += qb * u_in; }
            if (j > 0) {
                int64_t c = (int64_t)(j - 1) * nx + i;
                GN[3 * c] = f[0]; GN[3 * c + 1] = f[2]; GN[3 * c + 2] = f[1] - or_press(g, hLs);
            }
            if (j < ny) {
                int64_t c = (int64_t)j * nx + i;
                GS[3 * c] = f[0]; GS[3 * c + 1] = f[2]; GS[3 * c + 2] = f[1] - or_press(g, hRs);
            }
            if (j == 0) S->bflux[i] += f[0] * dt * dx;
            if (j == ny) S->bflux[nx + i] -= f[0] * dt * dx;
        }
    }
    const double lx = dt / dx, ly = dt / dx;
    for (int64_t c = 0; c < n; ++c) {
        double h = S->h[c] - lx * (FE[3 * c] - FW[3 * c]) - ly * (GN[3 * c] - GS[3 * c]);
        double hu = S->hu[c] - lx * (FE[3 * c + 1] - FW[3 * c + 1]) - ly * (GN[3 * c + 1] - GS[3 * c + 1]);
        double hv = S->hv[c] - lx * (FE[3 * c + 2] - FW[3 * c + 2]) - ly * (GN[3 * c + 2] - GS[3 * c + 2]);
        if (h < 0.0) { S->neg_depth += 1; h = 0.0; }
        if (h <= OR_H_EPS) {
            hu = 0.0; hv = 0.0;
        } else {
            double u = hu / h, v = hv / h;
            double speed = sqrt(u * u + v * v);
            double nm = n_eff[c];
            double denom = 1.0 + dt * g * nm * nm * speed / (h * cbrt(h));
            hu = hu / denom;
            hv = hv / denom;
        }
        S->h[c] = h; S->hu[c] = hu; S->hv[c] = hv;
    }
    free(FE); free(FW); free(GN); free(GS);
}

/* ------------------------------------------------------------------------ */
/* Second order (the cited scheme at full order; a build-added option).      */
/* Per direction and cell: minmod slopes of the surface eta = h + z, of h    */
/* and of the velocities u, v -- zero on the domain edge and where the cell  */
/* or a neighbour along that direction is dry -- give face values            */
/* eta_f = eta +- s_eta/2, h_f = h +- s_h/2, z_f = eta_f - h_f, u_f, v_f.    */
/* At a face z* = max(z_L, z_R), h*_{L,R} = max(0, eta_{L,R} - z*), the same */
/* Riemann flux, and each cell takes it minus the pressure 1/2 g h*^2 of its */
/* own side (as at first order); the cell adds the centred bed-slope term    */
/* -g/2 (h_+ + h_-)(eta_+ - eta_-), in which the reconstructed pressure      */
/* difference and the bed slope between the cell's two faces combine (so a  */
/* lake at rest, eta constant, stays exactly at rest).  Time: two Euler       */
/* stages, each followed by the point-implicit friction, and the mean of the */
/* start state and the second stage's result (SSP-RK2); the second stage    */
/* takes the inflow depth of t + dt; each stage adds half its boundary      */
/* volumes.  With all slopes zero a stage is exactly the first-order step.  */
/* ------------------------------------------------------------------------ */
static double or_minmod(double a, double b) {
    if (a > 0.0 && b > 0.0) return a < b ? a : b;
    if (a < 0.0 && b < 0.0) return a > b ? a : b;
    return 0.0;
}

/* face values of one cell along one direction: minus side [0], plus side [1] */
typedef struct { double eta[2], h[2], u[2], v[2]; } or_faces;

static void or_cell_faces(const double *z, const double *h, const double *hu, const double *hv, int64_t c,
                          int64_t cm, int64_t cp, int slope, or_faces *F) {
    double hc = h[c], uc = 0.0, vc = 0.0;
    if (hc > OR_H_EPS) { uc = hu[c] / hc; vc = hv[c] / hc; }
    double eta = hc + z[c];
    double se = 0.0, sh = 0.0, su = 0.0, sv = 0.0;
    if (slope && hc > OR_H_EPS && h[cm] > OR_H_EPS && h[cp] > OR_H_EPS) {
        double um = hu[cm] / h[cm], vm = hv[cm] / h[cm], up = hu[cp] / h[cp], vp = hv[cp] / h[cp];
        se = or_minmod((h[cp] + z[cp]) - eta, eta - (h[cm] + z[cm]));
        sh = or_minmod(h[cp] - hc, hc - h[cm]);
        su = or_minmod(up - uc, uc - um);
        sv = or_minmod(vp - vc, vc - vm);
    }
    F->eta[0] = eta - 0.5 * se; F->eta[1] = eta + 0.5 * se;
    F->h[0] = hc - 0.5 * sh;    F->h[1] = hc + 0.5 * sh;
    F->u[0] = uc - 0.5 * su;    F->u[1] = uc + 0.5 * su;
    F->v[0] = vc - 0.5 * sv;    F->v[1] = vc + 0.5 * sv;
}

/* one stage: (ho, huo, hvo) = friction(U + dt L(U)) */
static void or_muscl_stage(const or_params *P, const double *z, const double *h, const double *hu, const double *hv,
                           double *ho, double *huo, double *hvo, double dt, double h_in, double qb, double u_in,
                           const double *n_eff, double *bflux, int64_t *neg) {
    const int32_t nx = P->nx, ny = P->ny;
    const int64_t n = (int64_t)nx * ny;
    const double dx = P->dx, g = P->g;
    or_faces *FX = (or_faces *)malloc(sizeof(or_faces) * (size_t)n);
    or_faces *FY = (or_faces *)malloc(sizeof(or_faces) * (size_t)n);
    for (int32_t j = 0; j < ny; ++j)
        for (int32_t i = 0; i < nx; ++i) {
            int64_t c = (int64_t)j * nx + i;
            or_cell_faces(z, h, hu, hv, c, i > 0 ? c - 1 : c, i < nx - 1 ? c + 1 : c, i > 0 && i < nx - 1, &FX[c]);
            or_cell_faces(z, h, hu, hv, c, j > 0 ? c - nx : c, j < ny - 1 ? c + nx : c, j > 0 && j < ny - 1, &FY[c]);
        }
    double *FE = (double *)calloc((size_t)n * 3, sizeof(double));
    double *FW = (double *)calloc((size_t)n * 3, sizeof(double));
    double *GN = (double *)calloc((size_t)n * 3, sizeof(double));
    double *GS = (double *)calloc((size_t)n * 3, sizeof(double));
    double f[3];
    /* x faces: face i between cell i-1 (its plus side) and cell i (its minus side) */
    for (int32_t j = 0; j < ny; ++j) {
        for (int32_t i = 0; i <= nx; ++i) {
            double eL, hL, uL, vL, eR, hR, uR, vR;
            if (i > 0) {
                const or_faces *A = &FX[(int64_t)j * nx + i - 1];
                eL = A->eta[1]; hL = A->h[1]; uL = A->u[1]; vL = A->v[1];
            }
            if (i < nx) {
                const or_faces *B = &FX[(int64_t)j * nx + i];
                eR = B->eta[0]; hR = B->h[0]; uR = B->u[0]; vR = B->v[0];
            }
            if (i == 0 || i == nx) {  /* edge cells have no slope: the ghost of the cell state */
                or_side in;
                if (i == 0) { in.h = hR; in.u = uR; in.v = vR; in.z = z[(int64_t)j * nx]; }
                else { in.h = hL; in.u = uL; in.v = vL; in.z = z[(int64_t)j * nx + nx - 1]; }
                or_side gs = or_ghost(i == 0 ? P->bc_w[j] : P->bc_e[j], in, 1, h_in);
                double ge = gs.h + gs.z;
                if (i == 0) { eL = ge; hL = gs.h; uL = gs.u; vL = gs.v; }
                else { eR = ge; hR = gs.h; uR = gs.u; vR = gs.v; }
            }
            double zL = eL - hL, zR = eR - hR;
            double zf = zL > zR ? zL : zR;
            double hLs = eL - zf; if (hLs < 0.0) hLs = 0.0;
            double hRs = eR - zf; if (hRs < 0.0) hRs = 0.0;
            or_flux(P, g, hLs, uL, vL, hRs, uR, vR, f);
            if (i == 0 && P->bc_w[j] == OR_BC_DISCHARGE) { f[0] += qb; f[1] += qb * u_in; }
            if (i == nx && P->bc_e[j] == OR_BC_DISCHARGE) { f[0] -= qb; f[1] += qb * u_in; }
            if (i > 0) {
                int64_t c = (int64_t)j * nx + i - 1;
                FE[3 * c] = f[0]; FE[3 * c + 1] = f[1] - or_press(g, hLs); FE[3 * c + 2] = f[2];
            }
            if (i < nx) {
                int64_t c = (int64_t)j * nx + i;
                FW[3 * c] = f[0]; FW[3 * c + 1] = f[1] - or_press(g, hRs); FW[3 * c + 2] = f[2];
            }
            if (i == 0) bflux[2 * nx + j] += 0.5 * f[0] * dt * dx;
            if (i == nx) bflux[2 * nx + ny + j] -= 0.5 * f[0] * dt * dx;
        }
    }
    /* y faces: face j between row j-1 (plus side) and row j (minus side); normal velocity v */
    for (int32_t j = 0; j <= ny; ++j) {
        for (int32_t i = 0; i < nx; ++i) {
            double eL, hL, uL, vL, eR, hR, uR, vR;
            if (j > 0) {
                const or_faces *A = &FY[(int64_t)(j - 1) * nx + i];
                eL = A->eta[1]; hL = A->h[1]; uL = A->u[1]; vL = A->v[1];
            }
            if (j < ny) {
                const or_faces *B = &FY[(int64_t)j * nx + i];
                eR = B->eta[0]; hR = B->h[0]; uR = B->u[0]; vR = B->v[0];
            }
            if (j == 0 || j == ny) {
                or_side in;
                if (j == 0) { in.h = hR; in.u = uR; in.v = vR; in.z = z[i]; }
                else { in.h = hL; in.u = uL; in.v = vL; in.z = z[(int64_t)(ny - 1) * nx + i]; }
                or_side gs = or_ghost(j == 0 ? P->bc_s[i] : P->bc_n[i], in, 0, h_in);
                double ge = gs.h + gs.z;
                if (j == 0) { eL = ge; hL = gs.h; uL = gs.u; vL = gs.v; }
                else { eR = ge; hR = gs.h; uR = gs.u; vR = gs.v; }
            }
            double zL = eL - hL, zR = eR - hR;
            double zf = zL > zR ? zL : zR;
            double hLs = eL - zf; if (hLs < 0.0) hLs = 0.0;
            double hRs = eR - zf; if (hRs < 0.0) hRs = 0.0;
            or_flux(P, g, hLs, vL, uL, hRs, vR, uR, f);   /* f = (mass, hv-flux, hu-flux) */
            if (j == 0 && P->bc_s[i] == OR_BC_DISCHARGE) { f[0] += qb; f[1] += qb * u_in; }
            if (j == ny && P->bc_n[i] == OR_BC_DISCHARGE) { f[0] -= qb; f[1] += qb * u_in; }
            if (j > 0) {
                int64_t c = (int64_t)(j - 1) * nx + i;
                GN[3 * c] = f[0]; GN[3 * c + 1] = f[2]; GN[3 * c + 2] = f[1] - or_press(g, hLs);
            }
            if (j < ny) {
                int64_t c = (int64_t)j * nx + i;
                GS[3 * c] = f[0]; GS[3 * c + 1] = f[2]; GS[3 * c + 2] = f[1] - or_press(g, hRs);
            }
            if (j == 0) bflux[i] += 0.5 * f[0] * dt * dx;
            if (j == ny) bflux[nx + i] -= 0.5 * f[0] * dt * dx;
        }
    }
    const double l = dt / dx;
    for (int64_t c = 0; c < n; ++c) {
        /* centred bed-slope term of each direction */
        double sx = 0.5 * g * (FX[c].h[0] + FX[c].h[1]) * (FX[c].eta[1] - FX[c].eta[0]);
        double sy = 0.5 * g * (FY[c].h[0] + FY[c].h[1]) * (FY[c].eta[1] - FY[c].eta[0]);
        double hh = h[c] - l * (FE[3 * c] - FW[3 * c]) - l * (GN[3 * c] - GS[3 * c]);
        double qx = hu[c] - l * (FE[3 * c + 1] - FW[3 * c + 1]) - l * (GN[3 * c + 1] - GS[3 * c + 1]) - l * sx;
        double qy = hv[c] - l * (FE[3 * c + 2] - FW[3 * c + 2]) - l * (GN[3 * c + 2] - GS[3 * c + 2]) - l * sy;
        if (hh < 0.0) { *neg += 1; hh = 0.0; }
        if (hh <= OR_H_EPS) {
            qx = 0.0; qy = 0.0;
        } else {
            double u = qx / hh, v = qy / hh;
            double speed = sqrt(u * u + v * v);
            double nm = n_eff[c];
            double denom = 1.0 + dt * g * nm * nm * speed / (hh * cbrt(hh));
            qx = qx / denom;
            qy = qy / denom;
        }
        ho[c] = hh; huo[c] = qx; hvo[c] = qy;
    }
    free(FE); free(FW); free(GN); free(GS); free(FX); free(FY);
}

void or_flood_step2(const or_params *P, or_state *S, int64_t dt_ticks, const double *n_eff) {
    const int64_t n = (int64_t)P->nx * P->ny;
    const double dt = (double)dt_ticks / OR_TICKS;
    double qb = 0.0, u_in = 0.0;
    {
        const double B = or_discharge_width(P);
        const double t0 = (double)S->t_ticks / OR_TICKS, t1 = (double)(S->t_ticks + dt_ticks) / OR_TICKS;
        if (B > 0.0 && dt > 0.0) {
            qb = (or_discharge_volume(P, t1) - or_discharge_volume(P, t0)) / (dt * B);
            u_in = qb / P->h_qin;
        }
    }
    double *b1 = (double *)malloc(sizeof(double) * (size_t)n * 6);
    double *h1 = b1, *hu1 = b1 + n, *hv1 = b1 + 2 * n, *h2 = b1 + 3 * n, *hu2 = b1 + 4 * n, *hv2 = b1 + 5 * n;
    or_muscl_stage(P, S->z, S->h, S->hu, S->hv, h1, hu1, hv1, dt, or_hydro_depth(P, S->t_ticks), qb, u_in, n_eff,
                   S->bflux, &S->neg_depth);
    or_muscl_stage(P, S->z, h1, hu1, hv1, h2, hu2, hv2, dt, or_hydro_depth(P, S->t_ticks + dt_ticks), qb, u_in,
                   n_eff, S->bflux, &S->neg_depth);
    for (int64_t c = 0; c < n; ++c) {
        double h = 0.5 * (S->h[c] + h2[c]);
        double hu = 0.5 * (S->hu[c] + hu2[c]), hv = 0.5 * (S->hv[c] + hv2[c]);
        if (h <= OR_H_EPS) { hu = 0.0; hv = 0.0; }
        S->h[c] = h; S->hu[c] = hu; S->hv[c] = hv;
    }
    free(b1);
}

/* ------------------------------------------------------------------------ */
/* Pedestrian step (Sections 2.3-2.4) from the state at step n.             */
/* ------------------------------------------------------------------------ */
static int or_walkable_at(const or_params *P, double x, double y) {
    float dxf = (float)P->dx;
    int32_t i = or_cell_index(x, dxf), j = or_cell_index(y, dxf);
    if (i < 0 || j < 0 || i >= P->nx || j >= P->ny) return 0;
    return P->walkable[(int64_t)j * P->nx + i] != 0;
}

int32_t or_bags_per_cell(double dx) { return (int32_t)ceil((dx * dx) / (OR_BAG_L * OR_BAG_W)); }

enum { G_NONE = 0, G_EXIT = 1, G_DEPOT = 2, G_BARRIER = 3, G_STRAIGHT = 4, G_DOOR = 5 };

/* h, hu, hv are the flood state at step n (the step's input) */
int64_t or_ped_step(const or_params *P, or_state *S, int64_t dt_ticks, int32_t wet, int64_t bags_snap,
                    const double *h, const double *hu, const double *hv) {
    const int32_t np = S->np, nx = P->nx;
    const float dxf = (float)P->dx;
    const double dx = P->dx;
    const double dt = (double)dt_ticks / OR_TICKS;
    const int32_t bpc = or_bags_per_cell(dx);
    const int64_t cap = (int64_t)P->n_barrier * P->n_layers * bpc;
    int64_t drops = 0;
    double *nxp = (double *)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1) * 4);
    double *nyp = nxp + np, *nvx = nxp + 2 * (size_t)np, *nvy = nxp + 3 * (size_t)np;
    uint8_t *nfsm = (uint8_t *)malloc((size_t)(np > 0 ? np : 1) * 3);
    uint8_t *nhr = nfsm + np, *nex = nfsm + 2 * (size_t)np;
    int32_t *ntim = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
    for (int32_t p = 0; p < np; ++p) {
        nxp[p] = S->px[p]; nyp[p] = S->py[p]; nvx[p] = S->pvx[p]; nvy[p] = S->pvy[p];
        nfsm[p] = S->pfsm[p]; nhr[p] = S->phr[p]; nex[p] = S->pexit[p]; ntim[p] = S->ptimer[p];
    }
    for (int32_t p = 0; p < np; ++p) {
        if (S->pexit[p]) continue;
        const double x = S->px[p], y = S->py[p];
        const int32_t ci = or_cell_index(x, dxf), cj = or_cell_index(y, dxf);
        const int64_t c = (int64_t)cj * nx + ci;
        /* Table 1: flood-risk state and walking speed */
        const int hr = or_hr_state((float)h[c], (float)hu[c], (float)hv[c]);
        double speed = hr == OR_DRY ? S->pv0[p] : OR_SPEED[hr];
        int goal = G_NONE;
        int32_t target = -1;
        uint8_t fsm = S->pfsm[p];
        int32_t timer = S->ptimer[p];
        int32_t door = -1;
        if (S->prole[p] == OR_EVAC) {
            /* before the trigger a visitor walks to its door; once water is seen
             * (or with no trigger) every evacuee heads for the exit */
            if (P->evac_trigger == 0 || wet) {
                goal = G_EXIT;
                fsm = 0;
            } else if (fsm >= OR_VISIT0 && fsm - OR_VISIT0 < P->n_doors) {
                goal = G_DOOR;
                door = fsm - OR_VISIT0;
            }
        } else {
            if (fsm != OR_DONE && bags_snap >= cap) fsm = OR_DONE;
            switch (fsm) {
            case OR_DONE:
                goal = G_EXIT;
                break;
            case OR_TO_DEPOT:
                if (S->nav_depot[c] == OR_AT_GOAL) { fsm = OR_PICKUP; timer = OR_T_PICK; }
                else goal = G_DEPOT;
                break;
            case OR_PICKUP:
                timer = (int32_t)(timer - dt_ticks);
                if (timer <= 0) { fsm = OR_TO_BARRIER; timer = 0; }
                break;
            case OR_TO_BARRIER: {
                target = P->barrier_cells[(bags_snap / bpc) % P->n_barrier];
                if (c == target) { fsm = OR_DROP; timer = OR_T_DROP; }
                else if (S->nav_barrier[c] == OR_AT_GOAL) goal = G_STRAIGHT;
                else goal = G_BARRIER;
                break;
            }
            case OR_DROP:
                timer = (int32_t)(timer - dt_ticks);
                if (timer <= 0) { drops += 1; fsm = OR_TO_DEPOT; timer = 0; }
                break;
            default:
                break;
            }
        }
        /* a responder picking up or dropping a bag stands still for the wait */
        if (S->prole[p] == OR_RESP && (fsm == OR_PICKUP || fsm == OR_DROP)) speed = 0.0;
        /* desired velocity: toward the centre of the next cell on the navigation map
         * (or straight to the barrier cell being filled), plus a small random term;
         * when that cell is the destination, no faster than reaching its centre in dt */
        double ex = 0.0, ey = 0.0, sdes = speed;
        if (goal != G_NONE) {
            double tx = 0.0, ty = 0.0;
            int have = 0, arriving = 0;
            if (goal == G_STRAIGHT) {
                tx = ((double)(target % nx) + 0.5) * dx;
                ty = ((double)(target / nx) + 0.5) * dx;
                have = 1;
                arriving = 1;
            } else {
                const uint8_t *nav = goal == G_EXIT ? S->nav_exit : goal == G_DEPOT ? S->nav_depot
                                     : goal == G_BARRIER ? S->nav_barrier
                                     : S->nav_door + (int64_t)door * P->nx * P->ny;
                uint8_t code = nav[c];
                if (code < 8) {
                    int32_t ti = ci + OR_OX[code], tj = cj + OR_OY[code];
                    tx = ((double)ti + 0.5) * dx;
                    ty = ((double)tj + 0.5) * dx;
                    have = 1;
                    arriving = nav[(int64_t)tj * nx + ti] == OR_AT_GOAL;
                }
            }
            if (have) {
                double ddx = tx - x, ddy = ty - y;
                double len = sqrt(ddx * ddx + ddy * ddy);
                if (len > 0.0) { ex = ddx / len; ey = ddy / len; }
                if (arriving && dt > 0.0 && len / dt < sdes) sdes = len / dt;
            }
        }
        double vdx = 0.0, vdy = 0.0;
        if (goal != G_NONE && speed > 0.0) {
            uint64_t ctr[4] = {(uint64_t)S->pid[p], (uint64_t)S->step, 0, 0}, key[2] = {P->seed, 0}, r[4];
            or_philox4x64(ctr, key, r);
            vdx = sdes * ex + P->ped_noise * (or_uniform24(r[0]) - 0.5);
            vdy = sdes * ey + P->ped_noise * (or_uniform24(r[1]) - 0.5);
        }
        /* repulsion from every other present pedestrian within the neighbour radius */
        double Fx = 0.0, Fy = 0.0;
        const double vdn = sqrt(vdx * vdx + vdy * vdy);
        for (int32_t q = 0; q < np; ++q) {
            if (q == p || S->pexit[q]) continue;
            double rx = x - S->px[q], ry = y - S->py[q];
            if (fabs(rx) >= OR_R || fabs(ry) >= OR_R) continue;
            double d2 = rx * rx + ry * ry;
            if (d2 >= OR_R * OR_R || d2 <= 0.0) continue;
            double d = sqrt(d2);
            /* exponential repulsion shifted to vanish at the neighbour radius */
            double fm = OR_A * (exp((2.0 * OR_RB - d) / OR_B) - exp((2.0 * OR_RB - OR_R) / OR_B));
            Fx += fm * rx / d;
            Fy += fm * ry / d;
            /* walking toward the neighbour: part of the push turns to the walker's right,
             * weighted by the cosine of the approach angle (continuous in every input) */
            if (vdn > 0.0) {
                double w = -(vdx * rx + vdy * ry) / (vdn * d);
                if (w > 0.0) {
                    Fx += OR_SIDE * w * fm * (-ry / d);
                    Fy += OR_SIDE * w * fm * (rx / d);
                }
            }
        }
        /* relaxation toward the desired velocity, capped at the state's speed */
        double a = dt / OR_TAU; if (a > 1.0) a = 1.0;
        double vx = S->pvx[p] + a * (vdx - S->pvx[p]) + dt * Fx;
        double vy = S->pvy[p] + a * (vdy - S->pvy[p]) + dt * Fy;
        if (speed <= 0.0) { vx = 0.0; vy = 0.0; }
        else {
            double sp = sqrt(vx * vx + vy * vy);
            if (sp > speed) { vx = vx * (speed / sp); vy = vy * (speed / sp); }
        }
        /* move, sliding along non-walkable cells */
        double xn = x + dt * vx, yn = y + dt * vy;
        if (or_walkable_at(P, xn, yn)) { }
        else if (or_walkable_at(P, xn, y)) { yn = y; vy = 0.0; }
        else if (or_walkable_at(P, x, yn)) { xn = x; vx = 0.0; }
        else { xn = x; yn = y; vx = 0.0; vy = 0.0; }
        /* through the emergency exit (1), or a visitor in a cell of its door (2) */
        uint8_t exited = 0;
        {
            int32_t ii = or_cell_index(xn, dxf), jj = or_cell_index(yn, dxf);
            int64_t cn = (int64_t)jj * nx + ii;
            if (goal == G_EXIT && P->exit_mask[cn]) exited = 1;
            if (goal == G_DOOR && S->nav_door[(int64_t)door * P->nx * P->ny + cn] == OR_AT_GOAL) exited = 2;
        }
        nxp[p] = xn; nyp[p] = yn; nvx[p] = vx; nvy[p] = vy;
        nfsm[p] = fsm; ntim[p] = timer; nhr[p] = (uint8_t)hr; nex[p] = exited;
        S->hist[hr] += 1;
        if (exited == 1) S->n_exited += 1;
        if (exited == 2) S->n_left += 1;
    }
    for (int32_t p = 0; p < np; ++p) {
        S->px[p] = nxp[p]; S->py[p] = nyp[p]; S->pvx[p] = nvx[p]; S->pvy[p] = nvy[p];
        S->pfsm[p] = nfsm[p]; S->phr[p] = nhr[p]; S->pexit[p] = nex[p]; S->ptimer[p] = ntim[p];
    }
    free(nxp); free(nfsm); free(ntim);
    return drops;
}

/* ------------------------------------------------------------------------ */
/* Navigation fields for the three destinations.                             */
/* ------------------------------------------------------------------------ */
void or_prepare(const or_params *P, or_state *S) {
    int64_t n = (int64_t)P->nx * P->ny;
    uint8_t *goal = (uint8_t *)calloc((size_t)n, 1);
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    or_nav_field(P->nx, P->ny, P->walkable, P->exit_mask, S->nav_exit, dist);
    memset(goal, 0, (size_t)n);
    for (int k = 0; k < P->n_depot; ++k) goal[P->depot_cells[k]] = 1;
    or_nav_field(P->nx, P->ny, P->walkable, goal, S->nav_depot, dist);
    memset(goal, 0, (size_t)n);
    for (int k = 0; k < P->n_barrier; ++k) goal[P->barrier_cells[k]] = 1;
    or_nav_field(P->nx, P->ny, P->walkable, goal, S->nav_barrier, dist);
    for (int d = 0; d < P->n_doors; ++d) {
        memset(goal, 0, (size_t)n);
        for (int k = 0; k < P->n_door_cells; ++k)
            if (P->door_of[k] == d) goal[P->door_cells[k]] = 1;
        or_nav_field(P->nx, P->ny, P->walkable, goal, S->nav_door + (int64_t)d * n, dist);
    }
    free(goal);
    free(dist);
}

/* ------------------------------------------------------------------------ */
/* Entry flow (Sections 3, 3.2): while the evacuation trigger has not fired,  */
/* every door admits one visitor at each whole multiple of the entry period  */
/* in the step's interval (t, t + dt]; the step's visitors take the next ids */
/* door by door; each stands at rest at its draws' position in its door's   */
/* entry cell, bound for the drawn door.  Past the array capacity a visitor  */
/* is refused (counted).  t >= 0.                                            */
/* ------------------------------------------------------------------------ */
static void or_entries(const or_params *P, or_state *S, int64_t t, int64_t dt_ticks, int32_t wet) {
    if (P->n_doors <= 0 || P->evac_trigger == 0 || wet || dt_ticks <= 0) return;
    const int64_t T = P->entry_period_ticks;
    const float dxf = (float)P->dx;
    for (int32_t d = 0; d < P->n_doors; ++d) {
        int32_t cell = -1;
        for (int32_t k = 0; k < P->n_door_cells && cell < 0; ++k)
            if (P->door_of[k] == d) cell = P->door_cells[k];
        const int64_t count = (t + dt_ticks) / T - t / T;
        for (int64_t m = 0; m < count; ++m) {
            if (S->np >= S->cap) { S->entry_refused += 1; continue; }
            const int32_t p = S->np;
            float off[3];
            int32_t dest;
            or_visitor_draw(P->seed, (uint64_t)p, P->n_doors, (float)P->entry_v0_lo, (float)P->entry_v0_hi, off,
                            &dest);
            S->px[p] = (double)(((float)(cell % P->nx) + off[0]) * dxf);
            S->py[p] = (double)(((float)(cell / P->nx) + off[1]) * dxf);
            S->pvx[p] = 0.0; S->pvy[p] = 0.0;
            S->pv0[p] = (double)off[2];
            S->pid[p] = p;
            S->ptimer[p] = 0;
            S->prole[p] = OR_EVAC;
            S->pfsm[p] = (uint8_t)(OR_VISIT0 + dest);
            S->phr[p] = 0;
            S->pexit[p] = 0;
            S->np += 1;
            S->n_entered += 1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* One coupled step.  Both agent types advance from the state at step n     */
/* ("simultaneous update of multiple agent types"): the flood update uses   */
/* z^n and n_M from the evacuees at step n; pedestrians read h, u, v at     */
/* step n; sandbags dropped in step n raise z before step n+1.              */
/* Returns the step's dt in ticks (0 once t_end is reached).                */
/* ------------------------------------------------------------------------ */
int64_t or_step(const or_params *P, or_state *S) {
    if (S->t_ticks >= P->t_end_ticks) { S->last_dt_ticks = 0; return 0; }
    const int32_t nx = P->nx;
    const int64_t n = (int64_t)P->nx * P->ny;
    const float dxf = (float)P->dx;
    /* completed sandbag cell-layers raise their cell's bed by one bag thickness */
    if (P->n_barrier > 0 && P->n_layers > 0) {
        int64_t bpc = or_bags_per_cell(P->dx);
        int64_t done = S->total_bags / bpc;
        int64_t cap = (int64_t)P->n_barrier * P->n_layers;
        if (done > cap) done = cap;
        for (int64_t k = S->applied_layers; k < done; ++k) S->z[P->barrier_cells[k % P->n_barrier]] += OR_BAG_T;
        S->applied_layers = done;
    }
    const int64_t bags_snap = S->total_bags;
    for (int k = 0; k < 5; ++k) S->hist[k] = 0;   /* hazard-state counts of this step */
    /* evacuees per cell -> Manning n (Section 2.4) */
    double *n_eff = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *occ = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    for (int32_t p = 0; p < S->np; ++p) {
        if (S->pexit[p] || S->prole[p] != OR_EVAC) continue;
        int32_t i = or_cell_index(S->px[p], dxf), j = or_cell_index(S->py[p], dxf);
        occ[(int64_t)j * nx + i] += 1;
    }
    for (int64_t c = 0; c < n; ++c) {
        int32_t np_c = occ[c] < OR_NP_CAP ? occ[c] : OR_NP_CAP;
        n_eff[c] = P->coupling ? P->n0[c] + (double)np_c * P->n0[c] : P->n0[c];
    }
    const int64_t dt_ticks = or_dt_ticks(P, S->h, S->hu, S->hv, S->t_ticks);
    /* evacuation trigger: any cell with water at step n (sticky) */
    if (!S->wet) {
        for (int64_t c = 0; c < n; ++c) if ((float)S->h[c] >= OR_H_DRY_F) { S->wet = 1; break; }
    }
    double *h0 = (double *)malloc(sizeof(double) * (size_t)n * 3);
    memcpy(h0, S->h, sizeof(double) * (size_t)n);
    memcpy(h0 + n, S->hu, sizeof(double) * (size_t)n);
    memcpy(h0 + 2 * n, S->hv, sizeof(double) * (size_t)n);
    if (P->order == 2) or_flood_step2(P, S, dt_ticks, n_eff);
    else or_flood_step(P, S, dt_ticks, n_eff);
    int64_t drops = or_ped_step(P, S, dt_ticks, S->wet, bags_snap, h0, h0 + n, h0 + 2 * n);
    or_entries(P, S, S->t_ticks, dt_ticks, S->wet);
    S->total_bags += drops;
    S->t_ticks += dt_ticks;
    S->step += 1;
    S->last_dt_ticks = dt_ticks;
    free(h0); free(n_eff); free(occ);
    return dt_ticks;
}

int64_t or_run(const or_params *P, or_state *S, int64_t n_steps) {
    int64_t k = 0;
    for (; k < n_steps; ++k) {
        if (or_step(P, S) == 0) break;
    }
    return k;
}

/* Largest hazard rating HR = (max(|u|,|v|) + 0.5) h over the cells holding
 * water (h > h_eps), in FP32 from the FP32-rounded state (Section 2.4; the
 * time history of this maximum is Fig. 5(b)'s severity measure). */
float or_max_hr(const or_params *P, const or_state *S) {
    float m = 0.0f;
    int64_t n = (int64_t)P->nx * P->ny;
    for (int64_t c = 0; c < n; ++c) {
        float h = (float)S->h[c];
        if (!(h > (float)OR_H_EPS)) continue;
        float u = (float)S->hu[c] / h, v = (float)S->hv[c] / h;
        float hr = (fmaxf(fabsf(u), fabsf(v)) + 0.5f) * h;
        if (hr > m) m = hr;
    }
    return m;
}

double or_mass(const or_params *P, const or_state *S) {
    double m = 0.0;
    int64_t n = (int64_t)P->nx * P->ny;
    for (int64_t c = 0; c < n; ++c) m += S->h[c] * P->dx * P->dx;
    return m;
}

/* ------------------------------------------------------------------------ */
/* The learned surrogate's guard (build-added, not the paper's method): the  */
/* per-tile mass residual |dV - F| / max(V0, 1 cm x tile area) of a window   */
/* [t0, t1] whose start state is (h0, hu0, hv0) and end state (h1, hu1,      */
/* hv1): dV the change of the tile's water volume, F the window length times */
/* the mean of the water flowing in through the tile's edges in the start   */
/* and end states, each the HLL mass flux after the hydrostatic              */
/* reconstruction (ghost states at domain edges, with the inflow depth of    */
/* t0, resp. t1).  Tile: cells [x0, x1) x [y0, y1).                          */
/* ------------------------------------------------------------------------ */
static or_side or_side_arrays(const double *h, const double *hu, const double *hv, const double *z, int64_t c) {
    or_side s;
    s.h = h[c];
    s.z = z[c];
    if (s.h > OR_H_EPS) { s.u = hu[c] / s.h; s.v = hv[c] / s.h; }
    else { s.u = 0.0; s.v = 0.0; }
    return s;
}

static double or_face_mass(double g, or_side L, or_side R, int xface) {
    double zf = L.z > R.z ? L.z : R.z;
    double hL = L.h + L.z - zf; if (hL < 0.0) hL = 0.0;
    double hR = R.h + R.z - zf; if (hR < 0.0) hR = 0.0;
    double f[3];
    if (xface) or_hll(g, hL, L.u, L.v, hR, R.u, R.v, f);
    else or_hll(g, hL, L.v, L.u, hR, R.v, R.u, f);
    return f[0];
}

/* water flowing into the tile through its edges per unit time (m^3/s / dx) */
static double or_tile_inflow(const or_params *P, const double *z, const double *h, const double *hu,
                             const double *hv, int32_t x0, int32_t x1, int32_t y0, int32_t y1, double h_in) {
    const int32_t nx = P->nx, ny = P->ny;
    double q = 0.0;
    for (int32_t j = y0; j < y1; ++j) {
        /* west edge: face between x0 - 1 and x0 */
        or_side R = or_side_arrays(h, hu, hv, z, (int64_t)j * nx + x0), L;
        if (x0 == 0) L = or_ghost(P->bc_w[j], R, 1, h_in);
        else L = or_side_arrays(h, hu, hv, z, (int64_t)j * nx + x0 - 1);
        q += or_face_mass(P->g, L, R, 1);
        /* east edge: face between x1 - 1 and x1 */
        L = or_side_arrays(h, hu, hv, z, (int64_t)j * nx + x1 - 1);
        if (x1 == nx) R = or_ghost(P->bc_e[j], L, 1, h_in);
        else R = or_side_arrays(h, hu, hv, z, (int64_t)j * nx + x1);
        q -= or_face_mass(P->g, L, R, 1);
    }
    for (int32_t i = x0; i < x1; ++i) {
        /* south edge: face between y0 - 1 and y0 */
        or_side A = or_side_arrays(h, hu, hv, z, (int64_t)y0 * nx + i), B;
        if (y0 == 0) B = or_ghost(P->bc_s[i], A, 0, h_in);
        else B = or_side_arrays(h, hu, hv, z, (int64_t)(y0 - 1) * nx + i);
        q += or_face_mass(P->g, B, A, 0);
        /* north edge: face between y1 - 1 and y1 */
        B = or_side_arrays(h, hu, hv, z, (int64_t)(y1 - 1) * nx + i);
        if (y1 == ny) A = or_ghost(P->bc_n[i], B, 0, h_in);
        else A = or_side_arrays(h, hu, hv, z, (int64_t)y1 * nx + i);
        q -= or_face_mass(P->g, B, A, 0);
    }
    return q;
}

double or_guard_residual(const or_params *P, const double *z, const double *h0, const double *hu0,
                         const double *hv0, const double *h1, const double *hu1, const double *hv1, int32_t x0,
                         int32_t x1, int32_t y0, int32_t y1, int64_t t0_ticks, int64_t t1_ticks) {
    const int32_t nx = P->nx;
    const double dx = P->dx;
    double v0 = 0.0, v1 = 0.0;
    for (int32_t j = y0; j < y1; ++j)
        for (int32_t i = x0; i < x1; ++i) {
            v0 += h0[(int64_t)j * nx + i];
            v1 += h1[(int64_t)j * nx + i];
        }
    const double q0 = or_tile_inflow(P, z, h0, hu0, hv0, x0, x1, y0, y1, or_hydro_depth(P, t0_ticks));
    const double q1 = or_tile_inflow(P, z, h1, hu1, hv1, x0, x1, y0, y1, or_hydro_depth(P, t1_ticks));
    const double window = (double)(t1_ticks - t0_ticks) / OR_TICKS;
    const double dV = (v1 - v0) * dx * dx;
    const double F = window * dx * 0.5 * (q0 + q1);
    const double area = (double)(x1 - x0) * (double)(y1 - y0) * dx * dx;
    const double denom = v0 * dx * dx > 0.01 * area ? v0 * dx * dx : 0.01 * area;
    return fabs(dV - F) / denom;
}

/* ------------------------------------------------------------------------ */
/* Learned surrogate (build-added, not in the paper): a stack of 3x3 "valid" */
/* convolutions over NHWC tensors in FP64, with ReLU between layers, and the */
/* gradients of the mean squared error of its output.  Plain loops in the    */
/* definition's order.                                                       */
/* ------------------------------------------------------------------------ */

/* y[i][j][co] = b[co] + sum_{ky,kx,ci} x[i+ky][j+kx][ci] * w[ky][kx][ci][co],
 * x: H x W x Ci, y: (H-2) x (W-2) x Co; relu != 0 clamps y at 0. */
void or_conv3x3(const double *x, int H, int W, int Ci, const double *w, const double *b, int Co, double *y,
                int relu) {
    const int Ho = H - 2, Wo = W - 2;
    for (int i = 0; i < Ho; ++i)
        for (int j = 0; j < Wo; ++j)
            for (int co = 0; co < Co; ++co) {
                double acc = b[co];
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx)
                        for (int ci = 0; ci < Ci; ++ci)
                            acc += x[((size_t)(i + ky) * W + (j + kx)) * Ci + ci] *
                                   w[((size_t)(ky * 3 + kx) * Ci + ci) * Co + co];
                if (relu && acc < 0.0) acc = 0.0;
                y[((size_t)i * Wo + j) * Co + co] = acc;
            }
}

/* Gradients of a conv layer (pre-activation output y): given dy (Ho x Wo x Co),
 * accumulate dx (H x W x Ci, may be NULL), dw and db. */
void or_conv3x3_backward(const double *x, int H, int W, int Ci, const double *w, int Co, const double *dy,
                         double *dx, double *dw, double *db) {
    const int Ho = H - 2, Wo = W - 2;
    for (int i = 0; i < Ho; ++i)
        for (int j = 0; j < Wo; ++j)
            for (int co = 0; co < Co; ++co) {
                const double g = dy[((size_t)i * Wo + j) * Co + co];
                db[co] += g;
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx)
                        for (int ci = 0; ci < Ci; ++ci) {
                            const size_t xi = ((size_t)(i + ky) * W + (j + kx)) * Ci + ci;
                            const size_t wi = ((size_t)(ky * 3 + kx) * Ci + ci) * Co + co;
                            dw[wi] += g * x[xi];
                            if (dx) dx[xi] += g * w[wi];
                        }
            }
}

/* v rounded to FP32 and then to the nearest BF16 (8-bit significand, ties to
 * even), the storage format of the product's hidden activations.             */
static double or_round_bf16(double v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, sizeof(u));
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    memcpy(&f, &u, sizeof(f));
    return (double)f;
}

/* Forward through L layers (channels ch[0..L]); acts receives every layer's
 * output (post-ReLU except the last), laid out one after another.  Returns the
 * final output pointer inside acts.  act_bf16 != 0 stores each hidden layer's
 * output rounded to BF16 (the tensor-core path keeps activations in BF16), so
 * that comparisons with it see the same ReLU decisions; 0 is the plain FP64
 * net. */
double *or_net_forward(const double *x, int H, int W, int L, const int *ch, const double *const *ws,
                       const double *const *bs, double *acts, int act_bf16) {
    const double *in = x;
    double *out = acts;
    int h = H, w = W;
    for (int l = 0; l < L; ++l) {
        or_conv3x3(in, h, w, ch[l], ws[l], bs[l], ch[l + 1], out, l + 1 < L);
        const size_t n = (size_t)(h - 2) * (w - 2) * ch[l + 1];
        if (act_bf16 && l + 1 < L)
            for (size_t k = 0; k < n; ++k) out[k] = or_round_bf16(out[k]);
        in = out;
        h -= 2; w -= 2;
        out += n;
    }
    return (double *)in;
}

/* Loss = mean over the final output of (out - target)^2; fills dws/dbs
 * (zeroed first) with its gradients.  scratch holds 2 x the largest activation. */
double or_net_loss_grad(const double *x, int H, int W, int L, const int *ch, const double *const *ws,
                        const double *const *bs, const double *target, double *acts, double *const *dws,
                        double *const *dbs, double *scratch, size_t scratch_len, int act_bf16) {
    size_t off[16];
    int hs[17], wsz[17];
    hs[0] = H; wsz[0] = W;
    size_t o = 0;
    for (int l = 0; l < L; ++l) {
        off[l] = o;
        hs[l + 1] = hs[l] - 2; wsz[l + 1] = wsz[l] - 2;
        o += (size_t)hs[l + 1] * wsz[l + 1] * ch[l + 1];
    }
    const double *out = or_net_forward(x, H, W, L, ch, ws, bs, acts, act_bf16);
    const size_t n_out = (size_t)hs[L] * wsz[L] * ch[L];
    double loss = 0.0;
    double *g = scratch, *g2 = scratch + scratch_len / 2;
    for (size_t k = 0; k < n_out; ++k) {
        const double d = out[k] - target[k];
        loss += d * d;
        g[k] = 2.0 * d / (double)n_out;
    }
    loss /= (double)n_out;
    for (int l = L - 1; l >= 0; --l) {
        const size_t nw = (size_t)9 * ch[l] * ch[l + 1];
        memset(dws[l], 0, nw * sizeof(double));
        memset(dbs[l], 0, (size_t)ch[l + 1] * sizeof(double));
        const double *xin = l == 0 ? x : acts + off[l - 1];
        const size_t nin = (size_t)hs[l] * wsz[l] * ch[l];
        if (l > 0) memset(g2, 0, nin * sizeof(double));
        or_conv3x3_backward(xin, hs[l], wsz[l], ch[l], ws[l], ch[l + 1], g, l > 0 ? g2 : NULL, dws[l], dbs[l]);
        if (l > 0) {
            /* through the ReLU of layer l-1's output */
            for (size_t k = 0; k < nin; ++k) g[k] = xin[k] > 0.0 ? g2[k] : 0.0;
        }
    }
    return loss;
}
