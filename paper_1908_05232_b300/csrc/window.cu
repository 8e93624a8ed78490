// window.cu -- device side of the surrogate window (build-added; the paper has
// no surrogate): dry-tile classification, the net's BF16 input tiles, applying
// the predicted change with the per-tile mass guard, the evacuee counts of the
// plain fallback, the plain-check difference and the merge of recomputed
// tiles.  The window's order of work is in floodped.cu (fp_surrogate_advance).
#include <cuda_bf16.h>

#include <algorithm>

#include "flood_dev.cuh"
#include "floodped.h"

namespace {
using namespace fpdev;

constexpr int kT = FP_SUR_TILE;
constexpr int kHalo = FP_SUR_HALO;
constexpr int kIn = kT + 2 * kHalo;
constexpr int kWin = FP_SUR_WINDOW;

// The clock of a step whose flood update moves no water: slot + 1 gets
// t + dt, the step index, the inflow depth and the sticky wet flag; slot + 2 is
// cleared for reuse (as the flood tile (0, 0) does in a plain step).
__global__ void clock_advance_kernel(const __grid_constant__ FpSim S, int slot) {
    const FpClock c = S.clock[slot];
    const long long dt = fp_dt_ticks(S, c, c.h_in);
    FpClock *nxt = &S.clock[(slot + 1) & 3];
    const long long t1 = c.t + dt;
    nxt->t = t1;
    nxt->step = c.step + (dt > 0 ? 1 : 0);
    nxt->h_in = (float)fp_hydro_depth(S, t1);
    nxt->q_speed = fp_discharge_speed(S, t1);
    nxt->smax_bits = c.smax_bits;
    nxt->wet = c.wet;
    FpClock *old = &S.clock[(slot + 2) & 3];
    old->smax_bits = 0u;
    old->wet = 0;
}

// Largest inflow depth of the hydrograph over [t0, t1] (its breakpoints inside
// and both ends; the table is piecewise linear).
__device__ double max_inflow_depth(const FpSim &S, long long t0, long long t1) {
    double m = fmax(fp_hydro_depth(S, t0), fp_hydro_depth(S, t1));
    const double a = (double)t0 / 1048576.0, b = (double)t1 / 1048576.0;
    for (int k = 0; k < S.n_hydro; ++k)
        if (S.hydro_t[k] > a && S.hydro_t[k] < b) m = fmax(m, S.hydro_h[k]);
    return m;
}

// One CTA per tile: wet[tile] = 1 when the tile grown by kWin cells holds a cell
// with h != 0, or reaches an inflow edge cell while the inflow depth over the
// window is positive.
__global__ void __launch_bounds__(256) classify_kernel(const __grid_constant__ FpSim S, int par,
                                                       const FpClock *c0, int tiles_x, unsigned char *wet) {
    const int tile = blockIdx.x, tx = tile % tiles_x, ty = tile / tiles_x;
    const int xa = max(0, tx * kT - kWin), xb = min(S.nx, (tx + 1) * kT + kWin);
    const int ya = max(0, ty * kT - kWin), yb = min(S.ny, (ty + 1) * kT + kWin);
    const int w = xb - xa, n = w * (yb - ya);
    int found = 0;
    for (int k = threadIdx.x; k < n && !found; k += blockDim.x) {
        const int i = xa + k % w, j = ya + k / w;
        if (S.h[par][fp_pidx(S, i, j)] != 0.0f) found = 1;
    }
    if (S.has_inflow) {
        const long long t0 = c0->t, t1 = t0 + (long long)kWin * S.dt_fixed;
        if (max_inflow_depth(S, t0, t1) > 0.0) {
            for (int i = xa + (int)threadIdx.x; i < xb; i += blockDim.x) {
                if (ya == 0 && S.bc[0][i] == FP_BC_INFLOW) found = 1;
                if (yb == S.ny && S.bc[1][i] == FP_BC_INFLOW) found = 1;
            }
            for (int j = ya + (int)threadIdx.x; j < yb; j += blockDim.x) {
                if (xa == 0 && S.bc[2][j] == FP_BC_INFLOW) found = 1;
                if (xb == S.nx && S.bc[3][j] == FP_BC_INFLOW) found = 1;
            }
        }
    }
    found = __syncthreads_or(found);
    if (threadIdx.x == 0) wet[tile] = found ? 1 : 0;
}

// One CTA: list of wet tiles in tile order, batch_of[tile] = its index or -1.
__global__ void __launch_bounds__(1024) compact_kernel(const unsigned char *flags, int n, int *list, int *batch_of,
                                                       int *count) {
    __shared__ int s_w[32];
    __shared__ int s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c0 = 0; c0 < n; c0 += 1024) {
        const int t = c0 + (int)threadIdx.x;
        const int v = t < n && flags[t] ? 1 : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        if (lane == 0) s_w[wid] = __popc(bal);
        __syncthreads();
        int pre = 0, tot = 0;
        for (int k = 0; k < 32; ++k) {
            pre += k < wid ? s_w[k] : 0;
            tot += s_w[k];
        }
        const int idx = s_base + pre + __popc(bal & ((1u << lane) - 1u));
        if (t < n) {
            batch_of[t] = v ? idx : -1;
            if (v) list[idx] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = s_base;
}

// Net input: per listed tile a kIn x kIn image of (h, hu, hv, z) as BF16 values
// and remainders (fp_sur_pack_pixel), cells past the domain edge repeating the
// edge cell.
__global__ void input_kernel(const __grid_constant__ FpSim S, const float *__restrict__ h,
                             const float *__restrict__ hu, const float *__restrict__ hv, const int *__restrict__ list,
                             int count, int tiles_x, __nv_bfloat16 *__restrict__ out) {
    const long long total = (long long)count * kIn * kIn;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(p / (kIn * kIn));
        const int rc = (int)(p % (kIn * kIn));
        const int r = rc / kIn, c = rc % kIn;
        const int tile = list[b];
        const int i = min(max((tile % tiles_x) * kT - kHalo + c, 0), S.nx - 1);
        const int j = min(max((tile / tiles_x) * kT - kHalo + r, 0), S.ny - 1);
        const size_t o = fp_pidx(S, i, j);
        constexpr int kP = fp_sur_pitch(kIn);
        __nv_bfloat16 *g0 = out + (((size_t)(b * kIn + r) * 2) * kP + c) * 8;
        fp_sur_pack_pixel(h[o], hu[o], hv[o], S.z[o], g0, g0 + kP * 8);
    }
}

struct Cell {
    float h, hu, hv;
};

// U + dU with h >= 0 and no momentum where h < 1 mm (the net's momentum
// change is not reliable on films thinner than that: a small error there is a
// large velocity)
__device__ __forceinline__ Cell updated(Cell u, const float *d) {
    Cell r;
    r.h = u.h + d[0];
    if (r.h < 0.0f) r.h = 0.0f;
    if (r.h < FP_H_DRY_F) {
        r.hu = 0.0f;
        r.hv = 0.0f;
    } else {
        r.hu = u.hu + d[1];
        r.hv = u.hv + d[2];
    }
    return r;
}

struct WindowView {
    const float *h0, *hu0, *hv0;  // start state (padded planes)
    const float *dU;              // [count][kT][kT][3]
    const int *batch_of;
    int tiles_x;
};

__device__ __forceinline__ Cell start_cell(const FpSim &S, const WindowView &V, int i, int j) {
    const size_t o = fp_pidx(S, i, j);
    return Cell{V.h0[o], V.hu0[o], V.hv0[o]};
}

// end-of-window state of any cell: start state of dry tiles, updated otherwise
__device__ __forceinline__ Cell end_cell(const FpSim &S, const WindowView &V, int i, int j) {
    const Cell u = start_cell(S, V, i, j);
    const int tx = i / kT, ty = j / kT;
    const int b = V.batch_of[ty * V.tiles_x + tx];
    if (b < 0) return u;
    return updated(u, V.dU + (((size_t)b * kT + (j - ty * kT)) * kT + (i - tx * kT)) * 3);
}

__device__ __forceinline__ Side side_of(Cell c, float z) {
    Side s{c.h, 0.0f, 0.0f, z};
    if (c.h > FP_H_EPS_F) {
        s.u = c.hu / c.h;
        s.v = c.hv / c.h;
    }
    return s;
}

// HLL mass flux across a face after the hydrostatic reconstruction, from side
// L (west / south) to side R (east / north)
__device__ __forceinline__ float face_mass(float g, Side L, Side R, bool xface) {
    const float zf = fmaxf(L.z, R.z);
    const float hL = fmaxf(0.0f, (L.h + L.z) - zf), hR = fmaxf(0.0f, (R.h + R.z) - zf);
    float fm, fn, ft;
    const float hg = 0.5f * g;
    if (xface) hll(g, hL, L.u, L.v, press(hg, hL), hR, R.u, R.v, press(hg, hR), fm, fn, ft);
    else hll(g, hL, L.v, L.u, press(hg, hL), hR, R.v, R.u, press(hg, hR), fm, fn, ft);
    return fm;
}

// inflow (m^2/s summed over faces, positive into the tile) across one tile-edge
// face, in the start (end = false) or end state
__device__ float edge_inflow(const FpSim &S, const WindowView &V, int e, int k, int x0, int x1, int y0, int y1,
                             bool end, float h_in) {
    auto cell = [&](int i, int j) { return end ? end_cell(S, V, i, j) : start_cell(S, V, i, j); };
    const float g = S.g;
    if (e < 2) {  // west (e = 0) / east (e = 1) edge, row j
        const int j = y0 + k;
        const int xl = e == 0 ? x0 - 1 : x1 - 1, xr = xl + 1;
        Side L, R;
        if (xr < S.nx) R = side_of(cell(xr, j), S.z[fp_pidx(S, xr, j)]);
        if (xl >= 0) L = side_of(cell(xl, j), S.z[fp_pidx(S, xl, j)]);
        if (xl < 0) L = ghost(S.bc[2][j], R, true, h_in);
        if (xr == S.nx) R = ghost(S.bc[3][j], L, true, h_in);
        const float f = face_mass(g, L, R, true);
        return e == 0 ? f : -f;
    }
    const int i = x0 + k;  // south (e = 2) / north (e = 3) edge, column i
    const int jb = e == 2 ? y0 - 1 : y1 - 1, ja = jb + 1;
    Side B, A;
    if (ja < S.ny) A = side_of(cell(i, ja), S.z[fp_pidx(S, i, ja)]);
    if (jb >= 0) B = side_of(cell(i, jb), S.z[fp_pidx(S, i, jb)]);
    if (jb < 0) B = ghost(S.bc[0][i], A, false, h_in);
    if (ja == S.ny) A = ghost(S.bc[1][i], B, false, h_in);
    const float f = face_mass(g, B, A, false);
    return e == 2 ? f : -f;
}

// One CTA per net tile: write U' into the state planes of parity par, FP64 tile
// volumes before / after, the trapezoid inflow through the tile edges, and the
// guard decision; with fix_tol > 0 an accepted tile's U' is then scaled to
// close its mass balance.
__global__ void __launch_bounds__(256) apply_kernel(const __grid_constant__ FpSim S, int par, WindowView V,
                                                    const int *__restrict__ list, const FpClock *c0, float mass_tol,
                                                    float fix_tol, unsigned char *fail, float *resid, int *n_fail) {
    __shared__ float s_scale;
    __shared__ double red[4][8];
    __shared__ float reds[8];
    __shared__ int redb[8];
    const int b = blockIdx.x, tile = list[b];
    const int x0 = (tile % V.tiles_x) * kT, y0 = (tile / V.tiles_x) * kT;
    const int x1 = min(S.nx, x0 + kT), y1 = min(S.ny, y0 + kT);
    const int w = x1 - x0, n = w * (y1 - y0);
    const float *d = V.dU + (size_t)b * kT * kT * 3;
    double m0 = 0.0, m1 = 0.0, q0 = 0.0, q1 = 0.0;
    float smax = 0.0f;
    int bad = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int r = k / w, c = k % w;
        const size_t o = fp_pidx(S, x0 + c, y0 + r);
        const Cell u = Cell{V.h0[o], V.hu0[o], V.hv0[o]};
        const Cell v = updated(u, d + ((size_t)r * kT + c) * 3);
        S.h[par][o] = v.h;
        S.hu[par][o] = v.hu;
        S.hv[par][o] = v.hv;
        m0 += (double)u.h;
        m1 += (double)v.h;
        if (!(v.h == v.h) || !(v.hu == v.hu) || !(v.hv == v.hv) || isinf(v.h) || isinf(v.hu) || isinf(v.hv))
            bad = 1;
        else if (v.h > FP_H_EPS_F)
            smax = fmaxf(smax, fp_wave_speed(S.g, v.h, v.hu, v.hv));
    }
    const long long t0 = c0->t, t1 = t0 + (long long)kWin * S.dt_fixed;
    const float hin0 = (float)fp_hydro_depth(S, t0), hin1 = (float)fp_hydro_depth(S, t1);
    for (int e = 0; e < 4; ++e) {
        const int len = e < 2 ? y1 - y0 : x1 - x0;
        for (int k = threadIdx.x; k < len; k += blockDim.x) {
            q0 += (double)edge_inflow(S, V, e, k, x0, x1, y0, y1, false, hin0);
            q1 += (double)edge_inflow(S, V, e, k, x0, x1, y0, y1, true, hin1);
        }
    }
    double acc[4] = {m0, m1, q0, q1};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
        smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        for (int a = 0; a < 4; ++a) red[a][wid] = acc[a];
        reds[wid] = smax;
        redb[wid] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        float sm = 0.0f;
        int bd = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            for (int a = 0; a < 4; ++a) s[a] += red[a][k];
            sm = fmaxf(sm, reds[k]);
            bd |= redb[k];
        }
        const double dx = (double)S.dx, dts = (double)S.dt_fixed / 1048576.0;
        const double dM = (s[1] - s[0]) * dx * dx;
        const double F = (double)kWin * dts * dx * 0.5 * (s[2] + s[3]);
        const double denom = fmax(s[0] * dx * dx, (double)n * dx * dx * 0.01);
        const double rs = fabs(dM - F) / denom;
        const bool cfl_bad = (double)sm * dts > (double)S.cfl * dx;
        bool mass_bad = !(rs <= (double)(fix_tol > 0.0f ? fix_tol : mass_tol));
        // mass fix: one factor on the tile's h, hu, hv brings its volume to
        // the start volume plus the inflow estimate
        double scale = 1.0;
        if (fix_tol > 0.0f && !(bd || cfl_bad || mass_bad)) {
            const double v1 = s[1] * dx * dx, target = s[0] * dx * dx + F;
            if (v1 > 0.0) scale = target / v1;
            else if (target != 0.0) mass_bad = true;
            if (!(scale >= 0.0)) mass_bad = true;
        }
        const bool f = bd || cfl_bad || mass_bad;
        s_scale = f ? 1.0f : (float)scale;
        fail[b] = (unsigned char)((bd ? 4 : 0) | (cfl_bad ? 2 : 0) | (mass_bad ? 1 : 0));
        resid[b] = bd ? __int_as_float(0x7f800000) : (float)rs;
        if (f) atomicAdd(n_fail, 1);
    }
    __syncthreads();
    const float scale = s_scale;
    if (scale != 1.0f) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const size_t o = fp_pidx(S, x0 + k % w, y0 + k / w);
            S.h[par][o] *= scale;
            S.hu[par][o] *= scale;
            S.hv[par][o] *= scale;
        }
    }
}

// evacuees per cell of the current records (B), for the plain fallback
__global__ void occupancy_kernel(const __grid_constant__ FpSim S, unsigned short *occ) {
    const int nB = S.cnt->nB;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nB; i += gridDim.x * blockDim.x) {
        const uint4 pa = S.pedB[2 * i], pb = S.pedB[2 * i + 1];
        const unsigned meta = pb.y;
        if (FP_META_EXITED(meta) || FP_META_ROLE(meta) != 0) continue;
        const int ci = fp_cell_of(__uint_as_float(pa.x), S.dx), cj = fp_cell_of(__uint_as_float(pa.y), S.dx);
        if (ci < 0 || cj < 0 || ci >= S.nx || cj >= S.ny) continue;
        const size_t o = fp_pidx(S, ci, cj);
        const unsigned shift = (unsigned)(o & 1) * 16u;
        atomicAdd(reinterpret_cast<unsigned *>(occ + (o & ~(size_t)1)), 1u << shift);
    }
}

// largest |a - b| over the cells of the tiles with keep[tile] != 0 (float bits;
// NaN counts as infinity)
__global__ void diff_kernel(const __grid_constant__ FpSim S, const float *__restrict__ a, const float *__restrict__ b,
                            const unsigned char *__restrict__ keep, int tiles_x, unsigned *max_bits) {
    float m = 0.0f;
    const long long n = (long long)S.nx * S.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % S.nx), j = (int)(c / S.nx);
        if (!keep[(j / kT) * tiles_x + i / kT]) continue;
        const size_t o = fp_pidx(S, i, j);
        const float d = fabsf(a[o] - b[o]);
        m = fmaxf(m, d == d ? d : __int_as_float(0x7f800000));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(max_bits, __float_as_uint(m));
}

// recomputed tiles (flags[tile] != 0) -> state planes of parity par
__global__ void merge_kernel(const __grid_constant__ FpSim S, int par, const float *__restrict__ h,
                             const float *__restrict__ hu, const float *__restrict__ hv,
                             const unsigned char *__restrict__ flags, int tiles_x) {
    const int tile = blockIdx.x;
    if (!flags[tile]) return;
    const int x0 = (tile % tiles_x) * kT, y0 = (tile / tiles_x) * kT;
    const int x1 = min(S.nx, x0 + kT), y1 = min(S.ny, y0 + kT);
    const int w = x1 - x0, n = w * (y1 - y0);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const size_t o = fp_pidx(S, x0 + k % w, y0 + k / w);
        S.h[par][o] = h[o];
        S.hu[par][o] = hu[o];
        S.hv[par][o] = hv[o];
    }
}

}  // namespace

void fp_launch_clock_advance(const FpSim &S, int slot, cudaStream_t st) {
    clock_advance_kernel<<<1, 1, 0, st>>>(S, slot);
}

void fp_launch_sur_classify(const FpSim &S, int par, const FpClock *c0, int tiles_x, int tiles_y, unsigned char *wet,
                            cudaStream_t st) {
    classify_kernel<<<tiles_x * tiles_y, 256, 0, st>>>(S, par, c0, tiles_x, wet);
}

void fp_launch_sur_compact(const unsigned char *flags, int n, int *list, int *batch_of, int *count, cudaStream_t st) {
    compact_kernel<<<1, 1024, 0, st>>>(flags, n, list, batch_of, count);
}

void fp_launch_sur_input(const FpSim &S, const float *h, const float *hu, const float *hv, const int *list, int count,
                         int tiles_x, void *x16, cudaStream_t st) {
    const long long total = (long long)count * kIn * kIn;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 148LL * 16);
    if (blocks > 0)
        input_kernel<<<blocks, 256, 0, st>>>(S, h, hu, hv, list, count, tiles_x, static_cast<__nv_bfloat16 *>(x16));
}

void fp_launch_sur_apply(const FpSim &S, int par, const float *h0, const float *hu0, const float *hv0,
                         const float *dU, const int *list, const int *batch_of, int count, int tiles_x,
                         const FpClock *c0, float mass_tol, float fix_tol, unsigned char *fail, float *resid,
                         int *n_fail, cudaStream_t st) {
    if (count <= 0) return;
    WindowView V{h0, hu0, hv0, dU, batch_of, tiles_x};
    apply_kernel<<<count, 256, 0, st>>>(S, par, V, list, c0, mass_tol, fix_tol, fail, resid, n_fail);
}

void fp_launch_sur_occupancy(const FpSim &S, unsigned short *occ, cudaStream_t st) {
    occupancy_kernel<<<148 * 4, 256, 0, st>>>(S, occ);
}

void fp_launch_sur_diff(const FpSim &S, const float *a, const float *b, const unsigned char *keep, int tiles_x,
                        unsigned *max_bits, cudaStream_t st) {
    diff_kernel<<<148 * 8, 256, 0, st>>>(S, a, b, keep, tiles_x, max_bits);
}

void fp_launch_sur_merge(const FpSim &S, int par, const float *h, const float *hu, const float *hv,
                         const unsigned char *flags, int tiles_x, int tiles_y, cudaStream_t st) {
    merge_kernel<<<tiles_x * tiles_y, 256, 0, st>>>(S, par, h, hu, hv, flags, tiles_x);
}
