// flood_dev.cuh -- device code of the hydrodynamic cell update (Section 2.2),
// shared by the per-step flood kernel and the persistent coupled-step kernel.
//
// flood_tiles<TY>: 64 x TY tiles of cells by 32 x TY threads, a CTA taking a
// strided list of tiles.
//   0. tile modes from 64 x 8-cell water flags: tiles that stayed dry are not
//      loaded (their update would write zeros);
//   1. one thread issues six 2D TMA loads (cp.async.bulk.tensor) of a tile
//      plus a one-cell halo (a 72-float-wide box starting 16-byte aligned) of
//      h, hu, hv, z, and of the tile's n0 and evacuee counts, into one of two
//      stage buffers, completing on that buffer's mbarrier; the next tile's
//      loads are issued before the current tile is processed;
//   2. velocities u = hu/h, v = hv/h per staged cell;
//   3. every x and y face of the tile once: non-negative hydrostatic
//      reconstruction h* = max(0, eta - max(z_L, z_R)) and the HLL flux;
//      each side keeps the flux minus the pressure 1/2 g h*^2 of its own
//      reconstructed depth (this carries the bed-slope source of Eq. 1);
//      domain-edge faces use ghost states from the boundary codes;
//   4. Eq. (2) per cell, point-implicit Manning friction with
//      n = n0 + N_p n0 (N_p <= 20), writes U^{n+1} (warp r: row r, lane l:
//      cells l and l + 32, so every shared-memory access is lane-contiguous);
//      the CFL wave-speed max of U^{n+1} and the wet flag are reduced per CTA
//      (warp shuffles) and folded into the next step's clock slot with one
//      atomic each; edge tiles add their boundary mass fluxes in FP64.
// Built with -fmad=false: every fused multiply-add is written out, and each one
// is sign-symmetric, so the update is exactly mirror-symmetric and gives the
// same bits in every kernel it is inlined into.
#pragma once
#include "fp_common.cuh"

namespace fpdev {


constexpr int ROWW = FP_TX + 8;  // staged row width: 4 guard floats each side

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float sqrt_fast(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// h^(-4/3) = 2^(-4/3 log2 h) for h > 0 (two special-function instructions)
__device__ __forceinline__ float pow_m43(float h) {
    float l, r;
    asm("lg2.approx.f32 %0, %1;" : "=f"(l) : "f"(h));
    const float e = -1.33333333f * l;
    asm("ex2.approx.f32 %0, %1;" : "=f"(r) : "f"(e));
    return r;
}

// face pressure 1/2 g h^2 from hg = 1/2 g (the same products in the same order)
__device__ __forceinline__ float press(float hg, float h) { return hg * h * h; }

// HLL flux across a face; un normal and ut tangential velocity, pL/pR the face
// pressures 1/2 g h^2 of the two sides.  out = (mass, normal momentum incl.
// pressure, tangential momentum).  Identical states give the physical flux
// exactly (lake at rest stays exactly at rest).  Faces with both sides dry
// leave at once; otherwise every case is computed and the one that applies is
// selected, in this order of precedence: both dry (no flux), identical states
// or sL >= 0 (left flux), sR <= 0 (right flux), the HLL average.
__device__ __forceinline__ void hll(float g, float hL, float unL, float utL, float pL, float hR, float unR,
                                    float utR, float pR, float &fm, float &fn, float &ft) {
    const bool dL = hL <= FP_H_EPS_F, dR = hR <= FP_H_EPS_F;
    if (dL && dR) {
        fm = 0.0f; fn = 0.0f; ft = 0.0f;
        return;
    }
    const float qL = hL * unL, qR = hR * unR;
    const float FL0 = qL, FL1 = __fmaf_rn(qL, unL, pL), FL2 = qL * utL;
    const float FR0 = qR, FR1 = __fmaf_rn(qR, unR, pR), FR2 = qR * utR;
    // wave speeds: Einfeldt-type bounds, or the dry-bed ones when a side is dry
    // (the left side's test first)
    const float cL = sqrt_fast(g * hL), cR = sqrt_fast(g * hR);
    const float us = __fmaf_rn(0.5f, unL + unR, cL - cR);
    const float cs = __fmaf_rn(0.25f, unL - unR, 0.5f * (cL + cR));
    const float a = unL - cL, b = us - cs;
    float sL = a < b ? a : b;
    const float c = unR + cR, d = us + cs;
    float sR = c > d ? c : d;
    if (dR) { sL = unL - cL; sR = __fmaf_rn(2.0f, cL, unL); }
    if (dL) { sL = __fmaf_rn(-2.0f, cR, unR); sR = unR + cR; }
    // Differences of two products are rounded explicitly (no contraction), so the
    // flux of a mirrored face is exactly the mirrored flux (its sR - sL is the
    // same number, so any reciprocal keeps that).
    const float inv = rcp_fast(sR - sL);
    const float sLR = __fmul_rn(sL, sR);
    fm = __fadd_rn(__fsub_rn(__fmul_rn(sR, FL0), __fmul_rn(sL, FR0)), __fmul_rn(sLR, hR - hL)) * inv;
    fn = __fadd_rn(__fsub_rn(__fmul_rn(sR, FL1), __fmul_rn(sL, FR1)), __fmul_rn(sLR, qR - qL)) * inv;
    ft = __fadd_rn(__fsub_rn(__fmul_rn(sR, FL2), __fmul_rn(sL, FR2)),
                   __fmul_rn(sLR, __fsub_rn(__fmul_rn(hR, utR), __fmul_rn(hL, utL)))) * inv;
    if (sR <= 0.0f) { fm = FR0; fn = FR1; ft = FR2; }
    if (sL >= 0.0f || (hL == hR && unL == unR && utL == utR)) { fm = FL0; fn = FL1; ft = FL2; }
}

struct Side {
    float h, u, v, z;
};

// Ghost state outside a boundary cell: a wall (code 0) and a discharge breach
// (code 3, whose inflow is added to the face flux) reflect the normal velocity,
// a transmissive edge (1) copies the cell, a depth inflow (2) is water at rest
// at the hydrograph depth.
__device__ __forceinline__ Side ghost(unsigned char code, Side in, bool normal_x, float h_in) {
    Side g = in;
    if (code == 0 || code == 3) {
        if (normal_x) g.u = -in.u; else g.v = -in.v;
    } else if (code == 2) {
        g.h = h_in; g.u = 0.0f; g.v = 0.0f;
    }
    return g;
}

// staged plane stride, padded to 32 floats so every TMA destination is 128-byte aligned
template <int TY>
__host__ __device__ constexpr int plane_stride() {
    return (((TY + 2) * ROWW + 31) / 32) * 32;
}

// Shared memory of the flood tiles, in bytes: two stage buffers, each holding
// the staged h, hu, hv, z (tile + one-cell halo, ROWW x (TY + 2) floats each),
// n0 (ROWW x TY floats) and evacuee counts (ROWW x TY uint16, box starting at
// the tile's first cell - 4 so that its x coordinate is 16-byte aligned); then
// the south-face fluxes [TY+1][64] and the east tile-edge fluxes [TY].
template <int TY>
struct FloodSmem {
    static constexpr int PLANE = plane_stride<TY>();  // floats
    static constexpr int N0 = 4 * PLANE * 4;            // byte offsets within a buffer
    static constexpr int OCC = N0 + TY * ROWW * 4;
    static constexpr int BUF = OCC + TY * ROWW * 2;
    static constexpr int TX_BYTES = 4 * (TY + 2) * ROWW * 4 + TY * ROWW * 4 + TY * ROWW * 2;
    static constexpr int YF = 2 * BUF;
    static constexpr int XE = YF + (TY + 1) * FP_TX * 16;
    static constexpr int BYTES = XE + TY * 16;
    static_assert(N0 % 128 == 0 && OCC % 128 == 0 && BUF % 128 == 0, "TMA destinations 128-byte aligned");
};

template <int TY>
__host__ __device__ constexpr int smem_bytes() {
    return FloodSmem<TY>::BYTES;
}

// a staged cell as a face side: depth, velocities (0 at h <= h_eps), bed
__device__ __forceinline__ Side staged_side(const float *s_h, const float *s_hu, const float *s_hv, const float *s_z,
                                            int o) {
    Side c{s_h[o], 0.0f, 0.0f, s_z[o]};
    if (c.h > FP_H_EPS_F) {
        c.u = __fdividef(s_hu[o], c.h);
        c.v = __fdividef(s_hv[o], c.h);
    }
    return c;
}

__device__ __forceinline__ Side shfl_side(Side c, int src) {
    return Side{__shfl_sync(0xffffffffu, c.h, src), __shfl_sync(0xffffffffu, c.u, src),
                __shfl_sync(0xffffffffu, c.v, src), __shfl_sync(0xffffffffu, c.z, src)};
}

__device__ __forceinline__ Side shfl_up_side(Side c) {
    return Side{__shfl_up_sync(0xffffffffu, c.h, 1), __shfl_up_sync(0xffffffffu, c.u, 1),
                __shfl_up_sync(0xffffffffu, c.v, 1), __shfl_up_sync(0xffffffffu, c.z, 1)};
}

__device__ __forceinline__ float4 shfl_f4(float4 f, int src) {
    return make_float4(__shfl_sync(0xffffffffu, f.x, src), __shfl_sync(0xffffffffu, f.y, src),
                       __shfl_sync(0xffffffffu, f.z, src), __shfl_sync(0xffffffffu, f.w, src));
}

__device__ __forceinline__ float4 shfl_down_f4(float4 f) {
    return make_float4(__shfl_down_sync(0xffffffffu, f.x, 1), __shfl_down_sync(0xffffffffu, f.y, 1),
                       __shfl_down_sync(0xffffffffu, f.z, 1), __shfl_down_sync(0xffffffffu, f.w, 1));
}

// Inflow of a discharge breach over one step: qd.x = mean unit discharge q
// (m^2/s) entering through each breach face, qd.y = the momentum it carries,
// q u_in with u_in = q / h_qin.  Added to the wall flux of a breach face, in
// the direction into the domain.
__device__ __forceinline__ void add_discharge(float dir, float2 qd, float &fm, float &fn) {
    fm = __fadd_rn(fm, dir * qd.x);
    fn = __fadd_rn(fn, qd.y);
}

// x face between cells i-1 (L) and i (R) of row j: (mass, normal momentum minus
// the L pressure, minus the R pressure, tangential momentum); ghosts on the
// domain's west / east edges; zero past the east edge.  edge (the same for the
// whole tile) is false when the tile touches no domain edge: no checks then.
__device__ __forceinline__ float4 x_face(const FpSim &S, float g, float hg, float h_in, float2 qd, Side L, Side R,
                                         int i, int j, bool edge) {
    float dir = 0.0f;  // +1 / -1: a discharge breach face on the west / east edge
    if (edge) {
        if (i > S.nx) return make_float4(0.f, 0.f, 0.f, 0.f);
        if (i == 0) {
            const unsigned char c = S.bc[2][j];
            L = ghost(c, R, true, h_in);
            if (c == 3) dir = 1.0f;
        }
        if (i == S.nx) {
            const unsigned char c = S.bc[3][j];
            R = ghost(c, L, true, h_in);
            if (c == 3) dir = -1.0f;
        }
    }
    const float zf = fmaxf(L.z, R.z);
    const float hLs = fmaxf(0.0f, (L.h + L.z) - zf);
    const float hRs = fmaxf(0.0f, (R.h + R.z) - zf);
    const float pL = press(hg, hLs), pR = press(hg, hRs);
    float fm, fn, ft;
    hll(g, hLs, L.u, L.v, pL, hRs, R.u, R.v, pR, fm, fn, ft);
    if (dir != 0.0f) add_discharge(dir, qd, fm, fn);
    return make_float4(fm, fn - pL, fn - pR, ft);
}

// y face between rows j-1 (B) and j (A) of column i: (mass, tangential momentum,
// normal momentum minus the B pressure, minus the A pressure); ghosts on the
// domain's south / north edges; zero past the east edge.
__device__ __forceinline__ float4 y_face(const FpSim &S, float g, float hg, float h_in, float2 qd, Side B, Side A,
                                         int i, int j, bool edge) {
    float dir = 0.0f;  // +1 / -1: a discharge breach face on the south / north edge
    if (edge) {
        if (i >= S.nx) return make_float4(0.f, 0.f, 0.f, 0.f);
        if (j == 0) {
            const unsigned char c = S.bc[0][i];
            B = ghost(c, A, false, h_in);
            if (c == 3) dir = 1.0f;
        }
        if (j == S.ny) {
            const unsigned char c = S.bc[1][i];
            A = ghost(c, B, false, h_in);
            if (c == 3) dir = -1.0f;
        }
    }
    const float zf = fmaxf(B.z, A.z);
    const float hBs = fmaxf(0.0f, (B.h + B.z) - zf);
    const float hAs = fmaxf(0.0f, (A.h + A.z) - zf);
    const float pB = press(hg, hBs), pA = press(hg, hAs);
    float fm, fn, ft;
    hll(g, hBs, B.v, B.u, pB, hAs, A.v, A.u, pA, fm, fn, ft);
    if (dir != 0.0f) add_discharge(dir, qd, fm, fn);
    return make_float4(fm, ft, fn - pB, fn - pA);
}

// Work of a tile in one step, decided before its loads are issued.
enum : unsigned char { kTileNone = 0, kTileDry = 1, kTileLoad = 2 };
constexpr int kModeChunk = 64;  // tile modes decided together by one CTA

// tid 0: the TMA loads of tile (x0, y0) into one stage buffer, completing on mbar
template <int TY>
__device__ __forceinline__ void stage_tile(const FpTmaSet &tm, unsigned char *buf, unsigned long long *mbar, int x0,
                                           int y0) {
    using L = FloodSmem<TY>;
    const unsigned bar = smem_u32(mbar);
    // the buffer was last read by generic loads of this CTA; the global data by
    // generic stores of earlier phases
    asm volatile("fence.proxy.async;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(L::TX_BYTES) : "memory");
    const CUtensorMap *maps[6] = {&tm.h, &tm.hu, &tm.hv, &tm.z, &tm.n0, &tm.occ};
    const int offs[6] = {0, L::PLANE * 4, 2 * L::PLANE * 4, 3 * L::PLANE * 4, L::N0, L::OCC};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        // planes with the halo row above the tile; n0 and counts from the tile's first row
        const int y = k < 4 ? y0 : y0 + 1;
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(smem_u32(buf + offs[k])),
            "l"(reinterpret_cast<unsigned long long>(maps[k])), "r"(x0), "r"(y), "r"(bar)
            : "memory");
    }
}

// bounded wait for phase `parity` of an mbarrier (false: it did not complete)
__device__ __forceinline__ bool mbar_wait_phase(unsigned long long *mbar, unsigned parity) {
    const unsigned bar = smem_u32(mbar);
    unsigned ok = 0;
    for (int it = 0; it < (1 << 22) && !ok; ++it) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
    }
    return ok != 0;
}

// Modes of the CTA's tiles first + k * stride, k in [k0, k0 + kModeChunk), into
// s_mode[k - k0]; warp w takes k0 + w, k0 + w + TY, ...; each lane loads one
// water flag of the tile's dependence region.  A tile is
//   kTileNone when the tile mask excludes it;
//   kTileDry  when no block of it or of its one-cell halo held water after the
//             last step (flags of the input plane), its own blocks of the output
//             plane already hold the zero state (flags from two steps back), no
//             inflow ghost is active on its edges and it is not tile 0 (which
//             advances the clock): every flux is zero and the update would
//             write zeros, so nothing is loaded and only the evacuee counts are
//             cleared;
//   kTileLoad otherwise.
template <int TY>
__device__ __forceinline__ void decide_modes(const FpSim &S, int par, int first, int stride, int ntiles, int k0,
                                             bool inflow_on, unsigned char *s_mode) {
    constexpr int R = kModeChunk / TY;
    static_assert((TY / FP_BLK_ROWS + 2) * 3 + TY / FP_BLK_ROWS <= 32, "one flag per lane");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nx = S.nx, ny = S.ny, bw = (nx + FP_TX - 1) / FP_TX;
    const bool flags = S.blk_wet[0] != nullptr;
    int f[R];
    unsigned char m[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = first + (k0 + w + r * TY) * stride;
        f[r] = 0;
        m[r] = 1;
        if (t < ntiles) {
            const int bx = t % bw, y0 = (t / bw) * TY;
            if (flags) {
                const int r0 = max(0, y0 - 1) / FP_BLK_ROWS, r1 = min(ny - 1, y0 + TY) / FP_BLK_ROWS;
                const int c0 = max(0, bx - 1), c1 = min(bw - 1, bx + 1);
                const int nc = c1 - c0 + 1, nin = (r1 - r0 + 1) * nc;
                const int q0 = y0 / FP_BLK_ROWS, nout = min(ny - 1, y0 + TY - 1) / FP_BLK_ROWS - q0 + 1;
                if (lane < nin) f[r] = S.blk_wet[par][(r0 + lane / nc) * bw + c0 + lane % nc];
                else if (lane < nin + nout) f[r] = S.blk_wet[par ^ 1][(q0 + lane - nin) * bw + bx];
            }
            if (lane == 0 && S.tile_mask != nullptr) m[r] = S.tile_mask[t];
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int k = k0 + w + r * TY, t = first + k * stride;
        const bool any = __any_sync(0xffffffffu, f[r] != 0);
        if (lane == 0 && t < ntiles) {
            const int x0 = (t % bw) * FP_TX, y0 = (t / bw) * TY;
            const bool edge = x0 == 0 || x0 + FP_TX >= nx || y0 == 0 || y0 + TY >= ny;
            unsigned char mode = kTileLoad;
            if (m[r] == 0) mode = kTileNone;
            else if (flags && !any && t != 0 && !(inflow_on && edge)) mode = kTileDry;
            s_mode[k - k0] = mode;
        }
    }
}

// The CTA's tiles first, first + stride, ... (< ntiles) of the 64 x TY tiling
// (tile t at column t % tiles_x, row t / tiles_x), by the 32 * TY threads of the
// CTA: warp r owns row r of a tile, lane l its cells l and l + 32.  Loads are
// double-buffered: the next tile's TMA copies are issued before the current
// tile waits for its own.  mbar[2] (initialised, count 1) and their phase bits
// (bit b: buffer b) belong to the caller (only the control thread's copy is
// used); no thread may still read the stage buffers of an earlier call.  Returns false if a TMA
// transfer did not complete (error flag set).  speculative: issue the first
// tile's loads before its mode is decided (lower latency; a skipped first tile
// is loaded all the same).
template <int TY>
__device__ bool flood_tiles(const FpTmaSet &tm, const FpSim &S, int par, int slot, int first, int stride,
                            int ntiles, unsigned char *smem_raw, unsigned long long *mbar, unsigned &phase,
                            bool speculative) {
    using L = FloodSmem<TY>;
    constexpr int NT = 32 * TY;
    static_assert(TY % FP_BLK_ROWS == 0 && TY >= 8, "whole water-flag blocks; edge-face, flux and control warps apart");
    __shared__ unsigned char s_mode[kModeChunk];
    __shared__ long long s_dt, s_t, s_step;
    __shared__ float s_hin, s_dtf, s_lx, s_accm;
    __shared__ float2 s_qd;
    __shared__ unsigned s_smax0;
    __shared__ int s_ok[2], s_accf, s_accn;
    __shared__ int2 s_xy[2];
    __shared__ int s_blk[TY / FP_BLK_ROWS];
    __shared__ float s_red[NT / 32];
    __shared__ int s_redi[NT / 32];
    __shared__ float s_bx[2][TY];      // mass flux through the west / east domain edge faces
    __shared__ float s_by[2][FP_TX];   // ... through the south / north domain edge faces
    float4 *s_yf = reinterpret_cast<float4 *>(smem_raw + L::YF);  // [TY+1][64] south faces; row TY: the tile's north edge
    float4 *s_xe = reinterpret_cast<float4 *>(smem_raw + L::XE);  // [TY] the tile's east-edge face of each row

    if (first >= ntiles) return true;
    const int tid = threadIdx.x, lane = tid & 31, row = tid >> 5;
    // the control thread (lane 0 of the last warp, which computes no edge
    // faces): waits for and issues the TMA loads, folds the reductions
    constexpr int CTL = NT - 32;
    const int nx = S.nx, ny = S.ny, tiles_x = (nx + FP_TX - 1) / FP_TX;

    // the step's clock, the same for every tile; an inflow is active while the
    // depth hydrograph is above h_eps or the discharge hydrograph has not ended
    const bool inflow_on = (S.has_inflow && S.clock[slot].h_in > FP_H_EPS_F) ||
                           (S.has_discharge && S.clock[slot].t < S.q_end_ticks);
    if (tid == 0) {
        const FpClock c = S.clock[slot];
        const long long dt = fp_dt_ticks(S, c, c.h_in);
        const float dtf = (float)dt * (1.0f / FP_TICKS_F);
        // the discharge breach: mean unit discharge over [t, t + dt] from the
        // exact volume of the hydrograph, and the momentum it carries
        float2 qd = make_float2(0.0f, 0.0f);
        if (S.has_discharge && dt > 0) {
            const double t0 = __ddiv_rn((double)c.t, 1048576.0), t1 = __ddiv_rn((double)(c.t + dt), 1048576.0);
            const double dV = __dsub_rn(fp_discharge_volume(S, t1), fp_discharge_volume(S, t0));
            const double q = __ddiv_rn(dV, __dmul_rn(__ddiv_rn((double)dt, 1048576.0), S.q_width));
            qd = make_float2((float)q, (float)__dmul_rn(q, __ddiv_rn(q, S.h_qin)));
        }
        s_qd = qd;
        s_hin = c.h_in;
        s_dt = dt;
        s_dtf = dtf;
        s_lx = __fdiv_rn(dtf, S.dx);
        s_t = c.t;
        s_step = c.step;
        s_smax0 = c.smax_bits;
        s_accm = 0.0f;
        s_accf = 0;
        s_accn = 0;
    }
    auto stage = [&](int t, int b) {
        stage_tile<TY>(tm, smem_raw + b * L::BUF, &mbar[b], (t % tiles_x) * FP_TX, (t / tiles_x) * TY);
    };
    // speculative: the first tile's loads go out before its mode is known
    // (they overlap the flag loads) and are waited for whatever the mode;
    // otherwise the mode is decided first, so that a skipped tile loads nothing
    if (tid == CTL && speculative) stage(first, 0);
    decide_modes<TY>(S, par, first, stride, ntiles, 0, inflow_on, s_mode);
    __syncthreads();
    if (tid == CTL && !speculative && s_mode[0] == kTileLoad) stage(first, 0);

    // Per tile k (buffer b = k & 1): the control thread waits for the tile's
    // loads; one barrier; it issues the next tile's loads into the other buffer
    // (every thread is past the previous tile, its last reader); the tile is
    // processed.  Values it publishes per tile are double-buffered too, so a
    // tile needs no closing barrier.
    int b = 0;
    for (int k = 0; first + k * stride < ntiles; ++k, b ^= 1) {
        const int t = first + k * stride, tn = t + stride;
        const int mode = s_mode[k % kModeChunk];
        if (tn < ntiles && (k + 1) % kModeChunk == 0) {
            __syncthreads();  // every thread has read this tile's mode
            decide_modes<TY>(S, par, first, stride, ntiles, k + 1, inflow_on, s_mode);
        }
        if (tid == CTL) {
            int ok = 1;
            if (mode == kTileLoad || (k == 0 && speculative)) {
                ok = mbar_wait_phase(&mbar[b], (phase >> b) & 1u);
                phase ^= 1u << b;
                if (!ok) fp_set_err(S, FP_ERR_TIMEOUT);
            }
            s_ok[b] = ok;
            s_xy[b] = make_int2((t % tiles_x) * FP_TX, (t / tiles_x) * TY);
        }
        __syncthreads();
        if (!s_ok[b]) return false;
        if (tid == CTL && tn < ntiles && s_mode[(k + 1) % kModeChunk] == kTileLoad) stage(tn, b ^ 1);
        const int x0 = s_xy[b].x, y0 = s_xy[b].y, bx = x0 / FP_TX;
        const int cj = y0 + row;
        // the tile or its halo touches a domain edge (then the faces check for
        // ghosts and for cells past the edge)
        const bool edge = x0 == 0 || y0 == 0 || x0 + FP_TX >= nx || y0 + TY >= ny;
        const bool okA = cj < ny && x0 + lane < nx, okB = cj < ny && x0 + lane + 32 < nx;
        const size_t gA = okA ? fp_pidx(S, x0 + lane, cj) : 0;
        if (mode != kTileLoad) {
            if (mode == kTileDry) {  // the evacuee counts this step read are cleared all the same
                if (okA) S.occ[par][gA] = 0;
                if (okB) S.occ[par][gA + 32] = 0;
            }
            continue;
        }
        unsigned char *buf = smem_raw + b * L::BUF;
        float *s_h = reinterpret_cast<float *>(buf);
        float *s_hu = s_h + L::PLANE;
        float *s_hv = s_hu + L::PLANE;
        float *s_z = s_hv + L::PLANE;
        const float *s_n0 = reinterpret_cast<const float *>(buf + L::N0);
        const unsigned short *s_occ = reinterpret_cast<const unsigned short *>(buf + L::OCC);
        if (tid < TY / FP_BLK_ROWS) s_blk[tid] = 0;
        if (tid == CTL && S.blk_runs != nullptr)  // profiling: the blocks this update computes
            for (int r = y0 / FP_BLK_ROWS; r <= (min(ny, y0 + TY) - 1) / FP_BLK_ROWS; ++r)
                S.blk_runs[r * tiles_x + bx] += 1u;
        // this thread's two cells' n0 and evacuee counts (staged from the tile's
        // first cell - 4)
        const float n0A = s_n0[row * ROWW + lane + 4], n0B = s_n0[row * ROWW + lane + 36];
        const unsigned short occA = s_occ[row * ROWW + lane + 4], occB = s_occ[row * ROWW + lane + 36];

        const float g = S.g, hg = 0.5f * g;
        const float h_in = s_hin;
        const float2 qd = s_qd;

        const int oA = (row + 1) * ROWW + lane + 4, oB = oA + 32;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

        // 2. faces from registers: this thread's cells A (column lane) and B (lane +
        // 32) of row `row`; each computes its west and south face.  West
        // neighbours arrive by shuffle (lane 0: the halo cell, and cell 31 for B).
        const int iA = x0 + lane, iB = iA + 32;
        float4 fwA = zero4, fwB = zero4;
        {
            const Side cA = staged_side(s_h, s_hu, s_hv, s_z, oA);
            const Side cB = staged_side(s_h, s_hu, s_hv, s_z, oB);
            Side wA = shfl_up_side(cA), wB = shfl_up_side(cB);
            const Side c31 = shfl_side(cA, 31);
            if (lane == 0) {
                wA = staged_side(s_h, s_hu, s_hv, s_z, oA - 1);
                wB = c31;
            }
            if (cj < ny) {
                fwA = x_face(S, g, hg, h_in, qd, wA, cA, iA, cj, edge);
                fwB = x_face(S, g, hg, h_in, qd, wB, cB, iB, cj, edge);
                if (iA == 0) s_bx[0][row] = fwA.x;
                if (iA == nx) s_bx[1][row] = fwA.x;
                if (iB == nx) s_bx[1][row] = fwB.x;
            }
            if (cj <= ny) {
                const Side bA = staged_side(s_h, s_hu, s_hv, s_z, oA - ROWW);
                const Side bB = staged_side(s_h, s_hu, s_hv, s_z, oB - ROWW);
                const float4 gA = y_face(S, g, hg, h_in, qd, bA, cA, iA, cj, edge);
                const float4 gB = y_face(S, g, hg, h_in, qd, bB, cB, iB, cj, edge);
                s_yf[row * FP_TX + lane] = gA;
                s_yf[row * FP_TX + lane + 32] = gB;
                if (cj == 0) { s_by[0][lane] = gA.x; s_by[0][lane + 32] = gB.x; }
                if (cj == ny) { s_by[1][lane] = gA.x; s_by[1][lane + 32] = gB.x; }
            }
        }
        // 3. the tile's edge faces: north (row y0 + TY) of each column by warps 0
        // and 1, east (column x0 + 64) of each row by warp 2 (the control warp,
        // the last, has none)
        if (tid < FP_TX + TY) {
            if (tid >= FP_TX) {
                const int r = tid - FP_TX, j = y0 + r, i = x0 + FP_TX;
                float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < ny && i <= nx) {
                    const int o = (r + 1) * ROWW + FP_TX + 4;
                    f = x_face(S, g, hg, h_in, qd, staged_side(s_h, s_hu, s_hv, s_z, o - 1),
                               staged_side(s_h, s_hu, s_hv, s_z, o), i, j, edge);
                    if (i == nx) s_bx[1][r] = f.x;
                }
                s_xe[r] = f;
            } else {
                const int c = tid, i = x0 + c, j = y0 + TY;
                float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j <= ny) {
                    const int o = (TY + 1) * ROWW + c + 4;
                    f = y_face(S, g, hg, h_in, qd, staged_side(s_h, s_hu, s_hv, s_z, o - ROWW),
                               staged_side(s_h, s_hu, s_hv, s_z, o), i, j, edge);
                    if (j == ny && i < nx) s_by[1][c] = f.x;
                }
                s_yf[TY * FP_TX + c] = f;
            }
        }
        __syncthreads();

        // 4. Eq. (2) + friction for this thread's two cells; east fluxes by shuffle
        // (lane 31: cell 32's west face, and the tile's east edge for B)
        float sk_[2] = {-1.0f, -1.0f}, hk_[2] = {0.f, 0.f}, huk_[2] = {0.f, 0.f}, hvk_[2] = {0.f, 0.f};
        int wet = 0, neg = 0, bad = 0, nz = 0;
        const float dt = s_dtf, lx = s_lx, ly = s_lx;
        const int p2 = par ^ 1;
        float4 feA = shfl_down_f4(fwA), feB = shfl_down_f4(fwB);
        const float4 fB0 = shfl_f4(fwB, 0);
        if (lane == 31) {
            feA = fB0;
            feB = s_xe[row];
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const bool ok = k == 0 ? okA : okB;
            if (!ok) continue;
            const int c = lane + 32 * k;
            const int o = (row + 1) * ROWW + c + 4;
            const float4 fw = k == 0 ? fwA : fwB;
            const float4 fe = k == 0 ? feA : feB;
            const float4 gs = s_yf[row * FP_TX + c];
            const float4 gn = s_yf[(row + 1) * FP_TX + c];
            float h = __fmaf_rn(-ly, gn.x - gs.x, __fmaf_rn(-lx, fe.x - fw.x, s_h[o]));
            float hu = __fmaf_rn(-ly, gn.y - gs.y, __fmaf_rn(-lx, fe.y - fw.z, s_hu[o]));
            float hv = __fmaf_rn(-ly, gn.z - gs.w, __fmaf_rn(-lx, fe.w - fw.w, s_hv[o]));
            if (h < 0.0f) { neg += 1; h = 0.0f; }
            if (h <= FP_H_EPS_F) {
                hu = 0.0f; hv = 0.0f;
            } else {
                const float u = __fdividef(hu, h), v = __fdividef(hv, h);
                const float sp = sqrt_fast(__fmaf_rn(u, u, v * v));
                const unsigned short oc = k == 0 ? occA : occB;
                const float n0 = k == 0 ? n0A : n0B;
                const int np = oc < FP_NP_CAP ? oc : FP_NP_CAP;
                const float nm = S.coupling ? n0 + (float)np * n0 : n0;
                const float denom = __fmaf_rn(dt * g * nm * nm * sp, pow_m43(h), 1.0f);
                hu = __fdividef(hu, denom);
                hv = __fdividef(hv, denom);
            }
            if (!(h == h) || !(hu == hu) || !(hv == hv)) bad = 1;
            if (h > FP_H_EPS_F) {
                hk_[k] = h; huk_[k] = hu; hvk_[k] = hv;
                sk_[k] = __fdividef(fmaxf(fabsf(hu), fabsf(hv)), h) + sqrt_fast(g * h);
            }
            if (h >= FP_H_DRY_F) wet = 1;
            if (h != 0.0f) nz = 1;
            const size_t gi = gA + 32 * k;
            S.h[p2][gi] = h;
            S.hu[p2][gi] = hu;
            S.hv[p2][gi] = hv;
            if ((k == 0 ? occA : occB) != 0) S.occ[par][gi] = 0;
        }
        // water flags of the output plane's 64 x 8 blocks (h = 0 implies hu = hv = 0 above)
        if (__any_sync(0xffffffffu, nz) && lane == 0) atomicOr(&s_blk[row / FP_BLK_ROWS], 1);
        // CFL: the exact (correctly rounded) wave speed only for cells whose
        // approximate speed is within 1e-5 of the warp's approximate maximum -- the
        // approximation errs by < 1e-6, so the exact maximum is among them.  A
        // lane evaluates its faster candidate, and its other cell only when that
        // is a candidate too.  (Non-negative floats order as their bit patterns:
        // one warp-reduce instruction each.)
        float smax = 0.0f;
        {
            const float a = fmaxf(sk_[0], sk_[1]);
            const float amax = __uint_as_float(__reduce_max_sync(0xffffffffu, a >= 0.0f ? __float_as_uint(a) : 0u));
            const float thr = amax * (1.0f - 1e-5f);
            const bool c0 = sk_[0] >= 0.0f && sk_[0] >= thr, c1 = sk_[1] >= 0.0f && sk_[1] >= thr;
            const bool f1 = sk_[1] > sk_[0];  // cell B is the faster one
            if (c0 || c1)
                smax = fp_wave_speed(g, f1 ? hk_[1] : hk_[0], f1 ? huk_[1] : huk_[0], f1 ? hvk_[1] : hvk_[0]);
            if (c0 && c1)
                smax = fmaxf(smax, fp_wave_speed(g, f1 ? hk_[0] : hk_[1], f1 ? huk_[0] : huk_[1], f1 ? hvk_[0] : hvk_[1]));
        }
        // CTA reductions -> next clock slot
        smax = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(smax)));
        {
            const unsigned fl = __reduce_or_sync(0xffffffffu, (unsigned)(wet | (bad << 1)));
            wet = (int)(fl & 1u);
            bad = (int)(fl >> 1);
            neg = (int)__reduce_add_sync(0xffffffffu, (unsigned)neg);
        }
        if (lane == 0) {
            s_red[row] = smax;
            s_redi[row] = wet | (bad << 1) | (neg << 2);
        }
        __syncthreads();
        if (S.blk_wet[0] != nullptr && tid < TY / FP_BLK_ROWS && y0 + tid * FP_BLK_ROWS < ny)
            S.blk_wet[p2][(y0 / FP_BLK_ROWS + tid) * ((nx + FP_TX - 1) / FP_TX) + bx] = (unsigned char)s_blk[tid];
        // boundary tiles only: FP64 accumulation of the mass through the domain edges (one warp)
        const bool edge_x0 = x0 == 0, edge_x1 = x0 + FP_TX >= nx, edge_y0 = y0 == 0, edge_y1 = y0 + TY >= ny;
        if (row == TY - 2 && (edge_x0 || edge_x1 || edge_y0 || edge_y1)) {
            const double dtdx = (double)dt * (double)S.dx;
            for (int r = lane; r < TY; r += 32) {
                const int j = y0 + r;
                if (j >= ny) break;
                if (edge_x0) S.bflux[2 * nx + j] += (double)s_bx[0][r] * dtdx;
                if (edge_x1) S.bflux[2 * nx + ny + j] -= (double)s_bx[1][r] * dtdx;
            }
            for (int c = lane; c < FP_TX; c += 32) {
                const int i = x0 + c;
                if (i >= nx) break;
                if (edge_y0) S.bflux[i] += (double)s_by[0][c] * dtdx;
                if (edge_y1) S.bflux[nx + i] -= (double)s_by[1][c] * dtdx;
            }
        }
        if (row == TY - 1) {  // the control warp folds the tile's warp results into the CTA's
            const float m = lane < NT / 32 ? s_red[lane] : 0.0f;
            const int fl = lane < NT / 32 ? s_redi[lane] : 0;
            const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
            const unsigned fo = __reduce_or_sync(0xffffffffu, (unsigned)(fl & 3));
            const unsigned ng = __reduce_add_sync(0xffffffffu, (unsigned)(fl >> 2));
            if (lane == 0) {
                s_accm = fmaxf(s_accm, __uint_as_float(mb));
                s_accf |= (int)fo;
                s_accn += (int)ng;
                if (t == 0) {  // tile 0 advances the clock
                    FpClock *nxt = &S.clock[(slot + 1) & 3];
                    const long long dt_ticks = s_dt;
                    const long long t1 = s_t + dt_ticks;
                    if (S.dt_fixed > 0) {
                        float sm = __uint_as_float(s_smax0);
                        if (S.has_inflow && s_hin > FP_H_EPS_F) sm = fmaxf(sm, __fsqrt_rn(__fmul_rn(S.g, s_hin)));
                        if (__fmul_rn(sm, s_dtf) > __fmul_rn(S.cfl, S.dx)) atomicAdd(&S.cnt->cfl_over, 1u);
                    }
                    nxt->t = t1;
                    nxt->step = s_step + (dt_ticks > 0 ? 1 : 0);
                    nxt->h_in = (float)fp_hydro_depth(S, t1);
                    nxt->q_speed = fp_discharge_speed(S, t1);
                    if (S.clock[slot].wet) atomicOr(&nxt->wet, 1);
                    FpClock *old = &S.clock[(slot + 2) & 3];
                    old->smax_bits = 0u;
                    old->wet = 0;
                }
            }
        }
    }
    // the CTA's reductions -> the next clock slot
    if (tid == CTL) {
        FpClock *nxt = &S.clock[(slot + 1) & 3];
        if (s_accm > 0.0f) atomicMax(&nxt->smax_bits, __float_as_uint(s_accm));
        if (s_accf & 1) atomicOr(&nxt->wet, 1);
        if (s_accf & 2) fp_set_err(S, FP_ERR_NAN);
        if (s_accn) atomicAdd(&S.cnt->neg_depth, (unsigned long long)s_accn);
    }
    return true;
}

__device__ __forceinline__ void mbar_init(unsigned long long *mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

}  // namespace fpdev
