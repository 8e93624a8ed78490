// flood_dev.cuh -- device code of the hydrodynamic cell update (Section 2.2),
// shared by the per-step flood kernel, the batched-ensemble kernel and the
// persistent coupled-step kernel.
//
// The grid is cut into runs of 64 columns x TY rows; one warp takes a run and
// marches north through it (flood_march): lane l owns two neighbouring cells
// of every row, loaded with coalesced float2 loads of h, hu, hv, z (and n0,
// the evacuee counts), and keeps the previous row's cells, their x-flux
// differences and their south-face fluxes in registers, so every face is
// formed once, with no shared memory and no barrier inside a run:
//   - per face: non-negative hydrostatic reconstruction h* = max(0, eta -
//     max(z_L, z_R)) and the HLL flux; each side keeps the flux minus the
//     pressure 1/2 g h*^2 of its own reconstructed depth (this carries the
//     bed-slope source of Eq. 1); domain-edge faces use ghost states from the
//     boundary codes, a discharge breach adds its inflow;
//   - per cell: Eq. (2), point-implicit Manning friction with n = n0 + N_p n0
//     (N_p <= 20); the CFL wave-speed maximum of U^{n+1} (exact only for
//     candidates) and the wet flag are reduced per warp and folded into the
//     next step's clock slot; edge faces add their mass fluxes in FP64.
// 8-row groups whose cells and halo stayed dry are skipped (their update
// would write zeros).
// Built with -fmad=false: every fused multiply-add is written out, and each one
// is sign-symmetric, so the update is exactly mirror-symmetric and gives the
// same bits in every kernel it is inlined into and whatever the run height.
#pragma once
#include "fp_common.cuh"

namespace fpdev {


// Single-instruction approximations (relative error ~1e-7) with denormal
// inputs and results flushed to zero: every value they see here is a depth
// above h_eps, a wave speed or a velocity, far from the denormal range, so the
// flush changes nothing and saves the denormal handling of the plain forms.
__device__ __forceinline__ float sqrt_fast(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// a / b as a times the approximate reciprocal of b (sign-symmetric in a)
__device__ __forceinline__ float div_fast(float a, float b) { return __fmul_rn(a, rcp_fast(b)); }

// h^(-4/3) = 2^(-4/3 log2 h) for h > 0 (two special-function instructions)
__device__ __forceinline__ float pow_m43(float h) {
    float l, r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(h));
    const float e = -1.33333333f * l;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e));
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

// ---- paired FP32 arithmetic: two faces or two cells per instruction ---------
// fma.rn.f32x2 rounds each half exactly as the scalar fma.rn does.  Products
// and sums are written as fused multiply-adds with a run-time 1 and -0 (K2),
// so that the code generator merges none of them into a neighbour: a b + (-0)
// and a 1 + b round once, to the bits of the plain product and sum.
struct K2 {
    float2 one, nz;
};
__device__ __forceinline__ K2 make_k2(const FpSim &S) {
    const float one = __fdiv_rn(S.dx, S.dx), nz = -__fmul_rn(0.0f, S.dx);
    return K2{make_float2(one, one), make_float2(nz, nz)};
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{ .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
        " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd; }"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2_mul(const K2 &k, float2 a, float2 b) { return f2_fma(a, b, k.nz); }
__device__ __forceinline__ float2 f2_add(const K2 &k, float2 a, float2 b) { return f2_fma(a, k.one, b); }
__device__ __forceinline__ float2 f2_sub(const K2 &k, float2 a, float2 b) { return f2_fma(f2_neg(b), k.one, a); }
__device__ __forceinline__ float2 f2_max0(float2 a) { return make_float2(fmaxf(0.0f, a.x), fmaxf(0.0f, a.y)); }
__device__ __forceinline__ float2 f2_sqrt(float2 a) { return make_float2(sqrt_fast(a.x), sqrt_fast(a.y)); }
__device__ __forceinline__ float2 f2_rcp(float2 a) { return make_float2(rcp_fast(a.x), rcp_fast(a.y)); }
__device__ __forceinline__ float2 f2_sel(bool cx, bool cy, float2 t, float2 f) {
    return make_float2(cx ? t.x : f.x, cy ? t.y : f.y);
}

// Two face sides (depth, normal and tangential velocity, bed) and two faces'
// fluxes: mass, normal momentum minus the L-side pressure, minus the R-side
// pressure, tangential momentum.
struct Sides2 {
    float2 h, un, ut, z;
};
struct Flux2 {
    float2 m, nl, nr, t;
};

// Two faces at once, each by the per-face definition: non-negative hydrostatic
// reconstruction z_f = max(z_L, z_R), h* = max(0, h + z - z_f); the HLL flux
// with Einfeldt-type wave speeds (dry-bed speeds when a side is dry: the left
// side's test first); in this order of precedence: both sides dry (no flux),
// identical states or s_L >= 0 (left flux), s_R <= 0 (right flux), the HLL
// average (identical states give the physical flux exactly: a lake at rest
// stays exactly at rest); then a discharge breach's inflow (dir = +1 / -1 into
// the domain, 0 elsewhere: qd.x mass, qd.y momentum); each side keeps the
// normal flux minus the pressure 1/2 g h*^2 of its own side.  Differences of
// two products are rounded explicitly, so a mirrored face gives exactly the
// mirrored flux.
__device__ __forceinline__ Flux2 face2(const K2 &k, float g, float hg, const Sides2 &L, const Sides2 &R, float2 dir,
                                       float2 qd, bool hllc) {
    const float2 zf = make_float2(fmaxf(L.z.x, R.z.x), fmaxf(L.z.y, R.z.y));
    const float2 hL = f2_max0(f2_sub(k, f2_add(k, L.h, L.z), zf));
    const float2 hR = f2_max0(f2_sub(k, f2_add(k, R.h, R.z), zf));
    const float2 pL = f2_mul(k, f2_mul(k, f2(hg), hL), hL), pR = f2_mul(k, f2_mul(k, f2(hg), hR), hR);
    const bool dLx = hL.x <= FP_H_EPS_F, dLy = hL.y <= FP_H_EPS_F, dRx = hR.x <= FP_H_EPS_F, dRy = hR.y <= FP_H_EPS_F;
    const bool nfx = dLx && dRx, nfy = dLy && dRy;  // no flow: both sides dry
    float2 fm = f2(0.0f), fn = f2(0.0f), ft = f2(0.0f);
    if (!(nfx && nfy)) {
        const float2 qL = f2_mul(k, hL, L.un), qR = f2_mul(k, hR, R.un);
        const float2 FL1 = f2_fma(qL, L.un, pL), FL2 = f2_mul(k, qL, L.ut);
        const float2 FR1 = f2_fma(qR, R.un, pR), FR2 = f2_mul(k, qR, R.ut);
        const float2 cL = f2_sqrt(f2_mul(k, f2(g), hL)), cR = f2_sqrt(f2_mul(k, f2(g), hR));
        const float2 us = f2_fma(f2(0.5f), f2_add(k, L.un, R.un), f2_sub(k, cL, cR));
        const float2 cs = f2_fma(f2(0.25f), f2_sub(k, L.un, R.un), f2_mul(k, f2(0.5f), f2_add(k, cL, cR)));
        const float2 a = f2_sub(k, L.un, cL), b = f2_sub(k, us, cs);
        const float2 c = f2_add(k, R.un, cR), d = f2_add(k, us, cs);
        float2 sL = make_float2(a.x < b.x ? a.x : b.x, a.y < b.y ? a.y : b.y);
        float2 sR = make_float2(c.x > d.x ? c.x : d.x, c.y > d.y ? c.y : d.y);
        sL = f2_sel(dRx, dRy, a, sL);
        sR = f2_sel(dRx, dRy, f2_fma(f2(2.0f), cL, L.un), sR);
        sL = f2_sel(dLx, dLy, f2_fma(f2(-2.0f), cR, R.un), sL);
        sR = f2_sel(dLx, dLy, c, sR);
        const float2 inv = f2_rcp(f2_sub(k, sR, sL));
        const float2 sLR = f2_mul(k, sL, sR);
        const float2 am = f2_add(k, f2_sub(k, f2_mul(k, sR, qL), f2_mul(k, sL, qR)), f2_mul(k, sLR, f2_sub(k, hR, hL)));
        const float2 an = f2_add(k, f2_sub(k, f2_mul(k, sR, FL1), f2_mul(k, sL, FR1)), f2_mul(k, sLR, f2_sub(k, qR, qL)));
        const float2 at = f2_add(k, f2_sub(k, f2_mul(k, sR, FL2), f2_mul(k, sL, FR2)),
                                 f2_mul(k, sLR, f2_sub(k, f2_mul(k, hR, R.ut), f2_mul(k, hL, L.ut))));
        fm = f2_mul(k, am, inv);
        fn = f2_mul(k, an, inv);
        ft = f2_mul(k, at, inv);
        if (hllc) {
            // HLLC: the tangential momentum rides on the mass flux with the
            // tangential velocity of the side the contact wave S* leaves behind
            // (S* > 0: left, S* < 0: right, S* = 0: their mean); S* =
            // (sL hR (uR - sR) - sR hL (uL - sL)) / (hR (uR - sR) - hL (uL - sL)),
            // whose sign flips exactly under a mirror
            const float2 num = f2_sub(k, f2_mul(k, f2_mul(k, sL, hR), f2_sub(k, R.un, sR)),
                                      f2_mul(k, f2_mul(k, sR, hL), f2_sub(k, L.un, sL)));
            const float2 den = f2_sub(k, f2_mul(k, hR, f2_sub(k, R.un, sR)), f2_mul(k, hL, f2_sub(k, L.un, sL)));
            const float2 ss = f2_mul(k, num, f2_rcp(den));
            const float2 mid = f2_mul(k, f2(0.5f), f2_add(k, L.ut, R.ut));
            const float2 ut = make_float2(ss.x > 0.0f ? L.ut.x : (ss.x < 0.0f ? R.ut.x : mid.x),
                                          ss.y > 0.0f ? L.ut.y : (ss.y < 0.0f ? R.ut.y : mid.y));
            ft = f2_mul(k, fm, ut);
        }
        const bool rx = sR.x <= 0.0f, ry = sR.y <= 0.0f;
        fm = f2_sel(rx, ry, qR, fm);
        fn = f2_sel(rx, ry, FR1, fn);
        ft = f2_sel(rx, ry, FR2, ft);
        const bool lx = sL.x >= 0.0f || (hL.x == hR.x && L.un.x == R.un.x && L.ut.x == R.ut.x);
        const bool ly = sL.y >= 0.0f || (hL.y == hR.y && L.un.y == R.un.y && L.ut.y == R.ut.y);
        fm = f2_sel(lx, ly, qL, fm);
        fn = f2_sel(lx, ly, FL1, fn);
        ft = f2_sel(lx, ly, FL2, ft);
        fm = f2_sel(nfx, nfy, f2(0.0f), fm);
        fn = f2_sel(nfx, nfy, f2(0.0f), fn);
        ft = f2_sel(nfx, nfy, f2(0.0f), ft);
    }
    if (dir.x != 0.0f || dir.y != 0.0f) {
        const float2 m2 = f2_fma(dir, f2(qd.x), fm), n2 = f2_add(k, fn, f2(qd.y));
        fm = f2_sel(dir.x != 0.0f, dir.y != 0.0f, m2, fm);
        fn = f2_sel(dir.x != 0.0f, dir.y != 0.0f, n2, fn);
    }
    return Flux2{fm, f2_sub(k, fn, pL), f2_sub(k, fn, pR), ft};
}

// A cell as a face side: depth, velocities (0 at h <= h_eps), bed.
__device__ __forceinline__ Side make_side(float h, float hu, float hv, float z) {
    Side c{h, 0.0f, 0.0f, z};
    if (h > FP_H_EPS_F) {
        const float r = rcp_fast(h);
        c.u = __fmul_rn(hu, r);
        c.v = __fmul_rn(hv, r);
    }
    return c;
}

// The lane's two cells of a row as two face sides (element x: cell i0, y: i1).
struct Cells2 {
    float2 h, u, v, z;
};
__device__ __forceinline__ Cells2 make_cells2(const K2 &k, float2 h, float2 hu, float2 hv, float2 z) {
    const float2 r = f2_rcp(h);
    const float2 u = f2_mul(k, hu, r), v = f2_mul(k, hv, r);
    const bool wx = h.x > FP_H_EPS_F, wy = h.y > FP_H_EPS_F;
    return Cells2{h, f2_sel(wx, wy, u, f2(0.0f)), f2_sel(wx, wy, v, f2(0.0f)), z};
}
__device__ __forceinline__ Side side_x(const Cells2 &c) { return Side{c.h.x, c.u.x, c.v.x, c.z.x}; }
__device__ __forceinline__ Side side_y(const Cells2 &c) { return Side{c.h.y, c.u.y, c.v.y, c.z.y}; }

// Two sides as face inputs, normal velocity u (x faces) or v (y faces).
__device__ __forceinline__ Sides2 sides_x(Side a, Side b) {
    return Sides2{make_float2(a.h, b.h), make_float2(a.u, b.u), make_float2(a.v, b.v), make_float2(a.z, b.z)};
}
__device__ __forceinline__ Sides2 sides_y(Side a, Side b) {
    return Sides2{make_float2(a.h, b.h), make_float2(a.v, b.v), make_float2(a.u, b.u), make_float2(a.z, b.z)};
}

// Per-step constants of the flood update, the same for every run of a step.
struct FloodStep {
    long long dt;    // ticks
    float dtf, lx;   // dt (s), dt / dx
    float h_in;      // depth of the depth-inflow ghost
    float2 qd;       // discharge breach over the step: mass flux q and the momentum q u_in it carries
    int inflow_on;   // an inflow can enter: runs at a domain edge always compute
};

__device__ __forceinline__ FloodStep flood_step_consts(const FpSim &S, int slot) {
    const FpClock c = S.clock[slot];
    FloodStep st;
    st.dt = fp_dt_ticks(S, c, c.h_in);
    st.dtf = (float)st.dt * (1.0f / FP_TICKS_F);
    st.lx = __fdiv_rn(st.dtf, S.dx);
    st.h_in = c.h_in;
    // the discharge breach: mean unit discharge over [t, t + dt] from the exact
    // volume of the hydrograph, and the momentum it carries
    st.qd = make_float2(0.0f, 0.0f);
    if (S.has_discharge && st.dt > 0) {
        const double t0 = __ddiv_rn((double)c.t, 1048576.0), t1 = __ddiv_rn((double)(c.t + st.dt), 1048576.0);
        const double dV = __dsub_rn(fp_discharge_volume(S, t1), fp_discharge_volume(S, t0));
        const double q = __ddiv_rn(dV, __dmul_rn(__ddiv_rn((double)st.dt, 1048576.0), S.q_width));
        st.qd = make_float2((float)q, (float)__dmul_rn(q, __ddiv_rn(q, S.h_qin)));
    }
    // an inflow is active while the depth hydrograph is above h_eps or the
    // discharge hydrograph has not ended
    st.inflow_on = ((S.has_inflow && c.h_in > FP_H_EPS_F) || (S.has_discharge && c.t < S.q_end_ticks)) ? 1 : 0;
    return st;
}

// The next step's clock (slot + 1): time, step index, inflow depth and inflow
// speed; the Courant check of a fixed step; slot + 2 cleared for the folds of
// the step after.  One thread per step.
__device__ __forceinline__ void flood_clock_advance(const FpSim &S, int slot, const FloodStep &st) {
    const FpClock c = S.clock[slot];
    FpClock *nxt = &S.clock[(slot + 1) & 3];
    const long long t1 = c.t + st.dt;
    if (S.dt_fixed > 0) {
        float sm = __uint_as_float(c.smax_bits);
        if (S.has_inflow && c.h_in > FP_H_EPS_F) sm = fmaxf(sm, __fsqrt_rn(__fmul_rn(S.g, c.h_in)));
        if (c.q_speed > 0.0f) sm = fmaxf(sm, c.q_speed);
        if (__fmul_rn(sm, st.dtf) > __fmul_rn(S.cfl, S.dx)) atomicAdd(&S.cnt->cfl_over, 1u);
    }
    nxt->t = t1;
    nxt->step = c.step + (st.dt > 0 ? 1 : 0);
    nxt->h_in = (float)fp_hydro_depth(S, t1);
    nxt->q_speed = fp_discharge_speed(S, t1);
    if (c.wet) atomicOr(&nxt->wet, 1);
    FpClock *old = &S.clock[(slot + 2) & 3];
    old->smax_bits = 0u;
    old->wet = 0;
}

// What a warp accumulates over its runs: the exact CFL wave-speed maximum of
// its lane's candidate cells, the warp's running approximate maximum (the same
// on every lane), and the wet / non-finite / negative-depth tallies.
struct FloodAcc {
    float smax, amax;
    int wet, bad, neg;
};

__device__ __forceinline__ FloodAcc flood_acc_init() { return FloodAcc{0.0f, 0.0f, 0, 0, 0}; }

// Folds a warp's accumulators into the clock of the next step and the counters
// (lane 0's atomics; every lane must call).
__device__ __forceinline__ void flood_acc_fold_warp(const FpSim &S, int slot, const FloodAcc &a) {
    const unsigned sm = __reduce_max_sync(0xffffffffu, __float_as_uint(a.smax));
    const unsigned fl = __reduce_or_sync(0xffffffffu, (unsigned)(a.wet | (a.bad << 1)));
    const unsigned ng = __reduce_add_sync(0xffffffffu, (unsigned)a.neg);
    if ((threadIdx.x & 31) == 0) {
        FpClock *nxt = &S.clock[(slot + 1) & 3];
        if (sm) atomicMax(&nxt->smax_bits, sm);
        if (fl & 1u) atomicOr(&nxt->wet, 1);
        if (fl & 2u) fp_set_err(S, FP_ERR_NAN);
        if (ng) atomicAdd(&S.cnt->neg_depth, (unsigned long long)ng);
    }
}

// The same folded over the CTA first (one set of atomics per CTA); every
// thread of the CTA must call.
template <int NW>
__device__ __forceinline__ void flood_acc_fold_cta(const FpSim &S, int slot, const FloodAcc &a) {
    __shared__ unsigned s_sm[NW], s_fl[NW], s_ng[NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned sm = __reduce_max_sync(0xffffffffu, __float_as_uint(a.smax));
    const unsigned fl = __reduce_or_sync(0xffffffffu, (unsigned)(a.wet | (a.bad << 1)));
    const unsigned ng = __reduce_add_sync(0xffffffffu, (unsigned)a.neg);
    if (lane == 0) {
        s_sm[w] = sm;
        s_fl[w] = fl;
        s_ng[w] = ng;
    }
    __syncthreads();
    if (w == 0) {
        const unsigned m = __reduce_max_sync(0xffffffffu, lane < NW ? s_sm[lane] : 0u);
        const unsigned f = __reduce_or_sync(0xffffffffu, lane < NW ? s_fl[lane] : 0u);
        const unsigned n = __reduce_add_sync(0xffffffffu, lane < NW ? s_ng[lane] : 0u);
        if (lane == 0) {
            FpClock *nxt = &S.clock[(slot + 1) & 3];
            if (m) atomicMax(&nxt->smax_bits, m);
            if (f & 1u) atomicOr(&nxt->wet, 1);
            if (f & 2u) fp_set_err(S, FP_ERR_NAN);
            if (n) atomicAdd(&S.cnt->neg_depth, (unsigned long long)n);
        }
    }
    __syncthreads();
}

// Rows ys..ye-1 (at most 32) of the 64 columns x0..x0+63 by one warp, marching
// north: lane l owns cells i0 = x0 + 2l and i1 = i0 + 1 of every row, and does
// their arithmetic on paired FP32 instructions.  Per row j the warp has the two
// cells' h, hu, hv, z (coalesced float2 loads issued one row ahead; lane 31
// also loads the cell just east of the run), forms the two y faces between row
// j - 1, carried in registers, and row j, then finishes row j - 1 (Eq. (2)
// with its carried x-flux differences and south-face fluxes, point-implicit
// Manning friction, wet / CFL tallies, stores), then forms row j's two x faces:
// the face between the lane's cells and the face east of them (its east side
// by shuffle), the west face arriving by shuffle from the lane below (lane 0:
// the run's west face of the row, formed for all rows at once before the
// march).  Row ys - 1 enters only through its faces with row ys, and row ye
// (the next run's first, or the north ghost row) only through its faces with
// row ye - 1.  Every face and every update is the per-face / per-cell
// definition, so the result does not depend on how the rows are split into
// runs.  Loads are plain (coherent) global loads: in the persistent kernel the
// planes read in one step were written by other SMs in the step before.
template <bool EDGE, bool HLLC>
__device__ __forceinline__ void flood_march(const FpSim &S, int par, const FloodStep &st, int x0, int ys, int ye,
                                            FloodAcc &acc) {
    constexpr bool edge = EDGE;
    const int lane = threadIdx.x & 31;
    const int nx = S.nx, ny = S.ny, p2 = par ^ 1;
    const int bw = (nx + FP_TX - 1) / FP_TX, bx = x0 / FP_TX;
    const int i0 = x0 + 2 * lane, i1 = i0 + 1;
    const bool v0 = i0 < nx, v1 = i1 < nx;
    const bool ld = i1 <= nx + 3;                      // the pair lies inside the padded row
    const bool ldh = lane == 31 && x0 + FP_TX <= nx;  // the cell east of the run (lane 31's east neighbour)
    const K2 k = make_k2(S);
    constexpr bool hllc = HLLC;
    const float g = S.g, hg = 0.5f * g;
    const float dt = st.dtf, h_in = st.h_in;
    const float2 nlx = f2(-st.lx), nly = f2(-st.lx), qd = st.qd, zero2 = f2(0.0f);
    const double dtdx = (double)dt * (double)S.dx;
    const float *hp = S.h[par], *hup = S.hu[par], *hvp = S.hv[par], *zp = S.z, *n0p = S.n0;
    const unsigned short *occp = S.occ[par];

    // the cells of row ys - 1
    Cells2 prev;
    {
        const size_t o = fp_pidx(S, i0, ys - 1);
        float2 h = zero2, hu = zero2, hv = zero2, z = zero2;
        if (ld) {
            h = *reinterpret_cast<const float2 *>(hp + o);
            hu = *reinterpret_cast<const float2 *>(hup + o);
            hv = *reinterpret_cast<const float2 *>(hvp + o);
            z = *reinterpret_cast<const float2 *>(zp + o);
        }
        prev = make_cells2(k, h, hu, hv, z);
    }
    // the pair of row ys, loaded ahead
    float2 nH = zero2, nHU = zero2, nHV = zero2, nZ = zero2;
    auto fetch = [&](int j) {
        const size_t o = fp_pidx(S, i0, j);
        if (ld) {
            nH = *reinterpret_cast<const float2 *>(hp + o);
            nHU = *reinterpret_cast<const float2 *>(hup + o);
            nHV = *reinterpret_cast<const float2 *>(hvp + o);
            nZ = *reinterpret_cast<const float2 *>(zp + o);
        } else {
            nH = nHU = nHV = nZ = zero2;
        }
    };
    fetch(ys);
    // The west faces of the march's rows (between cells x0 - 1 and x0), formed
    // together up front: lane k forms row ys + k's (a march has at most 32
    // rows); at row j lane 0 takes it from lane j - ys.
    float wM = 0.0f, wN = 0.0f, wT = 0.0f;
    {
        const int jb = ys + lane;
        if (jb < ye) {
            const size_t ob = fp_pidx(S, x0, jb);
            Side L = make_side(hp[ob - 1], hup[ob - 1], hvp[ob - 1], zp[ob - 1]);
            const Side R = make_side(hp[ob], hup[ob], hvp[ob], zp[ob]);
            float dir = 0.0f;
            if (edge && x0 == 0) {
                const unsigned char c = S.bc[2][jb];
                L = ghost(c, R, true, h_in);
                if (c == 3) dir = 1.0f;
            }
            const Flux2 f = face2(k, g, hg, sides_x(L, L), sides_x(R, R), f2(dir), qd, hllc);
            wM = f.m.x;
            wN = f.nr.x;
            wT = f.t.x;
            if (edge && x0 == 0) S.bflux[2 * nx + jb] += (double)wM * dtdx;
        }
    }
    // carried for row j - 1 (elements: cells i0, i1): conserved values, n0 and
    // evacuee counts, x-flux differences (east face - west face: mass, x
    // momentum, y momentum) and the south-face flux (mass, x momentum, y
    // momentum minus the cell's own pressure)
    float2 uH = zero2, uHU = zero2, uHV = zero2, uN0 = zero2;
    unsigned uOcc = 0u;
    float2 dM = zero2, dU = zero2, dV = zero2, sM = zero2, sU = zero2, sV = zero2;
    int nz = 0;
    for (int j = ys; j <= ye; ++j) {
        const float2 h = nH, hu = nHU, hv = nHV, z = nZ;
        // this row's n0, evacuee counts and east halo cell
        const size_t o = fp_pidx(S, i0, j);
        float2 n0 = zero2;
        unsigned occ = 0u;
        float4 hx = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < ye) {
            if (ld) {
                n0 = *reinterpret_cast<const float2 *>(n0p + o);
                occ = *reinterpret_cast<const unsigned *>(occp + o);
            }
            if (ldh) hx = make_float4(hp[o + 2], hup[o + 2], hvp[o + 2], zp[o + 2]);
            fetch(j + 1);
        }
        const Cells2 cur = make_cells2(k, h, hu, hv, z);
        // the two y faces between rows j - 1 and j
        Flux2 gy;
        if (!edge) {
            gy = face2(k, g, hg, Sides2{prev.h, prev.v, prev.u, prev.z}, Sides2{cur.h, cur.v, cur.u, cur.z}, zero2, qd, hllc);
        } else {
            Side B0 = side_x(prev), B1 = side_y(prev), A0 = side_x(cur), A1 = side_y(cur);
            float2 dir = zero2;
            if (j == 0) {
                const unsigned char c0 = v0 ? S.bc[0][i0] : 0, c1 = v1 ? S.bc[0][i1] : 0;
                B0 = ghost(c0, A0, false, h_in);
                B1 = ghost(c1, A1, false, h_in);
                dir = make_float2(c0 == 3 ? 1.0f : 0.0f, c1 == 3 ? 1.0f : 0.0f);
            }
            if (j == ny) {
                const unsigned char c0 = v0 ? S.bc[1][i0] : 0, c1 = v1 ? S.bc[1][i1] : 0;
                A0 = ghost(c0, B0, false, h_in);
                A1 = ghost(c1, B1, false, h_in);
                dir = make_float2(c0 == 3 ? -1.0f : 0.0f, c1 == 3 ? -1.0f : 0.0f);
            }
            gy = face2(k, g, hg, sides_y(B0, B1), sides_y(A0, A1), dir, qd, hllc);
            // no face past the east edge
            gy.m = f2_sel(!v0, !v1, zero2, gy.m);
            gy.nl = f2_sel(!v0, !v1, zero2, gy.nl);
            gy.nr = f2_sel(!v0, !v1, zero2, gy.nr);
            gy.t = f2_sel(!v0, !v1, zero2, gy.t);
            if (j == 0) {
                if (v0) S.bflux[i0] += (double)gy.m.x * dtdx;
                if (v1) S.bflux[i1] += (double)gy.m.y * dtdx;
            }
            if (j == ny) {
                if (v0) S.bflux[nx + i0] -= (double)gy.m.x * dtdx;
                if (v1) S.bflux[nx + i1] -= (double)gy.m.y * dtdx;
            }
        }
        // finish row j - 1
        if (j > ys) {
            const int jr = j - 1;
            float2 hh = f2_fma(nly, f2_sub(k, gy.m, sM), f2_fma(nlx, dM, uH));
            float2 qu = f2_fma(nly, f2_sub(k, gy.t, sU), f2_fma(nlx, dU, uHU));
            float2 qv = f2_fma(nly, f2_sub(k, gy.nl, sV), f2_fma(nlx, dV, uHV));
            const bool ngx = hh.x < 0.0f, ngy = hh.y < 0.0f;
            acc.neg += (v0 && ngx ? 1 : 0) + (v1 && ngy ? 1 : 0);
            hh = f2_sel(ngx, ngy, zero2, hh);
            const bool wx = hh.x > FP_H_EPS_F, wy = hh.y > FP_H_EPS_F;
            {
                // point-implicit Manning friction, n = n0 + N_p n0 (N_p <= 20)
                const float2 r = f2_rcp(hh);
                const float2 u = f2_mul(k, qu, r), v = f2_mul(k, qv, r);
                const float2 sp = f2_sqrt(f2_fma(u, u, f2_mul(k, v, v)));
                const unsigned oc0 = uOcc & 0xffffu, oc1 = uOcc >> 16;
                const float2 np = make_float2((float)(oc0 < FP_NP_CAP ? oc0 : FP_NP_CAP),
                                              (float)(oc1 < FP_NP_CAP ? oc1 : FP_NP_CAP));
                const float2 nm = S.coupling ? f2_add(k, uN0, f2_mul(k, np, uN0)) : uN0;
                const float2 c = f2_mul(k, f2_mul(k, f2_mul(k, f2_mul(k, f2(dt), f2(g)), nm), nm), sp);
                const float2 denom = f2_fma(c, make_float2(pow_m43(hh.x), pow_m43(hh.y)), k.one);
                const float2 rd = f2_rcp(denom);
                qu = f2_sel(wx, wy, f2_mul(k, qu, rd), zero2);
                qv = f2_sel(wx, wy, f2_mul(k, qv, rd), zero2);
            }
            if ((v0 && (!(hh.x == hh.x) || !(qu.x == qu.x) || !(qv.x == qv.x))) ||
                (v1 && (!(hh.y == hh.y) || !(qu.y == qu.y) || !(qv.y == qv.y))))
                acc.bad = 1;
            // approximate wave speeds max(|u|,|v|) + sqrt(g h) of the wet cells
            const float2 vm = make_float2(fmaxf(fabsf(qu.x), fabsf(qv.x)), fmaxf(fabsf(qu.y), fabsf(qv.y)));
            const float2 sk2 = f2_add(k, f2_mul(k, vm, f2_rcp(hh)), f2_sqrt(f2_mul(k, f2(g), hh)));
            const float sk0 = v0 && wx ? sk2.x : -1.0f, sk1 = v1 && wy ? sk2.y : -1.0f;
            if ((v0 && hh.x >= FP_H_DRY_F) || (v1 && hh.y >= FP_H_DRY_F)) acc.wet = 1;
            if ((v0 && hh.x != 0.0f) || (v1 && hh.y != 0.0f)) nz = 1;
            const size_t oo = fp_pidx(S, i0, jr);
            if (v1) {
                *reinterpret_cast<float2 *>(S.h[p2] + oo) = hh;
                *reinterpret_cast<float2 *>(S.hu[p2] + oo) = qu;
                *reinterpret_cast<float2 *>(S.hv[p2] + oo) = qv;
            } else if (v0) {
                S.h[p2][oo] = hh.x;
                S.hu[p2][oo] = qu.x;
                S.hv[p2][oo] = qv.x;
            }
            if (uOcc != 0u) {
                if (v1) *reinterpret_cast<unsigned *>(S.occ[par] + oo) = 0u;
                else if (v0) S.occ[par][oo] = 0;
            }
            // CFL: the exact (correctly rounded) wave speed only for cells whose
            // approximate speed is within 1e-5 of the warp's running approximate
            // maximum -- the approximation errs by < 1e-6, so every cell whose
            // exact speed can be the maximum is evaluated
            {
                const float a = fmaxf(sk0, sk1);
                const unsigned am = __reduce_max_sync(0xffffffffu, a >= 0.0f ? __float_as_uint(a) : 0u);
                acc.amax = fmaxf(acc.amax, __uint_as_float(am));
                const float thr = acc.amax * (1.0f - 1e-5f);
                if (sk0 >= 0.0f && sk0 >= thr) acc.smax = fmaxf(acc.smax, fp_wave_speed(g, hh.x, qu.x, qv.x));
                if (sk1 >= 0.0f && sk1 >= thr) acc.smax = fmaxf(acc.smax, fp_wave_speed(g, hh.y, qu.y, qv.y));
            }
            // water flag of the output plane's 64 x 8 block, at its last row
            if ((jr & (FP_BLK_ROWS - 1)) == FP_BLK_ROWS - 1 || jr == ye - 1) {
                const bool any = __any_sync(0xffffffffu, nz);
                if (lane == 0) {
                    const int q = (jr / FP_BLK_ROWS) * bw + bx;
                    if (S.blk_wet[0] != nullptr) S.blk_wet[p2][q] = any ? 1 : 0;
                    if (S.blk_runs != nullptr) S.blk_runs[q] += 1u;
                }
                nz = 0;
            }
        }
        if (j == ye) break;
        // the two x faces of row j: between the lane's cells (at i1) and east of
        // them (at i1 + 1, its east side from the lane above or the halo)
        Side east;
        {
            const Side hs = make_side(hx.x, hx.y, hx.z, hx.w);
            east.h = __shfl_down_sync(0xffffffffu, cur.h.x, 1);
            east.u = __shfl_down_sync(0xffffffffu, cur.u.x, 1);
            east.v = __shfl_down_sync(0xffffffffu, cur.v.x, 1);
            east.z = __shfl_down_sync(0xffffffffu, cur.z.x, 1);
            if (lane == 31) east = hs;
        }
        Flux2 fx;
        if (!edge) {
            fx = face2(k, g, hg, Sides2{cur.h, cur.u, cur.v, cur.z},
                       Sides2{make_float2(cur.h.y, east.h), make_float2(cur.u.y, east.u), make_float2(cur.v.y, east.v),
                              make_float2(cur.z.y, east.z)},
                       zero2, qd, hllc);
        } else {
            const Side L0 = side_x(cur), L1 = side_y(cur);
            Side R0 = side_y(cur), R1 = east;
            float2 dir = zero2;
            if (i1 == nx) {
                const unsigned char c = S.bc[3][j];
                R0 = ghost(c, L0, true, h_in);
                if (c == 3) dir.x = -1.0f;
            }
            if (i1 + 1 == nx) {
                const unsigned char c = S.bc[3][j];
                R1 = ghost(c, L1, true, h_in);
                if (c == 3) dir.y = -1.0f;
            }
            fx = face2(k, g, hg, sides_x(L0, L1), sides_x(R0, R1), dir, qd, hllc);
            const bool px = i1 > nx, py = i1 + 1 > nx;  // no face past the east edge
            fx.m = f2_sel(px, py, zero2, fx.m);
            fx.nl = f2_sel(px, py, zero2, fx.nl);
            fx.nr = f2_sel(px, py, zero2, fx.nr);
            fx.t = f2_sel(px, py, zero2, fx.t);
            double *bf = S.bflux + 2 * nx;
            if (i1 == nx) bf[ny + j] -= (double)fx.m.x * dtdx;
            if (i1 + 1 == nx) bf[ny + j] -= (double)fx.m.y * dtdx;
        }
        // the west face of cell i0: the east face of the lane below; lane 0's is
        // the run's west face of this row
        float wm = __shfl_up_sync(0xffffffffu, fx.m.y, 1);
        float wn = __shfl_up_sync(0xffffffffu, fx.nr.y, 1);
        float wt = __shfl_up_sync(0xffffffffu, fx.t.y, 1);
        {
            const float m = __shfl_sync(0xffffffffu, wM, j - ys), n = __shfl_sync(0xffffffffu, wN, j - ys),
                        t = __shfl_sync(0xffffffffu, wT, j - ys);
            if (lane == 0) { wm = m; wn = n; wt = t; }
        }
        dM = f2_sub(k, fx.m, make_float2(wm, fx.m.x));
        dU = f2_sub(k, fx.nl, make_float2(wn, fx.nr.x));
        dV = f2_sub(k, fx.t, make_float2(wt, fx.t.x));
        sM = gy.m;
        sU = gy.t;
        sV = gy.nr;
        uH = h; uHU = hu; uHV = hv; uN0 = n0; uOcc = occ;
        prev = cur;
    }
}

// One run: 64 columns x TY rows (run r at column block r % bw, rows from
// (r / bw) TY), by one warp.  Each 8-row group is
//   left alone when the tile mask excludes the run;
//   skipped    when no 64 x 8 block of it or of its one-cell halo held water
//              after the last step (flags of the input plane), its own block
//              of the output plane already holds the zero state (flags from
//              two steps back) and no inflow is active at a domain edge it
//              touches: every flux is zero and the update would write zeros,
//              so nothing is loaded and only the evacuee counts it read are
//              cleared;
//   computed   otherwise.
// Consecutive computed groups form one march.
template <int TY>
__device__ __forceinline__ void flood_run(const FpSim &S, int par, const FloodStep &st, int run, FloodAcc &acc) {
    constexpr int NG = TY / FP_BLK_ROWS;
    static_assert(TY % FP_BLK_ROWS == 0 && NG >= 1 && NG <= 4, "whole water-flag blocks");
    const int lane = threadIdx.x & 31;
    const int nx = S.nx, ny = S.ny, bw = (nx + FP_TX - 1) / FP_TX;
    const int bx = run % bw, x0 = bx * FP_TX, y0 = (run / bw) * TY;
    if (y0 >= ny) return;
    const int y1 = min(y0 + TY, ny);
    const int ng = (y1 - y0 + FP_BLK_ROWS - 1) / FP_BLK_ROWS;
    const bool flags = S.blk_wet[0] != nullptr;
    const bool masked = S.tile_mask != nullptr && S.tile_mask[run] == 0;
    const bool xedge = x0 == 0 || x0 + FP_TX >= nx;
    // modes: two groups per pass, lanes 0-15 for the first, 16-31 for the second
    unsigned load = 0u, dry = 0u;
    if (!masked) {
        for (int k0 = 0; k0 < ng; k0 += 2) {
            const int k = k0 + (lane >> 4), q = lane & 15;
            int f = 0;
            if (k < ng && flags) {
                const int y = y0 + k * FP_BLK_ROWS;
                const int r0 = max(0, y - 1) / FP_BLK_ROWS, r1 = min(ny - 1, y + FP_BLK_ROWS) / FP_BLK_ROWS;
                const int c0 = max(0, bx - 1), c1 = min(bw - 1, bx + 1);
                const int nc = c1 - c0 + 1, nin = (r1 - r0 + 1) * nc;
                if (q < nin) f = S.blk_wet[par][(r0 + q / nc) * bw + c0 + q % nc];
                else if (q == nin) f = S.blk_wet[par ^ 1][(y / FP_BLK_ROWS) * bw + bx];
            }
            const unsigned wetb = __ballot_sync(0xffffffffu, f != 0);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kk = k0 + h;
                if (kk >= ng) break;
                const int y = y0 + kk * FP_BLK_ROWS;
                const bool any = ((wetb >> (16 * h)) & 0xffffu) != 0u;
                const bool edge = xedge || y == 0 || y + FP_BLK_ROWS >= ny;
                if (flags && !any && !(st.inflow_on && edge)) dry |= 1u << kk;
                else load |= 1u << kk;
            }
        }
    }
    // dry groups: the evacuee counts this step read are cleared all the same
    if (dry) {
        const int i0 = x0 + 2 * lane;
        for (int k = 0; k < ng; ++k) {
            if (!((dry >> k) & 1u)) continue;
            const int ya = y0 + k * FP_BLK_ROWS, yb = min(ya + FP_BLK_ROWS, ny);
            for (int j = ya; j < yb; ++j) {
                const size_t o = fp_pidx(S, i0, j);
                if (i0 + 1 < nx) *reinterpret_cast<unsigned *>(S.occ[par] + o) = 0u;
                else if (i0 < nx) S.occ[par][o] = 0;
            }
        }
    }
    // marches over the runs of consecutive computed groups
    const bool edge = xedge || y0 == 0 || y1 >= ny;
    for (int k = 0; k < ng;) {
        if (!((load >> k) & 1u)) { ++k; continue; }
        int k1 = k;
        while (k1 + 1 < ng && ((load >> (k1 + 1)) & 1u)) ++k1;
        const int ys = y0 + k * FP_BLK_ROWS, ye = min(y0 + (k1 + 1) * FP_BLK_ROWS, ny);
        if (S.riemann == 1) {
            if (edge) flood_march<true, true>(S, par, st, x0, ys, ye, acc);
            else flood_march<false, true>(S, par, st, x0, ys, ye, acc);
        } else {
            if (edge) flood_march<true, false>(S, par, st, x0, ys, ye, acc);
            else flood_march<false, false>(S, par, st, x0, ys, ye, acc);
        }
        k = k1 + 1;
    }
}

}  // namespace fpdev
