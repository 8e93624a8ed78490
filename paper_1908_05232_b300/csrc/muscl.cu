// muscl.cu -- the flood update at second order: the cited scheme at full
// order (the paper runs it reduced to first order; a build-added option,
// fp_config.order = 2).  Per step two Euler stages of the same operator, the
// mean of the start state and the second stage's result (SSP-RK2):
//
//   reconstruction  per cell and direction, minmod slopes of the surface
//                   eta = h + z, of h and of the velocities u, v (zero on the
//                   domain edge and where the cell or a neighbour along that
//                   direction is dry): eta_f = eta +- s_eta/2, h_f, u_f, v_f;
//   faces           z_f = eta_f - h_f on each side, z* = max, h* = max(0,
//                   eta_f - z*), the HLL (or HLLC) flux of the two h* states;
//                   each cell takes the flux minus the pressure 1/2 g h*^2 of
//                   its own side, as at first order; edge faces take the ghost
//                   of the edge cell and the discharge breach's flux;
//   cell            the centred bed-slope term -g/2 (h_+ + h_-)(eta_+ - eta_-)
//                   per direction (a lake at rest, eta constant, stays exactly
//                   at rest), Eq. 2, point-implicit Manning friction with the
//                   evacuee roughness, every cell computed (no dry skipping).
//
// One thread per cell, CTAs of 32 x 8 cells; the CTA loads its cells with a
// two-cell halo into shared memory, forms the face values of its cells and a
// one-cell ring, then each thread forms its cell's four faces (a face between
// two CTAs is formed by both) and updates its cell.  Stage 1 advances the
// clock; stage 2 takes the inflow depth of t + dt, averages, clears the
// evacuee counts it used and folds the wave-speed maximum, wet flag and
// tallies into the next step's clock.  Each stage adds half its boundary
// volumes.  A correctness-first path: no run ticket, no paired arithmetic.
#include "flood_dev.cuh"
#include "floodped.h"

namespace {
using namespace fpdev;

constexpr int kMx = 32, kMy = 8;               // cells per CTA
constexpr int kRx = kMx + 4, kRy = kMy + 4;    // loaded region (two-cell halo)
constexpr int kFx = kMx + 2, kFy = kMy + 2;    // face values: cells and a one-cell ring

struct FaceVals {
    float eta[2], h[2], u[2], v[2];  // [0] minus side, [1] plus side
};

__device__ __forceinline__ float minmod(float a, float b) {
    if (a > 0.0f && b > 0.0f) return fminf(a, b);
    if (a < 0.0f && b < 0.0f) return fmaxf(a, b);
    return 0.0f;
}

__device__ __forceinline__ float vel(float q, float h) { return h > FP_H_EPS_F ? __fdiv_rn(q, h) : 0.0f; }

// face values of the cell at region (rx, ry) along x (dx = 1) or y (dy = 1);
// slope only if the flag allows it and the cell and both neighbours are wet
__device__ __forceinline__ FaceVals faces_of(const float (*sh)[kRx], const float (*shu)[kRx], const float (*shv)[kRx],
                                             const float (*sz)[kRx], int rx, int ry, int ddx, int ddy, bool slope) {
    const float hc = sh[ry][rx], z = sz[ry][rx];
    const float uc = vel(shu[ry][rx], hc), vc = vel(shv[ry][rx], hc);
    const float eta = __fadd_rn(hc, z);
    float se = 0.0f, sh_ = 0.0f, su = 0.0f, sv = 0.0f;
    const float hm = sh[ry - ddy][rx - ddx], hp = sh[ry + ddy][rx + ddx];
    if (slope && hc > FP_H_EPS_F && hm > FP_H_EPS_F && hp > FP_H_EPS_F) {
        const float em = __fadd_rn(hm, sz[ry - ddy][rx - ddx]), ep = __fadd_rn(hp, sz[ry + ddy][rx + ddx]);
        const float um = vel(shu[ry - ddy][rx - ddx], hm), up = vel(shu[ry + ddy][rx + ddx], hp);
        const float vm = vel(shv[ry - ddy][rx - ddx], hm), vp = vel(shv[ry + ddy][rx + ddx], hp);
        se = minmod(__fsub_rn(ep, eta), __fsub_rn(eta, em));
        sh_ = minmod(__fsub_rn(hp, hc), __fsub_rn(hc, hm));
        su = minmod(__fsub_rn(up, uc), __fsub_rn(uc, um));
        sv = minmod(__fsub_rn(vp, vc), __fsub_rn(vc, vm));
    }
    FaceVals f;
    f.eta[0] = __fsub_rn(eta, 0.5f * se); f.eta[1] = __fadd_rn(eta, 0.5f * se);
    f.h[0] = __fsub_rn(hc, 0.5f * sh_);   f.h[1] = __fadd_rn(hc, 0.5f * sh_);
    f.u[0] = __fsub_rn(uc, 0.5f * su);    f.u[1] = __fadd_rn(uc, 0.5f * su);
    f.v[0] = __fsub_rn(vc, 0.5f * sv);    f.v[1] = __fadd_rn(vc, 0.5f * sv);
    return f;
}

// One face from the two sides' (eta, h, normal, tangential velocity): the
// hydrostatic reconstruction, the flux (mass, normal momentum with pressure,
// tangential momentum) and the pressures of the two reconstructed depths.
struct FaceFlux {
    float m, n, t, pL, pR;
};

__device__ __forceinline__ FaceFlux face_flux(const FpSim &S, float eL, float hL, float unL, float utL, float eR,
                                              float hR, float unR, float utR) {
    const float g = S.g, hg = 0.5f * g;
    const float zL = __fsub_rn(eL, hL), zR = __fsub_rn(eR, hR);
    const float zf = fmaxf(zL, zR);
    const float hLs = fmaxf(0.0f, __fsub_rn(eL, zf)), hRs = fmaxf(0.0f, __fsub_rn(eR, zf));
    FaceFlux f;
    f.pL = press(hg, hLs);
    f.pR = press(hg, hRs);
    hll(g, hLs, unL, utL, f.pL, hRs, unR, utR, f.pR, f.m, f.n, f.t);
    if (S.riemann == 1 && !(hLs <= FP_H_EPS_F && hRs <= FP_H_EPS_F) && !(hLs == hRs && unL == unR && utL == utR)) {
        // HLLC: the tangential momentum rides on the mass flux with the
        // tangential velocity of the side the contact wave leaves behind
        const bool dL = hLs <= FP_H_EPS_F, dR = hRs <= FP_H_EPS_F;
        const float cL = __fsqrt_rn(g * hLs), cR = __fsqrt_rn(g * hRs);
        float sL, sR;
        if (dL) { sL = __fsub_rn(unR, 2.0f * cR); sR = __fadd_rn(unR, cR); }
        else if (dR) { sL = __fsub_rn(unL, cL); sR = __fadd_rn(unL, 2.0f * cL); }
        else {
            const float us = __fadd_rn(0.5f * __fadd_rn(unL, unR), __fsub_rn(cL, cR));
            const float cs = __fadd_rn(0.5f * __fadd_rn(cL, cR), 0.25f * __fsub_rn(unL, unR));
            sL = fminf(__fsub_rn(unL, cL), __fsub_rn(us, cs));
            sR = fmaxf(__fadd_rn(unR, cR), __fadd_rn(us, cs));
        }
        if (sL < 0.0f && sR > 0.0f) {
            const float a = __fmul_rn(hRs, __fsub_rn(unR, sR)), b = __fmul_rn(hLs, __fsub_rn(unL, sL));
            const float ss = __fdiv_rn(__fsub_rn(__fmul_rn(sL, a), __fmul_rn(sR, b)), __fsub_rn(a, b));
            const float ut = ss > 0.0f ? utL : (ss < 0.0f ? utR : 0.5f * __fadd_rn(utL, utR));
            f.t = __fmul_rn(f.m, ut);
        }
    }
    return f;
}

// stage 1: U -> U1 (into the scratch planes); stage 2: U1 -> U2, then
// U^{n+1} = (U + U2) / 2 into the other parity's planes
template <int STAGE>
__global__ void __launch_bounds__(kMx * kMy) muscl_stage_kernel(const __grid_constant__ FpSim S, int par, int slot) {
    __shared__ float sh[kRy][kRx], shu[kRy][kRx], shv[kRy][kRx], sz[kRy][kRx];
    __shared__ FaceVals fx[kFy][kFx], fy[kFy][kFx];
    const int nx = S.nx, ny = S.ny;
    const int x0 = blockIdx.x * kMx, y0 = blockIdx.y * kMy;
    const int tid = threadIdx.x;
    const FloodStep st = flood_step_consts(S, slot);
    if (STAGE == 1 && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) flood_clock_advance(S, slot, st);
    const float *ih = STAGE == 1 ? S.h[par] : S.mh, *ihu = STAGE == 1 ? S.hu[par] : S.mhu,
                *ihv = STAGE == 1 ? S.hv[par] : S.mhv;
    for (int k = tid; k < kRx * kRy; k += kMx * kMy) {
        const int rx = k % kRx, ry = k / kRx, gi = x0 + rx - 2, gj = y0 + ry - 2;
        float a = 0.0f, b = 0.0f, c = 0.0f, d = 0.0f;
        if (gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
            const size_t o = fp_pidx(S, gi, gj);
            a = ih[o]; b = ihu[o]; c = ihv[o]; d = S.z[o];
        }
        sh[ry][rx] = a; shu[ry][rx] = b; shv[ry][rx] = c; sz[ry][rx] = d;
    }
    __syncthreads();
    for (int k = tid; k < kFx * kFy; k += kMx * kMy) {
        const int fxi = k % kFx, fyi = k / kFx, gi = x0 + fxi - 1, gj = y0 + fyi - 1;
        if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) continue;
        fx[fyi][fxi] = faces_of(sh, shu, shv, sz, fxi + 1, fyi + 1, 1, 0, gi > 0 && gi < nx - 1);
        fy[fyi][fxi] = faces_of(sh, shu, shv, sz, fxi + 1, fyi + 1, 0, 1, gj > 0 && gj < ny - 1);
    }
    __syncthreads();
    const int tx = tid % kMx, ty = tid / kMx, gi = x0 + tx, gj = y0 + ty;
    const bool in = gi < nx && gj < ny;
    FloodAcc acc = flood_acc_init();
    if (in) {
        const float h_in = STAGE == 1 ? st.h_in : S.clock[(slot + 1) & 3].h_in;
        const double half_dtdx = 0.5 * (double)st.dtf * (double)S.dx;
        const int rx = tx + 2, ry = ty + 2, cx = tx + 1, cy = ty + 1;
        const float hc = sh[ry][rx], zc = sz[ry][rx];
        const Side cell{hc, vel(shu[ry][rx], hc), vel(shv[ry][rx], hc), zc};
        // x faces: west (own side R) and east (own side L)
        float mW, nW, tW, mE, nE, tE;
        {
            const FaceVals &c = fx[cy][cx];
            float eL, hL, uL, vL;
            if (gi == 0) {
                const Side gs = ghost(S.bc[2][gj], cell, true, h_in);
                eL = __fadd_rn(gs.h, gs.z); hL = gs.h; uL = gs.u; vL = gs.v;
            } else {
                const FaceVals &a = fx[cy][cx - 1];
                eL = a.eta[1]; hL = a.h[1]; uL = a.u[1]; vL = a.v[1];
            }
            FaceFlux f = face_flux(S, eL, hL, uL, vL, c.eta[0], c.h[0], c.u[0], c.v[0]);
            if (gi == 0 && S.bc[2][gj] == FP_BC_DISCHARGE) { f.m = __fadd_rn(f.m, st.qd.x); f.n = __fadd_rn(f.n, st.qd.y); }
            if (gi == 0) S.bflux[2 * nx + gj] += (double)f.m * half_dtdx;
            mW = f.m; nW = __fsub_rn(f.n, f.pR); tW = f.t;
            float eR, hR, uR, vR;
            if (gi == nx - 1) {
                const Side gs = ghost(S.bc[3][gj], cell, true, h_in);
                eR = __fadd_rn(gs.h, gs.z); hR = gs.h; uR = gs.u; vR = gs.v;
            } else {
                const FaceVals &b = fx[cy][cx + 1];
                eR = b.eta[0]; hR = b.h[0]; uR = b.u[0]; vR = b.v[0];
            }
            f = face_flux(S, c.eta[1], c.h[1], c.u[1], c.v[1], eR, hR, uR, vR);
            if (gi == nx - 1 && S.bc[3][gj] == FP_BC_DISCHARGE) { f.m = __fsub_rn(f.m, st.qd.x); f.n = __fadd_rn(f.n, st.qd.y); }
            if (gi == nx - 1) S.bflux[2 * nx + ny + gj] -= (double)f.m * half_dtdx;
            mE = f.m; nE = __fsub_rn(f.n, f.pL); tE = f.t;
        }
        // y faces: normal velocity v, tangential u
        float mS, nS, tS, mN, nN, tN;
        {
            const FaceVals &c = fy[cy][cx];
            float eL, hL, uL, vL;
            if (gj == 0) {
                const Side gs = ghost(S.bc[0][gi], cell, false, h_in);
                eL = __fadd_rn(gs.h, gs.z); hL = gs.h; uL = gs.u; vL = gs.v;
            } else {
                const FaceVals &a = fy[cy - 1][cx];
                eL = a.eta[1]; hL = a.h[1]; uL = a.u[1]; vL = a.v[1];
            }
            FaceFlux f = face_flux(S, eL, hL, vL, uL, c.eta[0], c.h[0], c.v[0], c.u[0]);
            if (gj == 0 && S.bc[0][gi] == FP_BC_DISCHARGE) { f.m = __fadd_rn(f.m, st.qd.x); f.n = __fadd_rn(f.n, st.qd.y); }
            if (gj == 0) S.bflux[gi] += (double)f.m * half_dtdx;
            mS = f.m; nS = __fsub_rn(f.n, f.pR); tS = f.t;
            float eR, hR, uR, vR;
            if (gj == ny - 1) {
                const Side gs = ghost(S.bc[1][gi], cell, false, h_in);
                eR = __fadd_rn(gs.h, gs.z); hR = gs.h; uR = gs.u; vR = gs.v;
            } else {
                const FaceVals &b = fy[cy + 1][cx];
                eR = b.eta[0]; hR = b.h[0]; uR = b.u[0]; vR = b.v[0];
            }
            f = face_flux(S, c.eta[1], c.h[1], c.v[1], c.u[1], eR, hR, vR, uR);
            if (gj == ny - 1 && S.bc[1][gi] == FP_BC_DISCHARGE) { f.m = __fsub_rn(f.m, st.qd.x); f.n = __fadd_rn(f.n, st.qd.y); }
            if (gj == ny - 1) S.bflux[nx + gi] -= (double)f.m * half_dtdx;
            mN = f.m; nN = __fsub_rn(f.n, f.pL); tN = f.t;
        }
        const float g = S.g, l = st.lx;
        const FaceVals &ax = fx[cy][cx], &ay = fy[cy][cx];
        const float sx = __fmul_rn(__fmul_rn(0.5f * g, __fadd_rn(ax.h[0], ax.h[1])), __fsub_rn(ax.eta[1], ax.eta[0]));
        const float sy = __fmul_rn(__fmul_rn(0.5f * g, __fadd_rn(ay.h[0], ay.h[1])), __fsub_rn(ay.eta[1], ay.eta[0]));
        float hh = __fsub_rn(__fsub_rn(hc, __fmul_rn(l, __fsub_rn(mE, mW))), __fmul_rn(l, __fsub_rn(mN, mS)));
        float qu = __fsub_rn(__fsub_rn(__fsub_rn(shu[ry][rx], __fmul_rn(l, __fsub_rn(nE, nW))),
                                       __fmul_rn(l, __fsub_rn(tN, tS))), __fmul_rn(l, sx));
        float qv = __fsub_rn(__fsub_rn(__fsub_rn(shv[ry][rx], __fmul_rn(l, __fsub_rn(tE, tW))),
                                       __fmul_rn(l, __fsub_rn(nN, nS))), __fmul_rn(l, sy));
        if (hh < 0.0f) { acc.neg += 1; hh = 0.0f; }
        const size_t o = fp_pidx(S, gi, gj);
        if (hh <= FP_H_EPS_F) {
            qu = 0.0f; qv = 0.0f;
        } else {
            // point-implicit Manning friction, n = n0 + N_p n0 (N_p <= 20)
            const float u = __fdiv_rn(qu, hh), v = __fdiv_rn(qv, hh);
            const float sp = __fsqrt_rn(__fadd_rn(__fmul_rn(u, u), __fmul_rn(v, v)));
            const unsigned oc = S.occ[par][o];
            const float n0 = S.n0[o];
            const float nm = S.coupling ? __fadd_rn(n0, __fmul_rn((float)(oc < FP_NP_CAP ? oc : FP_NP_CAP), n0)) : n0;
            const float c = __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(st.dtf, g), nm), nm), sp);
            const float denom = __fadd_rn(__fmul_rn(c, pow_m43(hh)), 1.0f);
            qu = __fdiv_rn(qu, denom);
            qv = __fdiv_rn(qv, denom);
        }
        if (STAGE == 1) {
            S.mh[o] = hh; S.mhu[o] = qu; S.mhv[o] = qv;
        } else {
            const float h0 = S.h[par][o];
            hh = 0.5f * __fadd_rn(h0, hh);
            qu = 0.5f * __fadd_rn(S.hu[par][o], qu);
            qv = 0.5f * __fadd_rn(S.hv[par][o], qv);
            if (hh <= FP_H_EPS_F) { qu = 0.0f; qv = 0.0f; }
            const int p2 = par ^ 1;
            S.h[p2][o] = hh; S.hu[p2][o] = qu; S.hv[p2][o] = qv;
            if (S.occ[par][o] != 0) S.occ[par][o] = 0;
            if (!(hh == hh) || !(qu == qu) || !(qv == qv)) acc.bad = 1;
            if (hh > FP_H_EPS_F) acc.smax = fp_wave_speed(g, hh, qu, qv);
            if (hh >= FP_H_DRY_F) acc.wet = 1;
        }
    }
    if (STAGE == 1) {
        const unsigned ng = __reduce_add_sync(0xffffffffu, (unsigned)acc.neg);
        if ((tid & 31) == 0 && ng) atomicAdd(&S.cnt->neg_depth, (unsigned long long)ng);
    } else {
        flood_acc_fold_cta<kMx * kMy / 32>(S, slot, acc);
    }
}

}  // namespace

void fp_launch_muscl(const FpSim &S, int par, int slot, cudaStream_t st) {
    const dim3 grid((S.nx + kMx - 1) / kMx, (S.ny + kMy - 1) / kMy);
    muscl_stage_kernel<1><<<grid, kMx * kMy, 0, st>>>(S, par, slot);
    muscl_stage_kernel<2><<<grid, kMx * kMy, 0, st>>>(S, par, slot);
}
