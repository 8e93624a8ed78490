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
// two-cell halo into shared memory (velocities formed once per cell), forms
// the face values of its cells and a one-cell ring, then every face of its
// cells once (a face between two CTAs is formed by both), then each thread
// updates its cell.  Stage 1 advances the
// clock; stage 2 takes the inflow depth of t + dt, averages, clears the
// evacuee counts it used and folds the wave-speed maximum, wet flag and
// tallies into the next step's clock.  Each stage adds half its boundary
// volumes.  No run ticket, no paired arithmetic, no dry skipping.
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

// a velocity q / h (0 where dry), sign-symmetric in q
__device__ __forceinline__ float vel(float q, float h) { return h > FP_H_EPS_F ? div_fast(q, h) : 0.0f; }

// The loaded region: depth, velocities, surface and bed per cell.
struct Region {
    float h[kRy][kRx], u[kRy][kRx], v[kRy][kRx], eta[kRy][kRx], z[kRy][kRx];
};

// face values of the cell at region (rx, ry) along x (ddx = 1) or y (ddy = 1);
// slope only if the flag allows it and the cell and both neighbours are wet
__device__ __forceinline__ FaceVals faces_of(const Region &R, int rx, int ry, int ddx, int ddy, bool slope) {
    const float hc = R.h[ry][rx], uc = R.u[ry][rx], vc = R.v[ry][rx], eta = R.eta[ry][rx];
    float se = 0.0f, sh = 0.0f, su = 0.0f, sv = 0.0f;
    const int xm = rx - ddx, ym = ry - ddy, xp = rx + ddx, yp = ry + ddy;
    const float hm = R.h[ym][xm], hp = R.h[yp][xp];
    if (slope && hc > FP_H_EPS_F && hm > FP_H_EPS_F && hp > FP_H_EPS_F) {
        se = minmod(__fsub_rn(R.eta[yp][xp], eta), __fsub_rn(eta, R.eta[ym][xm]));
        sh = minmod(__fsub_rn(hp, hc), __fsub_rn(hc, hm));
        su = minmod(__fsub_rn(R.u[yp][xp], uc), __fsub_rn(uc, R.u[ym][xm]));
        sv = minmod(__fsub_rn(R.v[yp][xp], vc), __fsub_rn(vc, R.v[ym][xm]));
    }
    FaceVals f;
    f.eta[0] = __fsub_rn(eta, 0.5f * se); f.eta[1] = __fadd_rn(eta, 0.5f * se);
    f.h[0] = __fsub_rn(hc, 0.5f * sh);    f.h[1] = __fadd_rn(hc, 0.5f * sh);
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
    __shared__ Region R;
    __shared__ FaceVals fx[kFy][kFx], fy[kFy][kFx];
    __shared__ FaceFlux xf[kMy][kMx + 1], yf[kMy + 1][kMx];
    const int nx = S.nx, ny = S.ny;
    const int x0 = blockIdx.x * kMx, y0 = blockIdx.y * kMy;
    const int tid = threadIdx.x;
    const FloodStep st = flood_step_consts(S, slot);
    if (STAGE == 1 && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) flood_clock_advance(S, slot, st);
    const float *ih = STAGE == 1 ? S.h[par] : S.mh, *ihu = STAGE == 1 ? S.hu[par] : S.mhu,
                *ihv = STAGE == 1 ? S.hv[par] : S.mhv;
    // the region with its two-cell halo (zeros outside the domain, never used),
    // loaded into registers first: the dry-tile test below runs beside the loads
    constexpr int kLoads = (kRx * kRy + kMx * kMy - 1) / (kMx * kMy);
    float lh[kLoads], lq[kLoads], lr[kLoads], lz[kLoads];
#pragma unroll
    for (int it = 0; it < kLoads; ++it) {
        const int k = tid + it * kMx * kMy;
        const int rx = k % kRx, ry = k / kRx, gi = x0 + rx - 2, gj = y0 + ry - 2;
        lh[it] = lq[it] = lr[it] = lz[it] = 0.0f;
        if (k < kRx * kRy && gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
            const size_t o = fp_pidx(S, gi, gj);
            lh[it] = ih[o]; lq[it] = ihu[o]; lr[it] = ihv[o]; lz[it] = S.z[o];
        }
    }
    // Dry tiles: when no cell this tile's faces reach holds water in the stage's
    // input (its 3 x 3 tile neighbourhood, all h = hu = hv = 0; for stage 2
    // also its own tile of the step's start state, which the average reads)
    // and it does not touch the domain edge (inflow, boundary fluxes), every
    // flux, slope term and friction term is zero and the output is zero: it
    // is written only where not already known to be zero, and the evacuee
    // counts the update would consume are cleared.  Interior tiles are full.
    const int tnx = gridDim.x, tny = gridDim.y, bx = blockIdx.x, by = blockIdx.y, tile = by * tnx + bx;
    const unsigned char *fin = S.mflag[0] == nullptr ? nullptr : STAGE == 1 ? S.mflag[par] : S.mflag[2];
    unsigned char *fout = S.mflag[0] == nullptr ? nullptr : STAGE == 1 ? S.mflag[2] : S.mflag[par ^ 1];
    if (fin != nullptr) {
        const bool edge = bx == 0 || by == 0 || bx == tnx - 1 || by == tny - 1;
        int wet = edge ? 1 : 0;
        if (!edge && tid < 9) wet = fin[(by - 1 + tid / 3) * tnx + bx - 1 + tid % 3] != 0;
        if (STAGE == 2 && !edge && tid == 9) wet = S.mflag[par][tile] != 0;
        if (!__syncthreads_or(wet)) {
            const bool need = fout[tile] != 0;
            const size_t o = fp_pidx(S, x0 + tid % kMx, y0 + tid / kMx);
            if (STAGE == 1) {
                if (need) {
                    S.mh[o] = 0.0f;
                    S.mhu[o] = 0.0f;
                    S.mhv[o] = 0.0f;
                }
            } else {
                const int p2 = par ^ 1;
                if (need) {
                    S.h[p2][o] = 0.0f;
                    S.hu[p2][o] = 0.0f;
                    S.hv[p2][o] = 0.0f;
                }
                if (S.occ[par][o] != 0) S.occ[par][o] = 0;
            }
            __syncthreads();  // every thread has read the flag
            if (need && tid == 0) fout[tile] = 0;
            return;
        }
    }
    const float h_in = STAGE == 1 ? st.h_in : S.clock[(slot + 1) & 3].h_in;
    const double half_dtdx = 0.5 * (double)st.dtf * (double)S.dx;
#pragma unroll
    for (int it = 0; it < kLoads; ++it) {
        const int k = tid + it * kMx * kMy;
        if (k >= kRx * kRy) continue;
        const int rx = k % kRx, ry = k / kRx;
        const float h = lh[it], z = lz[it];
        R.h[ry][rx] = h; R.u[ry][rx] = vel(lq[it], h); R.v[ry][rx] = vel(lr[it], h);
        R.eta[ry][rx] = __fadd_rn(h, z); R.z[ry][rx] = z;
    }
    __syncthreads();
    // face values of the cells and a one-cell ring
    for (int k = tid; k < kFx * kFy; k += kMx * kMy) {
        const int fxi = k % kFx, fyi = k / kFx, gi = x0 + fxi - 1, gj = y0 + fyi - 1;
        if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) continue;
        fx[fyi][fxi] = faces_of(R, fxi + 1, fyi + 1, 1, 0, gi > 0 && gi < nx - 1);
        fy[fyi][fxi] = faces_of(R, fxi + 1, fyi + 1, 0, 1, gj > 0 && gj < ny - 1);
    }
    __syncthreads();
    // every face of the CTA's cells once: x faces (kMx + 1 per row), then y
    // faces (kMy + 1 per column); a domain-edge face takes the ghost of its
    // edge cell, the breach's flux and the boundary volume
    for (int k = tid; k < kMy * (kMx + 1) + (kMy + 1) * kMx; k += kMx * kMy) {
        const bool xface = k < kMy * (kMx + 1);
        const int kk = xface ? k : k - kMy * (kMx + 1);
        const int a = xface ? kk % (kMx + 1) : kk % kMx, b = xface ? kk / (kMx + 1) : kk / kMx;
        // x face a of row b lies west of local cell a; y face b of column a south of local cell row b
        const int gi = x0 + a, gj = y0 + b;
        if (xface ? (gj >= ny || gi > nx) : (gi >= nx || gj > ny)) continue;
        const int n_ = xface ? nx : ny, gf = xface ? gi : gj;
        const unsigned char *bc = xface ? S.bc[gf == 0 ? 2 : 3] : S.bc[gf == 0 ? 0 : 1];
        const int along = xface ? gj : gi;
        float eL, hL, unL, utL, eR, hR, unR, utR;
        // own-side cells: local (a - 1, b) / (a, b) for x faces, (a, b - 1) / (a, b) for y faces
        const FaceVals *Lf = nullptr, *Rf = nullptr;
        if (gf > 0) Lf = xface ? &fx[b + 1][a] : &fy[b][a + 1];
        if (gf < n_) Rf = xface ? &fx[b + 1][a + 1] : &fy[b + 1][a + 1];
        if (Lf) { eL = Lf->eta[1]; hL = Lf->h[1]; unL = xface ? Lf->u[1] : Lf->v[1]; utL = xface ? Lf->v[1] : Lf->u[1]; }
        if (Rf) { eR = Rf->eta[0]; hR = Rf->h[0]; unR = xface ? Rf->u[0] : Rf->v[0]; utR = xface ? Rf->v[0] : Rf->u[0]; }
        if (gf == 0 || gf == n_) {
            // the edge cell's own state (no slope across the edge)
            const int rx = xface ? (gf == 0 ? a + 2 : a + 1) : a + 2, ry = xface ? b + 2 : (gf == 0 ? b + 2 : b + 1);
            const Side cell{R.h[ry][rx], R.u[ry][rx], R.v[ry][rx], R.z[ry][rx]};
            const Side gs = ghost(bc[along], cell, xface, h_in);
            const float ge = __fadd_rn(gs.h, gs.z);
            const float gn = xface ? gs.u : gs.v, gt = xface ? gs.v : gs.u;
            if (gf == 0) { eL = ge; hL = gs.h; unL = gn; utL = gt; }
            else { eR = ge; hR = gs.h; unR = gn; utR = gt; }
        }
        FaceFlux f = face_flux(S, eL, hL, unL, utL, eR, hR, unR, utR);
        if ((gf == 0 || gf == n_) && bc[along] == FP_BC_DISCHARGE) {
            f.m = gf == 0 ? __fadd_rn(f.m, st.qd.x) : __fsub_rn(f.m, st.qd.x);
            f.n = __fadd_rn(f.n, st.qd.y);
        }
        if (gf == 0) S.bflux[(xface ? 2 * nx : 0) + along] += (double)f.m * half_dtdx;
        if (gf == n_) S.bflux[(xface ? 2 * nx + ny : nx) + along] -= (double)f.m * half_dtdx;
        if (xface) xf[b][a] = f;
        else yf[b][a] = f;
    }
    __syncthreads();
    const int tx = tid % kMx, ty = tid / kMx, gi = x0 + tx, gj = y0 + ty;
    FloodAcc acc = flood_acc_init();
    int nz = 0;  // this cell's output holds water
    if (gi < nx && gj < ny) {
        const FaceFlux &W = xf[ty][tx], &E = xf[ty][tx + 1], &So = yf[ty][tx], &No = yf[ty + 1][tx];
        // x faces: (mass, u-momentum, v-momentum); y faces: (mass, v-momentum, u-momentum);
        // each cell's own side: R of its west / south face, L of its east / north face
        const float g = S.g, l = st.lx;
        const FaceVals &ax = fx[ty + 1][tx + 1], &ay = fy[ty + 1][tx + 1];
        const float sx = __fmul_rn(__fmul_rn(0.5f * g, __fadd_rn(ax.h[0], ax.h[1])), __fsub_rn(ax.eta[1], ax.eta[0]));
        const float sy = __fmul_rn(__fmul_rn(0.5f * g, __fadd_rn(ay.h[0], ay.h[1])), __fsub_rn(ay.eta[1], ay.eta[0]));
        const int rx = tx + 2, ry = ty + 2;
        const float hc = R.h[ry][rx];
        const size_t o = fp_pidx(S, gi, gj);
        const float quc = ihu[o], qvc = ihv[o];
        float hh = __fsub_rn(__fsub_rn(hc, __fmul_rn(l, __fsub_rn(E.m, W.m))), __fmul_rn(l, __fsub_rn(No.m, So.m)));
        float qu = __fsub_rn(__fsub_rn(__fsub_rn(quc, __fmul_rn(l, __fsub_rn(__fsub_rn(E.n, E.pL), __fsub_rn(W.n, W.pR)))),
                                       __fmul_rn(l, __fsub_rn(No.t, So.t))), __fmul_rn(l, sx));
        float qv = __fsub_rn(__fsub_rn(__fsub_rn(qvc, __fmul_rn(l, __fsub_rn(E.t, W.t))),
                                       __fmul_rn(l, __fsub_rn(__fsub_rn(No.n, No.pL), __fsub_rn(So.n, So.pR)))),
                             __fmul_rn(l, sy));
        if (hh < 0.0f) { acc.neg += 1; hh = 0.0f; }
        if (hh <= FP_H_EPS_F) {
            qu = 0.0f; qv = 0.0f;
        } else {
            // point-implicit Manning friction, n = n0 + N_p n0 (N_p <= 20)
            const float rh = rcp_fast(hh);
            const float u = __fmul_rn(qu, rh), v = __fmul_rn(qv, rh);
            const float sp = sqrt_fast(__fadd_rn(__fmul_rn(u, u), __fmul_rn(v, v)));
            const unsigned oc = S.occ[par][o];
            const float n0 = S.n0[o];
            const float nm = S.coupling ? __fadd_rn(n0, __fmul_rn((float)(oc < FP_NP_CAP ? oc : FP_NP_CAP), n0)) : n0;
            const float c = __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(st.dtf, g), nm), nm), sp);
            const float rd = rcp_fast(__fadd_rn(__fmul_rn(c, pow_m43(hh)), 1.0f));
            qu = __fmul_rn(qu, rd);
            qv = __fmul_rn(qv, rd);
        }
        if (STAGE == 1) {
            S.mh[o] = hh; S.mhu[o] = qu; S.mhv[o] = qv;
            nz = hh != 0.0f || qu != 0.0f || qv != 0.0f;
        } else {
            hh = 0.5f * __fadd_rn(S.h[par][o], hh);
            qu = 0.5f * __fadd_rn(S.hu[par][o], qu);
            qv = 0.5f * __fadd_rn(S.hv[par][o], qv);
            if (hh <= FP_H_EPS_F) { qu = 0.0f; qv = 0.0f; }
            const int p2 = par ^ 1;
            S.h[p2][o] = hh; S.hu[p2][o] = qu; S.hv[p2][o] = qv;
            nz = hh != 0.0f || qu != 0.0f || qv != 0.0f;
            if (S.occ[par][o] != 0) S.occ[par][o] = 0;
            if (!(hh == hh) || !(qu == qu) || !(qv == qv)) acc.bad = 1;
            if (hh > FP_H_EPS_F) acc.smax = fp_wave_speed(g, hh, qu, qv);
            if (hh >= FP_H_DRY_F) acc.wet = 1;
        }
    }
    if (fout != nullptr) {
        const int any = __syncthreads_or(nz);
        if (tid == 0) fout[tile] = any ? 1 : 0;
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
