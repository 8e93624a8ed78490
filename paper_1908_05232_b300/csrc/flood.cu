// flood.cu -- hydrodynamic cell update of the coupled step (Section 2.2).
//
// flood_kernel<TY>: one CTA per 64 x TY tile of cells.
//   1. one thread issues four 2D TMA loads (cp.async.bulk.tensor) of the tile
//      plus a one-cell halo (a 72-float-wide box starting 16-byte aligned) of
//      h, hu, hv, z into shared memory, completing on an mbarrier; meanwhile
//      every thread loads its four cells' n0 and evacuee counts;
//   2. velocities u = hu/h, v = hv/h per staged cell;
//   3. every x and y face of the tile once: non-negative hydrostatic
//      reconstruction h* = max(0, eta - max(z_L, z_R)) and the HLL flux;
//      each side keeps the flux minus the pressure 1/2 g h*^2 of its own
//      reconstructed depth (this carries the bed-slope source of Eq. 1);
//      domain-edge faces use ghost states from the boundary codes;
//   4. Eq. (2) per cell, point-implicit Manning friction with
//      n = n0 + N_p n0 (N_p <= 20), writes U^{n+1} as 16-byte vectors;
//      the CFL wave-speed max of U^{n+1} and the wet flag are reduced per CTA
//      (warp shuffles) and folded into the next step's clock slot with one
//      atomic each.
// Compiled with -fmad=false so that the update is exactly mirror-symmetric.
#include "fp_common.cuh"

namespace {

constexpr int ROWW = FP_TX + 8;  // staged row width: 4 guard floats each side

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float sqrt_fast(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float press(float g, float h) { return 0.5f * g * h * h; }

// HLL flux across a face; un normal and ut tangential velocity.  out = (mass,
// normal momentum incl. pressure, tangential momentum).  Identical states give
// the physical flux exactly (lake at rest stays exactly at rest).
__device__ __forceinline__ void hll(float g, float hL, float unL, float utL, float hR, float unR, float utR,
                                    float &fm, float &fn, float &ft) {
    if (hL <= FP_H_EPS_F && hR <= FP_H_EPS_F) {
        fm = 0.0f; fn = 0.0f; ft = 0.0f;
        return;
    }
    const float qL = hL * unL, qR = hR * unR;
    const float FL0 = qL, FL1 = qL * unL + press(g, hL), FL2 = qL * utL;
    const float FR0 = qR, FR1 = qR * unR + press(g, hR), FR2 = qR * utR;
    if (hL == hR && unL == unR && utL == utR) {
        fm = FL0; fn = FL1; ft = FL2;
        return;
    }
    const float cL = sqrt_fast(g * hL), cR = sqrt_fast(g * hR);
    float sL, sR;
    if (hL <= FP_H_EPS_F) {
        sL = unR - 2.0f * cR;
        sR = unR + cR;
    } else if (hR <= FP_H_EPS_F) {
        sL = unL - cL;
        sR = unL + 2.0f * cL;
    } else {
        const float us = 0.5f * (unL + unR) + (cL - cR);
        const float cs = 0.5f * (cL + cR) + 0.25f * (unL - unR);
        const float a = unL - cL, b = us - cs;
        sL = a < b ? a : b;
        const float c = unR + cR, d = us + cs;
        sR = c > d ? c : d;
    }
    if (sL >= 0.0f) { fm = FL0; fn = FL1; ft = FL2; return; }
    if (sR <= 0.0f) { fm = FR0; fn = FR1; ft = FR2; return; }
    const float den = sR - sL;
    const float sLR = sL * sR;
    fm = __fdividef(sR * FL0 - sL * FR0 + sLR * (hR - hL), den);
    fn = __fdividef(sR * FL1 - sL * FR1 + sLR * (qR - qL), den);
    ft = __fdividef(sR * FL2 - sL * FR2 + sLR * (hR * utR - hL * utL), den);
}

struct Side {
    float h, u, v, z;
};

__device__ __forceinline__ Side ghost(unsigned char code, Side in, bool normal_x, float h_in) {
    Side g = in;
    if (code == 0) {
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

template <int TY>
__host__ __device__ constexpr int smem_bytes() {
    return 6 * plane_stride<TY>() * 4 + TY * (FP_TX + 1) * 16 + (TY + 1) * FP_TX * 16;
}

template <int TY>
__global__ void __launch_bounds__(16 * TY) flood_kernel(const __grid_constant__ FpTmaSet tm,
                                                        const __grid_constant__ FpSim S, int par, int slot) {
    constexpr int NT = 16 * TY;
    constexpr int PLANE = plane_stride<TY>();
    constexpr int BOX_BYTES = (TY + 2) * ROWW * 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *s_h = reinterpret_cast<float *>(smem_raw);
    float *s_hu = s_h + PLANE;
    float *s_hv = s_hu + PLANE;
    float *s_z = s_hv + PLANE;
    float *s_u = s_z + PLANE;
    float *s_v = s_u + PLANE;
    float4 *s_xf = reinterpret_cast<float4 *>(s_v + PLANE);  // [TY][65]
    float4 *s_yf = s_xf + TY * (FP_TX + 1);                   // [TY+1][64]
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ long long s_dt, s_t, s_step;
    __shared__ float s_hin;
    __shared__ int s_ok;
    __shared__ float s_red[NT / 32];
    __shared__ int s_redi[NT / 32];

    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * FP_TX, y0 = blockIdx.y * TY;
    const int nx = S.nx, ny = S.ny;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned bar = smem_u32(&mbar);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(4 * BOX_BYTES)
                     : "memory");
        const CUtensorMap *maps[4] = {&tm.h, &tm.hu, &tm.hv, &tm.z};
        float *dsts[4] = {s_h, s_hu, s_hv, s_z};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
                    smem_u32(dsts[k])),
                "l"(reinterpret_cast<unsigned long long>(maps[k])), "r"(x0), "r"(y0), "r"(bar)
                : "memory");
        }
        const FpClock c = S.clock[slot];
        const float hin = (float)fp_hydro_depth(S, c.t);
        s_hin = hin;
        s_dt = fp_dt_ticks(S, c, hin);
        s_t = c.t;
        s_step = c.step;
    }
    // this thread's four cells: n0 and evacuee counts, loaded while the TMA is in flight
    const int tx = tid & 15, ty = tid >> 4;
    const int ci0 = x0 + 4 * tx, cj = y0 + ty;
    const bool row_ok = cj < ny && ci0 < nx;
    const bool full = row_ok && ci0 + 4 <= nx;
    float4 n0v = make_float4(0.f, 0.f, 0.f, 0.f);
    ushort4 occv = make_ushort4(0, 0, 0, 0);
    size_t gidx = 0;
    if (row_ok) {
        gidx = fp_pidx(S, ci0, cj);
        n0v = *reinterpret_cast<const float4 *>(S.n0 + gidx);
        occv = *reinterpret_cast<const ushort4 *>(S.occ + gidx);
    }
    if (tid == 0) {
        const unsigned bar = smem_u32(&mbar);
        unsigned ok = 0;
        for (int it = 0; it < (1 << 22) && !ok; ++it) {
            asm volatile(
                "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                : "=r"(ok)
                : "r"(bar)
                : "memory");
        }
        s_ok = ok;
        if (!ok) fp_set_err(S, FP_ERR_TIMEOUT);
    }
    __syncthreads();
    if (!s_ok) return;

    const float g = S.g;
    const long long dt_ticks = s_dt;
    const float dt = (float)dt_ticks * (1.0f / FP_TICKS_F);
    const float h_in = s_hin;

    // 2. velocities of staged cells x0-1 .. x0+64 (staged columns 3 .. 68)
    for (int idx = tid; idx < (TY + 2) * (FP_TX + 2); idx += NT) {
        const int r = idx / (FP_TX + 2), cc = idx % (FP_TX + 2) + 3;
        const int o = r * ROWW + cc;
        const float h = s_h[o];
        float u = 0.0f, v = 0.0f;
        if (h > FP_H_EPS_F) {
            u = __fdividef(s_hu[o], h);
            v = __fdividef(s_hv[o], h);
        }
        s_u[o] = u;
        s_v[o] = v;
    }
    __syncthreads();

    // 3a. x faces: face k of row r lies between cells x0+k-1 and x0+k
    const double dtdx = (double)dt * (double)S.dx;
    for (int idx = tid; idx < TY * (FP_TX + 1); idx += NT) {
        const int r = idx / (FP_TX + 1), k = idx % (FP_TX + 1);
        const int j = y0 + r, xl = x0 + k - 1, xr = x0 + k;
        if (j >= ny || xr > nx) continue;
        const int oL = (r + 1) * ROWW + k + 3, oR = oL + 1;
        Side L, R;
        if (xr < nx) R = Side{s_h[oR], s_u[oR], s_v[oR], s_z[oR]};
        if (xl >= 0) L = Side{s_h[oL], s_u[oL], s_v[oL], s_z[oL]};
        if (xl < 0) L = ghost(S.bc[2][j], R, true, h_in);
        if (xr == nx) R = ghost(S.bc[3][j], L, true, h_in);
        const float zf = fmaxf(L.z, R.z);
        const float hLs = fmaxf(0.0f, (L.h + L.z) - zf);
        const float hRs = fmaxf(0.0f, (R.h + R.z) - zf);
        float fm, fn, ft;
        hll(g, hLs, L.u, L.v, hRs, R.u, R.v, fm, fn, ft);
        s_xf[r * (FP_TX + 1) + k] = make_float4(fm, fn - press(g, hLs), fn - press(g, hRs), ft);
        if (xl < 0) S.bflux[2 * nx + j] += (double)fm * dtdx;
        if (xr == nx) S.bflux[2 * nx + ny + j] -= (double)fm * dtdx;
    }
    // 3b. y faces: face r of column c lies between rows y0+r-1 and y0+r
    for (int idx = tid; idx < (TY + 1) * FP_TX; idx += NT) {
        const int r = idx / FP_TX, c = idx % FP_TX;
        const int i = x0 + c, jb = y0 + r - 1, ja = y0 + r;
        if (i >= nx || ja > ny) continue;
        const int oB = r * ROWW + c + 4, oA = oB + ROWW;
        Side B, A;
        if (ja < ny) A = Side{s_h[oA], s_u[oA], s_v[oA], s_z[oA]};
        if (jb >= 0) B = Side{s_h[oB], s_u[oB], s_v[oB], s_z[oB]};
        if (jb < 0) B = ghost(S.bc[0][i], A, false, h_in);
        if (ja == ny) A = ghost(S.bc[1][i], B, false, h_in);
        const float zf = fmaxf(B.z, A.z);
        const float hBs = fmaxf(0.0f, (B.h + B.z) - zf);
        const float hAs = fmaxf(0.0f, (A.h + A.z) - zf);
        float fm, fn, ft;
        hll(g, hBs, B.v, B.u, hAs, A.v, A.u, fm, fn, ft);
        s_yf[r * FP_TX + c] = make_float4(fm, ft, fn - press(g, hBs), fn - press(g, hAs));
        if (jb < 0) S.bflux[i] += (double)fm * dtdx;
        if (ja == ny) S.bflux[nx + i] -= (double)fm * dtdx;
    }
    __syncthreads();

    // 4. Eq. (2) + friction for this thread's four cells
    float smax = 0.0f;
    int wet = 0, neg = 0, bad = 0;
    if (row_ok) {
        const float lx = __fdiv_rn(dt, S.dx);
        const float ly = lx;
        float outh[4], outhu[4], outhv[4];
        const float n0a[4] = {n0v.x, n0v.y, n0v.z, n0v.w};
        const unsigned short occa[4] = {occv.x, occv.y, occv.z, occv.w};
        const float4 hq = *reinterpret_cast<const float4 *>(s_h + (ty + 1) * ROWW + 4 * tx + 4);
        const float4 huq = *reinterpret_cast<const float4 *>(s_hu + (ty + 1) * ROWW + 4 * tx + 4);
        const float4 hvq = *reinterpret_cast<const float4 *>(s_hv + (ty + 1) * ROWW + 4 * tx + 4);
        const float ha[4] = {hq.x, hq.y, hq.z, hq.w};
        const float hua[4] = {huq.x, huq.y, huq.z, huq.w};
        const float hva[4] = {hvq.x, hvq.y, hvq.z, hvq.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (ci0 + k >= nx) { outh[k] = 0.0f; outhu[k] = 0.0f; outhv[k] = 0.0f; continue; }
            const float4 fw = s_xf[ty * (FP_TX + 1) + 4 * tx + k];
            const float4 fe = s_xf[ty * (FP_TX + 1) + 4 * tx + k + 1];
            const float4 gs = s_yf[ty * FP_TX + 4 * tx + k];
            const float4 gn = s_yf[(ty + 1) * FP_TX + 4 * tx + k];
            float h = ha[k] - lx * (fe.x - fw.x) - ly * (gn.x - gs.x);
            float hu = hua[k] - lx * (fe.y - fw.z) - ly * (gn.y - gs.y);
            float hv = hva[k] - lx * (fe.w - fw.w) - ly * (gn.z - gs.w);
            if (h < 0.0f) { neg += 1; h = 0.0f; }
            if (h <= FP_H_EPS_F) {
                hu = 0.0f; hv = 0.0f;
            } else {
                const float u = __fdividef(hu, h), v = __fdividef(hv, h);
                const float sp = sqrt_fast(u * u + v * v);
                const int np = occa[k] < FP_NP_CAP ? occa[k] : FP_NP_CAP;
                const float nm = S.coupling ? n0a[k] + (float)np * n0a[k] : n0a[k];
                const float denom = 1.0f + dt * g * nm * nm * sp / (h * cbrtf(h));
                hu = __fdividef(hu, denom);
                hv = __fdividef(hv, denom);
            }
            if (!(h == h) || !(hu == hu) || !(hv == hv)) bad = 1;
            outh[k] = h; outhu[k] = hu; outhv[k] = hv;
            if (h > FP_H_EPS_F) smax = fmaxf(smax, fp_wave_speed(g, h, hu, hv));
            if (h >= FP_H_DRY_F) wet = 1;
        }
        const int p2 = par ^ 1;
        if (full) {
            *reinterpret_cast<float4 *>(S.h[p2] + gidx) = make_float4(outh[0], outh[1], outh[2], outh[3]);
            *reinterpret_cast<float4 *>(S.hu[p2] + gidx) = make_float4(outhu[0], outhu[1], outhu[2], outhu[3]);
            *reinterpret_cast<float4 *>(S.hv[p2] + gidx) = make_float4(outhv[0], outhv[1], outhv[2], outhv[3]);
            if (occv.x | occv.y | occv.z | occv.w)
                *reinterpret_cast<ushort4 *>(S.occ + gidx) = make_ushort4(0, 0, 0, 0);
        } else {
            for (int k = 0; k < 4; ++k) {
                if (ci0 + k >= nx) break;
                S.h[p2][gidx + k] = outh[k];
                S.hu[p2][gidx + k] = outhu[k];
                S.hv[p2][gidx + k] = outhv[k];
                if (occa[k]) S.occ[gidx + k] = 0;
            }
        }
    }
    // CTA reductions -> next clock slot
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        wet |= __shfl_xor_sync(0xffffffffu, wet, o);
        neg += __shfl_xor_sync(0xffffffffu, neg, o);
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((tid & 31) == 0) {
        s_red[tid >> 5] = smax;
        s_redi[tid >> 5] = wet | (bad << 1) | (neg << 2);
    }
    __syncthreads();
    if (tid == 0) {
        float m = 0.0f;
        int w = 0, b = 0, ng = 0;
        for (int k = 0; k < NT / 32; ++k) {
            m = fmaxf(m, s_red[k]);
            w |= s_redi[k] & 1;
            b |= (s_redi[k] >> 1) & 1;
            ng += s_redi[k] >> 2;
        }
        FpClock *nxt = &S.clock[(slot + 1) & 3];
        if (m > 0.0f) atomicMax(&nxt->smax_bits, __float_as_uint(m));
        if (w) atomicOr(&nxt->wet, 1);
        if (b) fp_set_err(S, FP_ERR_NAN);
        if (ng) atomicAdd(&S.cnt->neg_depth, (unsigned long long)ng);
        if (blockIdx.x == 0 && blockIdx.y == 0) {
            nxt->t = s_t + dt_ticks;
            nxt->step = s_step + (dt_ticks > 0 ? 1 : 0);
            if (S.clock[slot].wet) atomicOr(&nxt->wet, 1);
            FpClock *old = &S.clock[(slot + 2) & 3];
            old->smax_bits = 0u;
            old->wet = 0;
        }
    }
}

// U^0 wave-speed max and wet flag into clock slot `slot` (after a state change).
__global__ void init_clock_kernel(const __grid_constant__ FpSim S, int par, int slot) {
    float smax = 0.0f;
    int wet = 0;
    const long long n = (long long)S.nx * S.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % S.nx), j = (int)(c / S.nx);
        const size_t o = fp_pidx(S, i, j);
        const float h = S.h[par][o];
        if (h > FP_H_EPS_F) smax = fmaxf(smax, fp_wave_speed(S.g, h, S.hu[par][o], S.hv[par][o]));
        if (h >= FP_H_DRY_F) wet = 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        wet |= __shfl_xor_sync(0xffffffffu, wet, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (smax > 0.0f) atomicMax(&S.clock[slot].smax_bits, __float_as_uint(smax));
        if (wet) atomicOr(&S.clock[slot].wet, 1);
    }
}

// Water volume sum h dx^2 in FP64: per-CTA partials, then the last CTA adds
// them (and the boundary inflow volumes) in index order -- deterministic.
__global__ void mass_kernel(const __grid_constant__ FpSim S, int par) {
    __shared__ double red[8];
    __shared__ bool last;
    double acc = 0.0;
    const long long n = (long long)S.nx * S.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % S.nx), j = (int)(c / S.nx);
        acc += (double)S.h[par][fp_pidx(S, i, j)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
        S.partials[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(&S.cnt->mass_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned k = 0; k < gridDim.x; ++k) s += ((volatile double *)S.partials)[k];
        const double dx = (double)S.dx;
        S.cnt->mass = s * dx * dx;
        double q = 0.0;
        for (int k = 0; k < 2 * S.nx + 2 * S.ny; ++k) q += S.bflux[k];
        S.cnt->inflow = q;
        S.cnt->mass_done = 0u;
    }
}

}  // namespace

int fp_flood_smem_bytes(int tile_rows) {
    if (tile_rows == 8) return smem_bytes<8>();
    if (tile_rows == 32) return smem_bytes<32>();
    return smem_bytes<16>();
}

cudaError_t fp_flood_init_attributes() {
    cudaError_t e = cudaFuncSetAttribute(flood_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<8>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(flood_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<16>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(flood_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<32>());
    return e;
}

template <int TY>
static void launch_flood_t(const FpSim &S, const FpTmaSet &tm, int par, int slot, cudaStream_t st) {
    constexpr int smem = smem_bytes<TY>();
    dim3 grid((S.nx + FP_TX - 1) / FP_TX, (S.ny + TY - 1) / TY);
    flood_kernel<TY><<<grid, 16 * TY, smem, st>>>(tm, S, par, slot);
}

void fp_launch_flood(const FpSim &S, const void *tma_set, int par, int slot, int tile_rows, cudaStream_t st) {
    const FpTmaSet &tm = *static_cast<const FpTmaSet *>(tma_set);
    if (tile_rows == 8) launch_flood_t<8>(S, tm, par, slot, st);
    else if (tile_rows == 32) launch_flood_t<32>(S, tm, par, slot, st);
    else launch_flood_t<16>(S, tm, par, slot, st);
}

void fp_launch_init_clock(const FpSim &S, int par, int slot, cudaStream_t st) {
    const long long n = (long long)S.nx * S.ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 148 * 8) blocks = 148 * 8;
    if (blocks < 1) blocks = 1;
    init_clock_kernel<<<blocks, 256, 0, st>>>(S, par, slot);
}

void fp_launch_mass(const FpSim &S, int par, cudaStream_t st) {
    const long long n = (long long)S.nx * S.ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 148 * 4) blocks = 148 * 4;
    if (blocks < 1) blocks = 1;
    mass_kernel<<<blocks, 256, 0, st>>>(S, par);
}
