// surrogate.cu -- the learned flood surrogate (build-added; the paper has no
// surrogate): a 5-layer 3x3 convolutional net 8 -> 32 -> 32 -> 32 -> 32 -> 3
// (ReLU between layers) mapping (h, hu, hv, z) around a cell to the change of
// (h, hu, hv) over 8 fixed time steps; the 8 input channels are the four inputs
// rounded to BF16 and the rounded remainders.
//
// Forward (inference and training): each layer is an implicit GEMM on the
// 5th-generation tensor cores -- tcgen05.mma, kind::f16 with BF16 operands in
// shared memory and an FP32 accumulator in tensor memory (TMEM):
//   M = 128 output pixels of one row; per input row and horizontal tap one
//   MMA with N = 3 x 32 (3 x 16 for the last layer, 3 channels used): the
//   three vertical taps' weights side by side, accumulating into three output
//   rows at once; K = input channels in steps of 16.
// A CTA is persistent over output row segments and warp-specialised (TMA
// producer, MMA issuer, eight epilogue warps).  It keeps the layer's weights
// in shared memory in the canonical no-swizzle K-major layout (core matrices
// of 8 rows x 16 bytes; k-cores LBO apart, 8-row groups SBO apart) and stages
// input rows as [k-core][pixel][8 channels]: the three horizontal taps of an
// input row are then the same operand shifted by 16 bytes.  The epilogue warps
// read their TMEM lanes with tcgen05.ld for the bias / ReLU / BF16 epilogue.
// Every wait is bounded; TMEM is freed on every exit path.
//
// Training: the backward pass (data and weight gradients of every
// layer, FP32 on the CUDA cores, deterministic reductions), the loss and Adam
// with FP32 master weights.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "floodped.h"
#include "fp_common.cuh"

namespace {

constexpr int kLayers = 5;
constexpr int kWidth = 32;
constexpr int kCin0 = 16;   // first layer: 8 real input channels padded to 16
constexpr int kCout4 = 16;  // last layer: 3 real output channels padded to 16
constexpr int kSeg = 128;   // output pixels per MMA (M)
constexpr float kOutScale = FP_SUR_OUT_SCALE;  // the net predicts delta U / 2^-10
// The first layer sees each of (h, hu, hv, z) as two BF16 numbers, the rounded
// value and the rounded remainder (channels 0-3 and 4-7): its FP32 accumulation
// then resolves free-surface differences far below one BF16 step of z.
constexpr int kCh[kLayers + 1] = {8, kWidth, kWidth, kWidth, kWidth, 3};

__device__ __forceinline__ unsigned sm_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: no swizzle, K-major canonical layout
__device__ __forceinline__ unsigned long long umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;  // descriptor version
    return d;         // base offset 0, relative LBO, layout type 0 (no swizzle)
}

// instruction descriptor, kind::f16: F32 accumulate, BF16 A and B, both K-major
__host__ __device__ constexpr unsigned umma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

constexpr int kStripRows = 32;  // output rows per work item (one column segment of one image)
constexpr int kRing = 4;        // staged input rows in the ring
constexpr int kEpiWarps = 8;    // epilogue warps: TMEM lane quarter w % 4, column half w / 4
constexpr int kConvWarps = kEpiWarps + 2;  // + one TMA producer warp + one MMA issuer warp
constexpr int kBlk = 4;         // TMEM accumulator blocks (COUT columns each), one per output row in flight

template <int CIN, int COUT>
struct ConvGeom {
    static constexpr int KC = CIN / 16;            // K chunks of 16 channels
    static constexpr int NKC = CIN / 8;            // 16-byte k-cores per pixel
    static constexpr int NPIX = kSeg + 32;         // staged input pixels per row (5 blocks of 32; 130 used)
    static constexpr int ROWB = NKC * NPIX * 16;   // bytes of one staged row (one TMA box)
    static constexpr int SLOT = (ROWB + 127) / 128 * 128;  // ring slot stride (TMA destinations 128-B aligned)
    static constexpr int WBLK = 2 * 3 * COUT * 16;  // bytes per (horizontal tap, chunk) weight block
    static constexpr int WB = 3 * KC * WBLK;        // weight bytes (a multiple of 128)
    static constexpr int TCOLS = kBlk * COUT;       // TMEM columns (a power of two, >= 32)
    static_assert((TCOLS & (TCOLS - 1)) == 0 && TCOLS >= 32 && TCOLS <= 512, "TMEM allocation");
    // guard region after the operands (a descriptor-field error reads garbage inside the allocation)
    static constexpr int SMEM = ((WB + kRing * SLOT + 2048) + 1023) / 1024 * 1024;
};

__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
    unsigned ok = 0;
    for (int it = 0; it < (1 << 22) && !ok; ++it) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
    }
    return ok != 0;
}

// the same, giving up early once another role has flagged an abort
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned bar, unsigned parity, const volatile int *abort_flag) {
    unsigned ok = 0;
    for (int it = 0; it < (1 << 22) && !ok; ++it) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (!ok && (it & 255) == 255 && *abort_flag) break;
    }
    return ok != 0;
}

__device__ __forceinline__ void mbar_init_n(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

template <int N>
__device__ __forceinline__ void tmem_load(unsigned taddr, unsigned (&r)[N]);

template <>
__device__ __forceinline__ void tmem_load<8>(unsigned taddr, unsigned (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <>
__device__ __forceinline__ void tmem_load<16>(unsigned taddr, unsigned (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// D (TMEM) += A (shared memory) x B (shared memory), kind::f16
__device__ __forceinline__ void mma_acc(unsigned dcol, unsigned long long ad, unsigned long long bd, unsigned idesc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
        "l"(ad), "l"(bd), "r"(idesc), "r"(1u)
        : "memory");
}

// clear N columns of this warp's 32 TMEM lanes (completion: tcgen05.wait::st)
template <int N>
__device__ __forceinline__ void tmem_zero(unsigned taddr);

template <>
__device__ __forceinline__ void tmem_zero<8>(unsigned taddr) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr), "r"(0u)
                 : "memory");
}

template <>
__device__ __forceinline__ void tmem_zero<16>(unsigned taddr) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1};" ::"r"(taddr),
        "r"(0u)
        : "memory");
}

// One 3x3 valid convolution of B images (BF16, CIN channels in groups of 8) with the
// packed weights (3 horizontal taps x CIN/16 chunks of [2 k-cores][3 COUT
// rows][8] BF16, the rows ordered vertical tap 2, 1, 0).  Hidden layers: bias
// + ReLU, BF16 output with COUT channels.  Last layer (LAST): bias, FP32
// output with 3 channels, times kOutScale.
//
// Work item: one column segment (128 output pixels) of up to kStripRows
// consecutive output rows of one image.  Input row i feeds output rows i - 2,
// i - 1, i through its vertical taps 2, 1, 0: one MMA per (horizontal tap,
// chunk) with N = 3 COUT covers all three, writing three consecutive COUT-column
// accumulator blocks (the block of output row g is g mod kBlk; a window that
// runs past the last block is split in two MMAs).  Blocks are zero when a row
// starts: the epilogue clears a block after reading it, so every MMA
// accumulates.  Warp-specialised pipeline, hand-offs by mbarriers only (every
// wait bounded):
//   producer warp (one thread): one TMA per input row into a ring of kRing slots --
//     the 5-D tensor map (8 channels, pixel, k-core, row, image) lands the row
//     as [k-core][pixel][8 channels], the MMA's canonical K-major layout;
//     a slot is refilled once the MMAs that read it completed (free[slot]);
//   issuer warp (one thread): for input row i, once it landed (full[]) and the
//     block of the output row it starts is clear (empty[]), issues its MMAs
//     (3 horizontal taps x chunks of 16 channels, the taps being the same
//     operand shifted by one pixel; descriptors precomputed), commits them to
//     free[] of the row and, once row i completes output row i - 2, to
//     acc_full[] of that row's block;
//   epilogue warps (8): wait acc_full, read their TMEM lane quarter and
//     column half (tcgen05.ld), clear it (tcgen05.st), free the block
//     (empty[]), then bias / ReLU / BF16 and the stores.
template <int CIN, int COUT, bool LAST>
__global__ void __launch_bounds__(kConvWarps * 32) conv3x3_tc_kernel(const __grid_constant__ CUtensorMap tmap, int B,
                                                                     int H, int W,
                                                                     const __nv_bfloat16 *__restrict__ wpack,
                                                                     const float *__restrict__ bias,
                                                                     void *__restrict__ y, unsigned *err) {
    using G = ConvGeom<CIN, COUT>;
    constexpr int HALF = COUT / 2;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *s_w = sm;
    unsigned char *s_x = sm + G::WB;
    __shared__ __align__(8) unsigned long long bar_full[kRing], bar_free[kRing], bar_accf[kBlk], bar_acce[kBlk];
    __shared__ unsigned s_taddr;
    __shared__ volatile int s_abort;
    __shared__ float s_bias[COUT];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Ho = H - 2, Wo = W - 2, Pout = fp_sur_pitch(Wo);
    const int segs = (Wo + kSeg - 1) / kSeg;
    const int chunks = (Ho + kStripRows - 1) / kStripRows;
    const int items = B * segs * chunks;
    if (tid < COUT) s_bias[tid] = bias[tid];

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_addr(&s_taddr)),
                     "n"(G::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int k = 0; k < kRing; ++k) {
            mbar_init_n(sm_addr(&bar_full[k]), 1);
            mbar_init_n(sm_addr(&bar_free[k]), 1);
        }
        for (int a = 0; a < kBlk; ++a) {
            mbar_init_n(sm_addr(&bar_accf[a]), 1);
            mbar_init_n(sm_addr(&bar_acce[a]), kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    for (int i = tid; i < G::WB / 16; i += kConvWarps * 32)
        reinterpret_cast<uint4 *>(s_w)[i] = reinterpret_cast<const uint4 *>(wpack)[i];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned taddr = s_taddr;
    const unsigned xs = sm_addr(s_x), ws = sm_addr(s_w);
    // the epilogue warps clear every accumulator block before the first MMA
    if (warp < kEpiWarps) {
        const unsigned lq = (unsigned)(32 * (warp & 3)) << 16;
        for (int a = 0; a < kBlk; ++a) tmem_zero<HALF>(taddr + lq + a * COUT + (warp >> 2) * HALF);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    auto fail = [&]() {
        atomicOr(err, FP_ERR_TIMEOUT);
        s_abort = 1;
    };

    if (warp == kEpiWarps) {
        // ---- TMA producer: one copy per input row segment; the 5-D tensor
        // map lands it as [k-core][pixel][8 channels]
        if (lane == 0) {
            unsigned q = 0;  // input rows issued by this CTA
            for (int item = blockIdx.x; item < items && !s_abort; item += gridDim.x) {
                const int img = item / (segs * chunks), rem = item % (segs * chunks);
                const int ox0 = (rem / chunks) * kSeg, oy0 = (rem % chunks) * kStripRows;
                const int nrow = min(kStripRows, Ho - oy0);
                bool ok = true;
                for (int i = 0; i < nrow + 2; ++i, ++q) {
                    const unsigned slot = q % kRing, use = q / kRing;
                    if (use > 0 && !mbar_wait_or_abort(sm_addr(&bar_free[slot]), (use - 1) & 1u, &s_abort)) {
                        fail();
                        ok = false;
                        break;
                    }
                    const unsigned fb = sm_addr(&bar_full[slot]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(G::ROWB)
                                 : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                        "%3, %4, %5, %6}], [%7];" ::"r"(xs + slot * G::SLOT),
                        "l"(reinterpret_cast<unsigned long long>(&tmap)), "r"(0), "r"(ox0 / 32), "r"(0), "r"(oy0 + i),
                        "r"(img), "r"(fb)
                        : "memory");
                }
                if (!ok) break;
            }
            // no copy of this CTA may still be landing when it exits
            const unsigned n = q < (unsigned)kRing ? q : (unsigned)kRing;
            for (unsigned k = 0; k < n; ++k) {
                const unsigned qq = q - 1 - k;
                mbar_wait_bounded(sm_addr(&bar_full[qq % kRing]), (qq / kRing) & 1u);
            }
        }
    } else if (warp == kEpiWarps + 1) {
        // ---- MMA issuer.  A descriptor's start-address field is its low bits,
        // so the descriptor of base + d is the base descriptor + d / 16 (every
        // shared address here is below 256 KB): the weight descriptors are
        // fixed, a vertical-tap range is one add (16 bytes per weight row), and
        // an input descriptor is one add.
        if (lane == 0) {
            unsigned long long bdesc[3 * G::KC];
#pragma unroll
            for (int k = 0; k < 3 * G::KC; ++k) bdesc[k] = umma_desc(ws + k * G::WBLK, 3 * COUT * 16, 128);
            const unsigned long long adesc0 = umma_desc(xs, G::NPIX * 16, 128);
            // instruction descriptors for N = COUT, 2 COUT, 3 COUT
            const unsigned id1 = umma_idesc(kSeg, COUT), id2 = umma_idesc(kSeg, 2 * COUT),
                           id3 = umma_idesc(kSeg, 3 * COUT);
            unsigned q = 0, g0 = 0;  // input rows consumed, output rows of earlier items
            bool ok = true;
            for (int item = blockIdx.x; item < items && ok && !s_abort; item += gridDim.x) {
                const int rem = item % (segs * chunks);
                const int oy0 = (rem % chunks) * kStripRows;
                const int nrow = min(kStripRows, Ho - oy0);
                for (int i = 0; i < nrow + 2 && ok; ++i, ++q) {
                    // output rows i - kyhi .. i - kylo of the item take this row
                    const int kylo = max(0, i - (nrow - 1)), kyhi = min(2, i);
                    ok = mbar_wait_or_abort(sm_addr(&bar_full[q % kRing]), (q / kRing) & 1u, &s_abort);
                    const unsigned gnew = g0 + (unsigned)i;  // the output row this input row starts
                    if (ok && kylo == 0 && gnew >= (unsigned)kBlk)
                        ok = mbar_wait_or_abort(sm_addr(&bar_acce[gnew % kBlk]), (gnew / kBlk - 1) & 1u, &s_abort);
                    if (!ok) {
                        fail();
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int nb = kyhi - kylo + 1;
                    const unsigned b0 = (g0 + (unsigned)(i - kyhi)) % kBlk;
                    const int n1 = min(nb, kBlk - (int)b0), n2 = nb - n1;
                    const unsigned slot_off = (q % kRing) * (G::SLOT / 16);
                    const unsigned brow = (unsigned)((2 - kyhi) * COUT);
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
                        for (int c = 0; c < G::KC; ++c) {
                            const unsigned long long ad =
                                adesc0 + slot_off + (unsigned)((2 * c * G::NPIX * 16 + kx * 16) / 16);
                            const unsigned long long bd = bdesc[kx * G::KC + c] + brow;
                            mma_acc(taddr + b0 * COUT, ad, bd, n1 == 1 ? id1 : n1 == 2 ? id2 : id3);
                            if (n2 > 0) mma_acc(taddr, ad, bd + (unsigned)(n1 * COUT), n2 == 1 ? id1 : id2);
                        }
                    }
                    // the input row is read by no later MMA
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     sm_addr(&bar_free[q % kRing]))
                                 : "memory");
                    if (kyhi == 2)  // output row i - 2 is complete
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                sm_addr(&bar_accf[(g0 + (unsigned)(i - 2)) % kBlk]))
                            : "memory");
                }
                g0 += (unsigned)nrow;
            }
        }
    } else {
        // ---- epilogue: warp w owns TMEM lanes (output pixels) 32 (w % 4) ..
        // 32 (w % 4) + 31 and accumulator columns HALF (w / 4) .. + HALF - 1
        // of a block (the last layer: warps 0-3 hold its three channels)
        const int quarter = warp & 3, half = warp >> 2;
        unsigned g = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
            const int img = item / (segs * chunks), rem = item % (segs * chunks);
            const int ox0 = (rem / chunks) * kSeg, oy0 = (rem % chunks) * kStripRows;
            const int nrow = min(kStripRows, Ho - oy0);
            for (int r = 0; r < nrow; ++r, ++g) {
                const unsigned a = g % kBlk;
                ok = mbar_wait_or_abort(sm_addr(&bar_accf[a]), (g / kBlk) & 1u, &s_abort);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    if (lane == 0) fail();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned v[HALF];
                const bool active = !LAST || half == 0;
                const unsigned ta = taddr + ((unsigned)(32 * quarter) << 16) + a * COUT + (unsigned)(half * HALF);
                if (active) tmem_load<HALF>(ta, v);
                tmem_zero<HALF>(ta);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(&bar_acce[a])) : "memory");
                const int oy = oy0 + r, ox = ox0 + 32 * quarter + lane;
                if (active && ox < Wo) {
                    const size_t pix = ((size_t)img * Ho + oy) * Wo + ox;
                    if constexpr (LAST) {
                        float *yo = static_cast<float *>(y) + pix * 3;
#pragma unroll
                        for (int co = 0; co < 3; ++co) yo[co] = (__uint_as_float(v[co]) + s_bias[co]) * kOutScale;
                    } else {
                        // channel groups of 8: group half * HALF / 8 + qd of the pixel
                        __nv_bfloat16 *yo = static_cast<__nv_bfloat16 *>(y) +
                                            ((((size_t)img * Ho + oy) * (COUT / 8) + half * (HALF / 8)) * Pout + ox) * 8;
                        const float *bb = s_bias + half * HALF;
#pragma unroll
                        for (int qd = 0; qd < HALF / 8; ++qd) {
                            __nv_bfloat162 o[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float a0 = fmaxf(__uint_as_float(v[8 * qd + 2 * e]) + bb[8 * qd + 2 * e], 0.0f);
                                const float a1 =
                                    fmaxf(__uint_as_float(v[8 * qd + 2 * e + 1]) + bb[8 * qd + 2 * e + 1], 0.0f);
                                o[e] = __floats2bfloat162_rn(a0, a1);
                            }
                            *reinterpret_cast<uint4 *>(yo + (size_t)qd * Pout * 8) = *reinterpret_cast<const uint4 *>(o);
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(G::TCOLS));
}

// FP32 (h, hu, hv, z) images [B][H][W] -> the net's 16-channel BF16 input
// (channel groups of 8: the rounded values and remainders, then zeros)
__global__ void pack_input_kernel(const float *__restrict__ x4, int B, int H, int W, __nv_bfloat16 *__restrict__ out) {
    const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (p >= (size_t)B * H * W) return;
    const float4 v = reinterpret_cast<const float4 *>(x4)[p];
    const size_t row = p / W;  // b H + y
    const int x = (int)(p % W);
    const int P = fp_sur_pitch(W);
    __nv_bfloat16 *g0 = out + ((row * 2) * P + x) * 8;
    fp_sur_pack_pixel(v.x, v.y, v.z, v.w, g0, g0 + (size_t)P * 8);
}


// ---- training: FP32 backward on the CUDA cores --------------------------------

// g = d loss / d (last layer pre-activation): loss = mean (s z - t)^2 over
// B x Ho x Wo x 3 with s = kOutScale, so dz = 2 s (s z - t) / n = 2 s (y - t) / n with y the
// scaled output.  Per-block FP64 partial losses, summed in block order later.
__global__ void loss_grad_kernel(const float *__restrict__ y, const float *__restrict__ t, size_t n,
                                 float *__restrict__ g, double *__restrict__ partial) {
    __shared__ double red[256 / 32];
    double acc = 0.0;
    const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (k < n) {
        const float d = y[k] - t[k];
        acc = (double)d * (double)d;
        g[k] = 2.0f * kOutScale * d / (float)n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s2 += red[w];
        partial[blockIdx.x] = s2;
    }
}

__global__ void sum_partials_kernel(const double *__restrict__ partial, int n, double scale, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s2 = 0.0;
        for (int k = 0; k < n; ++k) s2 += partial[k];
        *out = s2 * scale;
    }
}

// activation (image b, row y, column x, channel c) of an H x W x C image, by channel groups of 8
__device__ __forceinline__ float act_at(const __nv_bfloat16 *a, int b, int y, int x, int c, int H, int W, int C) {
    return __bfloat162float(a[((((size_t)b * H + y) * (C / 8) + c / 8) * fp_sur_pitch(W) + x) * 8 + (c & 7)]);
}

// dW[t][ci][co] += sum_p X[p + off_t][ci] dY[p][co] and db[co] += sum_p dY[p][co],
// one CTA per (tap, input channel); threads stride over output pixels; fixed-order
// tree reduction.  X: BF16 H x W images with CX >= CIN channels (groups of 8).
template <int COUT>
__global__ void __launch_bounds__(256) conv_bwd_weight_kernel(const __nv_bfloat16 *__restrict__ X, int CX, int CIN,
                                                              const float *__restrict__ dY, int B, int H, int W,
                                                              float *__restrict__ dw, float *__restrict__ db) {
    const int t = blockIdx.x / CIN, ci = blockIdx.x % CIN;
    const int ky = t / 3, kx = t % 3;
    const int Ho = H - 2, Wo = W - 2;
    const size_t npix = (size_t)B * Ho * Wo;
    float acc[COUT], accb[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) { acc[c] = 0.0f; accb[c] = 0.0f; }
    const bool do_b = blockIdx.x == 0;
    for (size_t p = threadIdx.x; p < npix; p += blockDim.x) {
        const int b = (int)(p / ((size_t)Ho * Wo));
        const int r = (int)(p % ((size_t)Ho * Wo));
        const int oy = r / Wo, ox = r % Wo;
        const float xv = act_at(X, b, oy + ky, ox + kx, ci, H, W, CX);
        const float *g = dY + p * COUT;
#pragma unroll
        for (int c = 0; c < COUT; ++c) {
            acc[c] = fmaf(xv, g[c], acc[c]);
            if (do_b) accb[c] += g[c];
        }
    }
    __shared__ float red[256][COUT + 1];
#pragma unroll
    for (int c = 0; c < COUT; ++c) red[threadIdx.x][c] = acc[c];
    __syncthreads();
    for (int sz = 128; sz > 0; sz >>= 1) {
        if ((int)threadIdx.x < sz)
            for (int c = 0; c < COUT; ++c) red[threadIdx.x][c] += red[threadIdx.x + sz][c];
        __syncthreads();
    }
    if ((int)threadIdx.x < COUT) dw[((size_t)t * CIN + ci) * COUT + threadIdx.x] = red[0][threadIdx.x];
    if (do_b) {
        __syncthreads();
#pragma unroll
        for (int c = 0; c < COUT; ++c) red[threadIdx.x][c] = accb[c];
        __syncthreads();
        for (int sz = 128; sz > 0; sz >>= 1) {
            if ((int)threadIdx.x < sz)
                for (int c = 0; c < COUT; ++c) red[threadIdx.x][c] += red[threadIdx.x + sz][c];
            __syncthreads();
        }
        if ((int)threadIdx.x < COUT) db[threadIdx.x] = red[0][threadIdx.x];
    }
}

// dX[q][ci] = sum_{t, co} dY[q - off_t][co] W[t][ci][co] over valid output
// positions, masked by the ReLU of X (the previous layer's output): the
// gradient of the previous layer's pre-activation.  W is taken rounded to BF16,
// the weights the forward multiplied by.  One thread per (q, ci).
template <int CIN, int COUT>
__global__ void conv_bwd_data_kernel(const float *__restrict__ dY, const float *__restrict__ w,
                                     const __nv_bfloat16 *__restrict__ X, int B, int H, int W,
                                     float *__restrict__ dXm) {
    const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t n = (size_t)B * H * W * CIN;
    if (k >= n) return;
    const int ci = (int)(k % CIN);
    const size_t q = k / CIN;
    const int b = (int)(q / ((size_t)H * W));
    const int r = (int)(q % ((size_t)H * W));
    const int iy = r / W, ix = r % W;
    const int Ho = H - 2, Wo = W - 2;
    float acc = 0.0f;
    if (act_at(X, b, iy, ix, ci, H, W, CIN) > 0.0f) {
        for (int ky = 0; ky < 3; ++ky) {
            const int oy = iy - ky;
            if (oy < 0 || oy >= Ho) continue;
            for (int kx = 0; kx < 3; ++kx) {
                const int ox = ix - kx;
                if (ox < 0 || ox >= Wo) continue;
                const float *g = dY + (((size_t)b * Ho + oy) * Wo + ox) * COUT;
                const float *wr = w + ((size_t)(ky * 3 + kx) * CIN + ci) * COUT;
#pragma unroll 8
                for (int co = 0; co < COUT; ++co)
                    acc = fmaf(g[co], __bfloat162float(__float2bfloat16(wr[co])), acc);
            }
        }
    }
    dXm[k] = acc;
}

// Adam on the FP32 master parameters
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + eps);
}

// FP32 master (one layer) -> packed BF16 operand blocks and padded bias: per
// (horizontal tap kx, chunk c) a block [2 k-cores][3 co_pad rows][8], row
// (2 - ky) co_pad + n holding output channel n of vertical tap ky
__global__ void pack_layer_kernel(const float *__restrict__ w, const float *__restrict__ b, int ci_real, int co_real,
                                  int ci_pad, int co_pad, __nv_bfloat16 *__restrict__ pk, float *__restrict__ bias) {
    const int kc = ci_pad / 16, rows = 3 * co_pad;
    const int total = 3 * kc * 2 * rows * 8;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < co_pad) bias[k] = k < co_real ? b[k] : 0.0f;
    if (k >= total) return;
    const int e = k % 8, n3 = (k / 8) % rows, j = (k / (8 * rows)) % 2;
    const int c = (k / (16 * rows)) % kc, kx = k / (16 * rows * kc);
    const int ky = 2 - n3 / co_pad, n = n3 % co_pad, t = 3 * ky + kx;
    const int ci = 16 * c + 8 * j + e;
    float v = 0.0f;
    if (ci < ci_real && n < co_real) v = w[((size_t)t * ci_real + ci) * co_real + n];
    pk[k] = __float2bfloat16(v);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct fp_surrogate {
    size_t n_params = 0;
    std::vector<size_t> w_off, b_off;             // offsets of each layer's w and b
    float *d_master = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr;
    __nv_bfloat16 *d_wpack[kLayers] = {};         // packed BF16 weights per layer
    float *d_bias[kLayers] = {};                  // padded FP32 biases per layer
    unsigned *d_err = nullptr;
    double *d_loss = nullptr, *d_partial = nullptr;
    long long adam_t = 0;
    // cached scratch: activations (BF16), output and gradients (FP32)
    size_t cap_pix = 0, cap_partial = 0;
    __nv_bfloat16 *d_a[kLayers] = {};             // inputs of every layer (a[0] packed input)
    float *d_out = nullptr, *d_g0 = nullptr, *d_g1 = nullptr;
    std::vector<void *> allocs;
    int sms = 148;
};

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 5-D view of a BF16 activation (H x W images, CIN channels in groups of 8,
// row pitch P): (256 elements = 32 pixels x 8 channels, 32-pixel block, group,
// row, image); a box of (256, 5, CIN / 8, 1, 1) is one staged input row
// segment of 160 pixels in the [k-core][pixel][8 channels] layout, read as
// 512-byte runs.
template <int CIN>
cudaError_t encode_act_map(CUtensorMap *m, const __nv_bfloat16 *x, int B, int H, int W) {
    auto enc = tmap_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t P = (cuuint64_t)fp_sur_pitch(W);
    const cuuint64_t dims[5] = {256, P / 32, (cuuint64_t)(CIN / 8), (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[4] = {512, P * 16, P * CIN * 2, (cuuint64_t)H * P * CIN * 2};
    const cuuint32_t box[5] = {256, (cuuint32_t)((kSeg + 32) / 32), (cuuint32_t)(CIN / 8), 1, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(x), dims, strides,
                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CIN, int COUT, bool LAST>
cudaError_t launch_conv(const fp_surrogate *s, int layer, const __nv_bfloat16 *x, int B, int H, int W, void *y,
                        cudaStream_t st) {
    using G = ConvGeom<CIN, COUT>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv3x3_tc_kernel<CIN, COUT, LAST>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap m;
    cudaError_t e = encode_act_map<CIN>(&m, x, B, H, W);
    if (e != cudaSuccess) return e;
    const long long items =
        (long long)B * (((W - 2) + kSeg - 1) / kSeg) * (((H - 2) + kStripRows - 1) / kStripRows);
    // resident CTAs per SM: three (shared memory allows three), at most 512 / TCOLS (TMEM)
    const int per_sm = std::min(3, 512 / G::TCOLS);
    int grid = (int)std::min<long long>(items, (long long)s->sms * per_sm);
    if (grid < 1) grid = 1;
    conv3x3_tc_kernel<CIN, COUT, LAST><<<grid, kConvWarps * 32, G::SMEM, st>>>(m, B, H, W, s->d_wpack[layer],
                                                                              s->d_bias[layer], y, s->d_err);
    return cudaGetLastError();
}

size_t param_count() {
    size_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += (size_t)9 * kCh[l] * kCh[l + 1] + kCh[l + 1];
    return n;
}

// FP32 master -> packed BF16 operand blocks and padded biases (on the device)
cudaError_t repack(fp_surrogate *s, cudaStream_t st) {
    for (int l = 0; l < kLayers; ++l) {
        const int ci_pad = l == 0 ? kCin0 : kWidth, co_pad = l == kLayers - 1 ? kCout4 : kWidth;
        const int total = 9 * (ci_pad / 16) * 2 * co_pad * 8;
        pack_layer_kernel<<<(total + 255) / 256, 256, 0, st>>>(s->d_master + s->w_off[l], s->d_master + s->b_off[l],
                                                              kCh[l], kCh[l + 1], ci_pad, co_pad, s->d_wpack[l],
                                                              s->d_bias[l]);
    }
    return cudaGetLastError();
}

// pix: images x rows x row pitch (pixels) of the largest input
bool ensure_scratch(fp_surrogate *s, size_t pix) {
    if (pix <= s->cap_pix) return true;
    for (int l = 0; l < kLayers; ++l) cudaFree(s->d_a[l]);
    cudaFree(s->d_out); cudaFree(s->d_g0); cudaFree(s->d_g1); cudaFree(s->d_partial);
    s->cap_pix = 0;
    bool ok = cudaMalloc(&s->d_a[0], pix * kCin0 * sizeof(__nv_bfloat16)) == cudaSuccess;
    for (int l = 1; l < kLayers; ++l) ok &= cudaMalloc(&s->d_a[l], pix * kWidth * sizeof(__nv_bfloat16)) == cudaSuccess;
    ok &= cudaMalloc(&s->d_out, pix * 3 * sizeof(float)) == cudaSuccess;
    ok &= cudaMalloc(&s->d_g0, pix * kWidth * sizeof(float)) == cudaSuccess;
    ok &= cudaMalloc(&s->d_g1, pix * kWidth * sizeof(float)) == cudaSuccess;
    s->cap_partial = (pix * 3 + 255) / 256 + 1;
    ok &= cudaMalloc(&s->d_partial, s->cap_partial * sizeof(double)) == cudaSuccess;
    // activation rows are padded to 32 pixels: keep the padding finite
    for (int l = 0; l < kLayers && ok; ++l)
        ok = cudaMemset(s->d_a[l], 0, pix * (l == 0 ? kCin0 : kWidth) * sizeof(__nv_bfloat16)) == cudaSuccess;
    if (ok) s->cap_pix = pix;
    return ok;
}

// the five layers from a packed BF16 input in0 [B][H][W][16]; every later
// layer's input stays in d_a; output to out
cudaError_t forward_layers(fp_surrogate *s, const __nv_bfloat16 *in0, int B, int H, int W, float *out,
                           cudaStream_t st) {
    cudaError_t e = launch_conv<kCin0, kWidth, false>(s, 0, in0, B, H, W, s->d_a[1], st);
    int h = H - 2, w = W - 2;
    for (int l = 1; l < kLayers - 1 && e == cudaSuccess; ++l) {
        e = launch_conv<kWidth, kWidth, false>(s, l, s->d_a[l], B, h, w, s->d_a[l + 1], st);
        h -= 2; w -= 2;
    }
    if (e == cudaSuccess) e = launch_conv<kWidth, kCout4, true>(s, kLayers - 1, s->d_a[kLayers - 1], B, h, w, out, st);
    return e;
}

// forward of B images x [B][H][W][4] keeping every layer's input in d_a; output to out
cudaError_t forward_keep(fp_surrogate *s, const float *x, int B, int H, int W, float *out, cudaStream_t st) {
    const size_t npix0 = (size_t)B * H * W;
    pack_input_kernel<<<(unsigned)((npix0 + 255) / 256), 256, 0, st>>>(x, B, H, W, s->d_a[0]);
    return forward_layers(s, s->d_a[0], B, H, W, out, st);
}

// loss and gradients (into d_grad, master layout) of the last forward_keep
cudaError_t backward(fp_surrogate *s, const float *target, int B, int H, int W, cudaStream_t st) {
    const int H5 = H - 2 * kLayers, W5 = W - 2 * kLayers;
    const size_t n_out = (size_t)B * H5 * W5 * 3;
    const unsigned nb = (unsigned)((n_out + 255) / 256);
    loss_grad_kernel<<<nb, 256, 0, st>>>(s->d_out, target, n_out, s->d_g0, s->d_partial);
    sum_partials_kernel<<<1, 32, 0, st>>>(s->d_partial, (int)nb, 1.0 / (double)n_out, s->d_loss);
    float *g = s->d_g0, *gprev = s->d_g1;
    for (int l = kLayers - 1; l >= 0; --l) {
        const int Hl = H - 2 * l, Wl = W - 2 * l;  // input size of layer l
        float *dw = s->d_grad + s->w_off[l], *db = s->d_grad + s->b_off[l];
        if (l == kLayers - 1) {
            conv_bwd_weight_kernel<3><<<9 * kWidth, 256, 0, st>>>(s->d_a[l], kWidth, kWidth, g, B, Hl, Wl, dw, db);
            const size_t n = (size_t)B * Hl * Wl * kWidth;
            conv_bwd_data_kernel<kWidth, 3><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                g, s->d_master + s->w_off[l], s->d_a[l], B, Hl, Wl, gprev);
        } else if (l > 0) {
            conv_bwd_weight_kernel<kWidth><<<9 * kWidth, 256, 0, st>>>(s->d_a[l], kWidth, kWidth, g, B, Hl, Wl, dw, db);
            const size_t n = (size_t)B * Hl * Wl * kWidth;
            conv_bwd_data_kernel<kWidth, kWidth><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                g, s->d_master + s->w_off[l], s->d_a[l], B, Hl, Wl, gprev);
        } else {
            conv_bwd_weight_kernel<kWidth><<<9 * kCh[0], 256, 0, st>>>(s->d_a[0], kCin0, kCh[0], g, B, Hl, Wl, dw, db);
        }
        std::swap(g, gprev);
    }
    return cudaGetLastError();
}

int check_err(fp_surrogate *s, cudaError_t e, const char *what) {
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        fp_note_error((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
        return FP_ECUDA;
    }
    unsigned herr = 0;
    cudaMemcpy(&herr, s->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (herr & FP_ERR_TIMEOUT) {
        fp_note_error((std::string(what) + ": tensor-core completion wait timed out").c_str());
        return FP_ETIMEOUT;
    }
    return FP_OK;
}

}  // namespace

cudaError_t fp_sur_forward_packed(fp_surrogate *s, const void *x16, int B, int H, int W, float *y, cudaStream_t st) {
    if (!ensure_scratch(s, (size_t)B * H * fp_sur_pitch(W))) return cudaErrorMemoryAllocation;
    return forward_layers(s, static_cast<const __nv_bfloat16 *>(x16), B, H, W, y, st);
}

unsigned fp_sur_error_bits(fp_surrogate *s) {
    unsigned herr = 0;
    cudaMemcpy(&herr, s->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    return herr;
}

extern "C" {

int fp_surrogate_num_params(void) { return (int)param_count(); }

int fp_surrogate_create(uint64_t seed, fp_surrogate **out) {
    if (!out) return FP_EINVAL;
    *out = nullptr;
    fp_surrogate *s = new fp_surrogate();
    size_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        s->w_off.push_back(o);
        o += (size_t)9 * kCh[l] * kCh[l + 1];
        s->b_off.push_back(o);
        o += kCh[l + 1];
    }
    s->n_params = o;
    std::vector<float> init(o, 0.0f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < kLayers; ++l) {
        std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / (9.0f * kCh[l])));
        const float scale = l == kLayers - 1 ? 0.1f : 1.0f;
        for (size_t k = 0; k < (size_t)9 * kCh[l] * kCh[l + 1]; ++k) init[s->w_off[l] + k] = scale * nd(rng);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, bytes);
        s->allocs.push_back(p);
        return p;
    };
    bool ok = true;
    ok &= (s->d_master = static_cast<float *>(alloc(o * sizeof(float)))) != nullptr;
    ok &= (s->d_m = static_cast<float *>(alloc(o * sizeof(float)))) != nullptr;
    ok &= (s->d_v = static_cast<float *>(alloc(o * sizeof(float)))) != nullptr;
    ok &= (s->d_grad = static_cast<float *>(alloc(o * sizeof(float)))) != nullptr;
    for (int l = 0; l < kLayers; ++l) {
        const int ci_pad = l == 0 ? kCin0 : kWidth, co_pad = l == kLayers - 1 ? kCout4 : kWidth;
        ok &= (s->d_wpack[l] = static_cast<__nv_bfloat16 *>(alloc((size_t)9 * ci_pad * co_pad * 2))) != nullptr;
        ok &= (s->d_bias[l] = static_cast<float *>(alloc((size_t)co_pad * sizeof(float)))) != nullptr;
    }
    ok &= (s->d_err = static_cast<unsigned *>(alloc(sizeof(unsigned)))) != nullptr;
    ok &= (s->d_loss = static_cast<double *>(alloc(sizeof(double)))) != nullptr;
    if (ok) ok = cudaMemcpy(s->d_master, init.data(), o * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok) ok = repack(s, 0) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        for (void *p : s->allocs) cudaFree(p);
        delete s;
        fp_note_error("fp_surrogate_create: device allocation or upload failed");
        return FP_ENOMEM;
    }
    *out = s;
    return FP_OK;
}

int fp_surrogate_destroy(fp_surrogate *s) {
    if (!s) return FP_EINVAL;
    cudaDeviceSynchronize();
    for (int l = 0; l < kLayers; ++l) cudaFree(s->d_a[l]);
    cudaFree(s->d_out); cudaFree(s->d_g0); cudaFree(s->d_g1); cudaFree(s->d_partial);
    for (void *p : s->allocs) cudaFree(p);
    delete s;
    return FP_OK;
}

int fp_surrogate_get_params(fp_surrogate *s, float *dst, size_t n) {
    if (!s || !dst || n < s->n_params) return FP_EINVAL;
    return cudaMemcpy(dst, s->d_master, s->n_params * sizeof(float), cudaMemcpyDefault) == cudaSuccess ? FP_OK
                                                                                                         : FP_ECUDA;
}

int fp_surrogate_set_params(fp_surrogate *s, const float *src, size_t n) {
    if (!s || !src || n < s->n_params) return FP_EINVAL;
    cudaError_t e = cudaMemcpy(s->d_master, src, s->n_params * sizeof(float), cudaMemcpyDefault);
    if (e == cudaSuccess) e = repack(s, 0);
    return check_err(s, e, "fp_surrogate_set_params");
}

int fp_surrogate_forward(fp_surrogate *s, const float *x, int32_t B, int32_t H, int32_t W, float *y) {
    if (!s || !x || !y || B < 1 || H < 11 || W < 11) return FP_EINVAL;
    if (!ensure_scratch(s, (size_t)B * H * fp_sur_pitch(W))) {
        fp_note_error("fp_surrogate_forward: allocation failed");
        return FP_ENOMEM;
    }
    return check_err(s, forward_keep(s, x, B, H, W, y, 0), "fp_surrogate_forward");
}

int fp_surrogate_gradients(fp_surrogate *s, const float *x, const float *target, int32_t B, int32_t H, int32_t W,
                           float *grads, double *loss) {
    if (!s || !x || !target || B < 1 || H < 11 || W < 11) return FP_EINVAL;
    if (!ensure_scratch(s, (size_t)B * H * fp_sur_pitch(W))) {
        fp_note_error("fp_surrogate_gradients: allocation failed");
        return FP_ENOMEM;
    }
    cudaError_t e = forward_keep(s, x, B, H, W, s->d_out, 0);
    if (e == cudaSuccess) e = backward(s, target, B, H, W, 0);
    int rc = check_err(s, e, "fp_surrogate_gradients");
    if (rc != FP_OK) return rc;
    if (grads && cudaMemcpy(grads, s->d_grad, s->n_params * sizeof(float), cudaMemcpyDefault) != cudaSuccess)
        return FP_ECUDA;
    if (loss && cudaMemcpy(loss, s->d_loss, sizeof(double), cudaMemcpyDefault) != cudaSuccess) return FP_ECUDA;
    return FP_OK;
}

int fp_surrogate_train_step(fp_surrogate *s, const float *x, const float *target, int32_t B, int32_t H, int32_t W,
                            float lr, double *loss) {
    int rc = fp_surrogate_gradients(s, x, target, B, H, W, nullptr, loss);
    if (rc != FP_OK) return rc;
    s->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f / (1.0f - std::pow(b1, (float)s->adam_t));
    const float c2 = 1.0f / (1.0f - std::pow(b2, (float)s->adam_t));
    const int n = (int)s->n_params;
    adam_kernel<<<(n + 255) / 256, 256>>>(s->d_master, s->d_grad, s->d_m, s->d_v, n, lr, b1, b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = repack(s, 0);
    return check_err(s, e, "fp_surrogate_train_step");
}

}  // extern "C"
