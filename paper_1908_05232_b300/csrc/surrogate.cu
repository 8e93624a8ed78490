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
// Training: the loss, the backward pass on the same tensor cores and Adam with
// FP32 master weights.  A layer's output gradient is carried as two BF16
// numbers per value (the rounded value and the rounded remainder, FP32-level
// precision) in a zero-padded image:
//   data gradient   = the same implicit-GEMM convolution of the padded output
//                     gradient (both halves as input channels) with the
//                     flipped, transposed BF16 weights; its epilogue applies
//                     the previous ReLU, splits the result for the next layer
//                     and keeps the bias-gradient partial sums;
//   weight gradient = per tap sum over pixels of input x output gradient:
//                     tcgen05.mma with both operands MN-major (pixels are K)
//                     as TMA lands whole rows of them,
//                     M = 128 = the input channels of four (eight) stacked
//                     input rows, N = the split gradient channels, one TMEM
//                     accumulator per horizontal tap; per-CTA partials summed
//                     in a fixed order.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <cstring>
#include <mutex>
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

constexpr int kStripRows = 32;  // output rows per work item at most (one column segment of one image)
constexpr int kRing = 4;        // staged input rows in the ring
constexpr int kEpiWarps = 8;    // epilogue warps: TMEM lane quarter w % 4, column half w / 4
constexpr int kConvWarps = kEpiWarps + 2;  // + one TMA producer warp + one MMA issuer warp
constexpr int kBlk = 4;         // TMEM accumulator blocks (COUT columns each), one per output row in flight

// epilogues of the implicit-GEMM convolution
constexpr int kHidden = 0;   // bias + ReLU, BF16 activations
constexpr int kLast = 1;     // bias, times kOutScale, FP32 changes of (h, hu, hv)
constexpr int kBwdData = 2;  // data gradient: ReLU mask, BF16 split into a padded image, bias-gradient partials

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
    // ring slots: four, two for 64 input channels (two CTAs then fit on an SM)
    static constexpr int RING = CIN >= 64 ? 2 : kRing;
    static constexpr int SMEM = ((WB + RING * SLOT + 2048) + 1023) / 1024 * 1024;
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
// rows][8] BF16, the rows ordered vertical tap 2, 1, 0).  Hidden layers
// (kHidden): bias + ReLU, BF16 output with COUT channels.  Last layer (kLast):
// bias, FP32 output with 3 channels, times kOutScale.  Data gradient
// (kBwdData): the input is a padded, split output gradient and the weights
// are flipped and transposed; the output is masked by the ReLU of act (the
// activation the forward layer read, Ho x Wo x COUT) and written split into
// a zero-padded (Ho + 4) x (Wo + 4) image of 2 COUT channels; each lane
// quarter of each CTA leaves its bias-gradient sums in dbpart.
//
// Work item: one column segment (128 output pixels) of up to strip (<= kStripRows)
// consecutive output rows of one image.  Input row i feeds output rows i - 2,
// i - 1, i through its vertical taps 2, 1, 0: one MMA per (horizontal tap,
// chunk) with N = 3 COUT covers all three, writing three consecutive COUT-column
// accumulator blocks (the block of output row g is g mod kBlk; a window that
// runs past the last block is split in two MMAs).  Blocks are zero when a row
// starts: the epilogue clears a block after reading it, so every MMA
// accumulates.  Warp-specialised pipeline, hand-offs by mbarriers only (every
// wait bounded):
//   producer warp (one thread): one TMA per input row into a ring of G::RING slots --
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
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(kConvWarps * 32) conv3x3_tc_kernel(const __grid_constant__ CUtensorMap tmap, int B,
                                                                     int H, int W, int strip,
                                                                     const __nv_bfloat16 *__restrict__ wpack,
                                                                     const float *__restrict__ bias,
                                                                     void *__restrict__ y,
                                                                     const __nv_bfloat16 *__restrict__ act,
                                                                     float *__restrict__ dbpart, unsigned *err) {
    using G = ConvGeom<CIN, COUT>;
    constexpr bool LAST = MODE == kLast;
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
    const int chunks = (Ho + strip - 1) / strip;
    const int items = B * segs * chunks;
    if (MODE != kBwdData && tid < COUT) s_bias[tid] = bias[tid];

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_addr(&s_taddr)),
                     "n"(G::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int k = 0; k < G::RING; ++k) {
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
                const int ox0 = (rem / chunks) * kSeg, oy0 = (rem % chunks) * strip;
                const int nrow = min(strip, Ho - oy0);
                bool ok = true;
                for (int i = 0; i < nrow + 2; ++i, ++q) {
                    const unsigned slot = q % G::RING, use = q / G::RING;
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
            const unsigned n = q < (unsigned)G::RING ? q : (unsigned)G::RING;
            for (unsigned k = 0; k < n; ++k) {
                const unsigned qq = q - 1 - k;
                mbar_wait_bounded(sm_addr(&bar_full[qq % G::RING]), (qq / G::RING) & 1u);
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
                const int oy0 = (rem % chunks) * strip;
                const int nrow = min(strip, Ho - oy0);
                for (int i = 0; i < nrow + 2 && ok; ++i, ++q) {
                    // output rows i - kyhi .. i - kylo of the item take this row
                    const int kylo = max(0, i - (nrow - 1)), kyhi = min(2, i);
                    ok = mbar_wait_or_abort(sm_addr(&bar_full[q % G::RING]), (q / G::RING) & 1u, &s_abort);
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
                    const unsigned slot_off = (q % G::RING) * (G::SLOT / 16);
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
                                     sm_addr(&bar_free[q % G::RING]))
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
        float dbacc[HALF];  // data gradient: this thread's bias-gradient sums
#pragma unroll
        for (int c = 0; c < HALF; ++c) dbacc[c] = 0.0f;
        for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
            const int img = item / (segs * chunks), rem = item % (segs * chunks);
            const int ox0 = (rem / chunks) * kSeg, oy0 = (rem % chunks) * strip;
            const int nrow = min(strip, Ho - oy0);
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
                    } else if constexpr (MODE == kBwdData) {
                        // the gradient of the previous pre-activation: masked by
                        // its ReLU (the activation this layer read), split into
                        // the BF16 rounded value (groups 0-3) and remainder
                        // (groups 4-7) at (oy + 2, ox + 2) of the zero-padded image
                        const int Pa = fp_sur_pitch(Wo), Pp = fp_sur_pitch(Wo + 4);
#pragma unroll
                        for (int qd = 0; qd < HALF / 8; ++qd) {
                            const int grp = half * (HALF / 8) + qd;
                            const uint4 araw = *reinterpret_cast<const uint4 *>(
                                act + ((((size_t)img * Ho + oy) * (COUT / 8) + grp) * Pa + ox) * 8);
                            const __nv_bfloat162 *a2 = reinterpret_cast<const __nv_bfloat162 *>(&araw);
                            __nv_bfloat162 hi[4], lo[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float2 a = __bfloat1622float2(a2[e]);
                                const float d0 = a.x > 0.0f ? __uint_as_float(v[8 * qd + 2 * e]) : 0.0f;
                                const float d1 = a.y > 0.0f ? __uint_as_float(v[8 * qd + 2 * e + 1]) : 0.0f;
                                dbacc[8 * qd + 2 * e] += d0;
                                dbacc[8 * qd + 2 * e + 1] += d1;
                                hi[e] = __floats2bfloat162_rn(d0, d1);
                                const float2 hf = __bfloat1622float2(hi[e]);
                                lo[e] = __floats2bfloat162_rn(d0 - hf.x, d1 - hf.y);
                            }
                            __nv_bfloat16 *yo = static_cast<__nv_bfloat16 *>(y) +
                                                ((((size_t)img * (Ho + 4) + oy + 2) * 8 + grp) * Pp + ox + 2) * 8;
                            *reinterpret_cast<uint4 *>(yo) = *reinterpret_cast<const uint4 *>(hi);
                            *reinterpret_cast<uint4 *>(yo + (size_t)4 * Pp * 8) = *reinterpret_cast<const uint4 *>(lo);
                        }
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
        if constexpr (MODE == kBwdData) {
            // this warp's bias-gradient partials (lanes summed in a fixed
            // butterfly): slot (CTA, lane quarter), channels of its half
#pragma unroll
            for (int c = 0; c < HALF; ++c) {
                float x = dbacc[c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                dbacc[c] = x;
            }
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < HALF; ++c)
                    dbpart[((size_t)blockIdx.x * 4 + quarter) * 32 + half * HALF + c] = dbacc[c];
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


// ---- training: loss, backward on the tensor cores ----------------------------

// BF16 rounded value and rounded remainder of an FP32 number
__device__ __forceinline__ void split_bf16(float d, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(d);
    lo = __float2bfloat16_rn(d - __bfloat162float(hi));
}

// loss = mean (s z - t)^2 over B x Ho x Wo x 3 (s = kOutScale, z the last
// pre-activation) and its gradient dz = 2 s (y - t) / n with y = s z the
// scaled output.  One thread per pixel: dz goes split into channels 0-2
// (rounded values) and 3-5 (remainders) of group 0 of the zero-padded
// (Ho + 4) x (Wo + 4) gradient image (16 channels; cleared beforehand).
// Per-block FP64 partial losses and FP32 partial bias gradients (slot = block),
// summed in block order later.
__global__ void __launch_bounds__(256) loss_grad_kernel(const float *__restrict__ y, const float *__restrict__ t,
                                                        int B, int Ho, int Wo, size_t n,
                                                        __nv_bfloat16 *__restrict__ dpad,
                                                        double *__restrict__ partial, float *__restrict__ dbpart) {
    __shared__ double red[256 / 32];
    __shared__ float redb[256 / 32][3];
    const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double acc = 0.0;
    float gb[3] = {0.0f, 0.0f, 0.0f};
    if (p < (size_t)B * Ho * Wo) {
        const int img = (int)(p / ((size_t)Ho * Wo));
        const int r = (int)(p % ((size_t)Ho * Wo));
        const int oy = r / Wo, ox = r % Wo;
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = y[p * 3 + c] - t[p * 3 + c];
            acc += (double)d * (double)d;
            gb[c] = 2.0f * kOutScale * d / (float)n;
            split_bf16(gb[c], o[c], o[3 + c]);
        }
        o[6] = o[7] = __float2bfloat16_rn(0.0f);
        const int Pp = fp_sur_pitch(Wo + 4);
        *reinterpret_cast<uint4 *>(dpad + ((((size_t)img * (Ho + 4) + oy + 2) * 2) * Pp + ox + 2) * 8) =
            *reinterpret_cast<const uint4 *>(o);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
#pragma unroll
        for (int c = 0; c < 3; ++c) gb[c] += __shfl_xor_sync(0xffffffffu, gb[c], o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = acc;
#pragma unroll
        for (int c = 0; c < 3; ++c) redb[threadIdx.x >> 5][c] = gb[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s2 = 0.0;
        float b3[3] = {0.0f, 0.0f, 0.0f};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s2 += red[w];
            for (int c = 0; c < 3; ++c) b3[c] += redb[w][c];
        }
        partial[blockIdx.x] = s2;
        for (int c = 0; c < 3; ++c) dbpart[(size_t)blockIdx.x * 32 + c] = b3[c];
    }
}

// the loss: the block partials summed by 256 threads (thread i: partials i,
// i + 256, ...) and a fixed-order tree, times scale
__global__ void __launch_bounds__(256) sum_partials_kernel(const double *__restrict__ partial, int n, double scale,
                                                           double *out) {
    __shared__ double red[256];
    double s2 = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) s2 += partial[k];
    red[threadIdx.x] = s2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * scale;
}

// weight gradient of one layer: dW[ky][kx][ci][co] = sum over output pixels p of
// X[p + (ky, kx)][ci] dZ[p][co], dZ the layer's output gradient (split).
// Work item: kWgR output rows x kWgSK output pixels of one image.  Per item the
// TMA producer (warp 0, one thread) copies the item's input rows (kWgR + ROWS
// - 1 of them) and gradient rows (kWgR), kWgNP pixels each from the item's
// first 32-pixel block, in their natural [row][channel group][pixel][8
// channels] form -- MN-major operands, pixels being K -- into one of two
// stages; the MMA issuer (warp 1, one thread) then issues per output row r,
// horizontal tap kx and 16-pixel chunk j one MMA: A = the input channels of
// input rows r .. r + ROWS - 1 (M = 128; the first three are vertical taps
// 0-2, the rest discarded), shifted by kx pixels (16 bytes), B = the gradient
// channels of output row r (shifted by the image's 2-pixel padding);
// accumulator kx (NB TMEM columns), and commits the stage back to the
// producer.  Pixels and rows past the data come in as zeros (the copies' fill
// and the padded image's zero border), so no masking is needed.  Items are
// taken in a fixed order per CTA and each CTA writes its sums (value +
// remainder) as part[cta][tap][CA][32]: the result is deterministic.  Every
// wait is bounded; a CTA that gives up waits for its copies in flight and
// frees its TMEM.
constexpr int kWgR = 4;                 // output rows per work item
constexpr int kWgSK = 64;               // output pixels per work item (four 16-pixel K chunks)
constexpr int kWgBlocks = 3;            // 32-pixel blocks copied per row (64 + the 2 taps, rounded up)
constexpr int kWgNP = 32 * kWgBlocks;   // staged pixels per row
constexpr int kWgThreads = 128;         // warp 0 producer, warp 1 issuer; all four the epilogue

template <int CA, int NB>
struct WgGeom {
    static constexpr int ROWS = 128 / CA;                // input rows stacked in M
    static constexpr int AROWS = kWgR + ROWS - 1;        // staged input rows per item
    static constexpr int AROW = (CA / 8) * kWgNP * 16;   // bytes of one staged input row
    static constexpr int ABYTES = AROWS * AROW;
    static constexpr int BROW = (NB / 8) * kWgNP * 16;   // bytes of one staged gradient row
    static constexpr int BBYTES = kWgR * BROW;
    static constexpr int STAGE = ABYTES + BBYTES;        // bytes one item's two copies bring
    static constexpr int SMEM = 2 * STAGE + 1024;
    static constexpr int TCOLS = 3 * NB <= 64 ? 64 : 3 * NB <= 128 ? 128 : 256;
    static_assert(CA * ROWS == 128 && ABYTES % 1024 == 0 && STAGE % 1024 == 0 && 3 * NB <= TCOLS,
                  "weight-gradient geometry");
};

// X (the layer's input, B x H x W, CA channels) through tmX, boxes of (256,
// kWgBlocks, CA / 8, AROWS, 1); its output gradient split into NB channels,
// in the zero-padded (H - 2 + 4) x (W - 2 + 4) image, through tmD, boxes of
// (256, kWgBlocks, NB / 8, kWgR, 1).  NB = 64: a hidden layer (32 rounded
// values, then 32 remainders); NB = 16: the last layer (3 rounded values, 3
// remainders, zeros).  Column co of the result is accumulator column co plus
// column co + LO.
template <int CA, int NB>
__global__ void __launch_bounds__(kWgThreads) conv_wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmX,
                                                                   const __grid_constant__ CUtensorMap tmD, int B,
                                                                   int H, int W, float *__restrict__ part,
                                                                   unsigned *err) {
    using G = WgGeom<CA, NB>;
    constexpr int LO = NB == 64 ? 32 : 3;  // column of the remainder of channel 0
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) unsigned long long bar_full[2], bar_empty[2], bar_done;
    __shared__ unsigned s_taddr;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Ho = H - 2, Wo = W - 2;
    const int strips = (Ho + kWgR - 1) / kWgR, segs = (Wo + kWgSK - 1) / kWgSK;
    const int items = B * strips * segs;
    // stages from the first 1024-byte boundary of the dynamic buffer
    const unsigned sm0 = sm_addr(sm), base = (sm0 + 1023u) & ~1023u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sm_addr(&s_taddr)),
                     "n"(G::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init_n(sm_addr(&bar_full[k]), 1);
            mbar_init_n(sm_addr(&bar_empty[k]), 1);
        }
        mbar_init_n(sm_addr(&bar_done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned taddr = s_taddr;
    // the four warps clear the three accumulators in their lane quarters
#pragma unroll
    for (int c = 0; c < 3 * NB; c += 16) tmem_zero<16>(taddr + ((unsigned)(32 * warp) << 16) + c);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    auto fail = [&]() {
        atomicOr(err, FP_ERR_TIMEOUT);
        s_abort = 1;
    };

    if (warp == 0) {
        // ---- TMA producer: both copies of an item into its stage
        if (lane == 0) {
            int it = 0;
            for (int item = blockIdx.x; item < items && !s_abort; item += gridDim.x, ++it) {
                const int st = it & 1;
                if (it >= 2 && !mbar_wait_or_abort(sm_addr(&bar_empty[st]), ((it - 2) >> 1) & 1, &s_abort)) {
                    fail();
                    break;
                }
                const int img = item / (strips * segs), rem = item % (strips * segs);
                const int oy0 = (rem / segs) * kWgR, blk = (rem % segs) * (kWgSK / 32);
                const unsigned sa = base + st * G::STAGE, sb = sa + G::ABYTES, fb = sm_addr(&bar_full[st]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(G::STAGE)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                    "%4, %5, %6}], [%7];" ::"r"(sa),
                    "l"(reinterpret_cast<unsigned long long>(&tmX)), "r"(0), "r"(blk), "r"(0), "r"(oy0), "r"(img),
                    "r"(fb)
                    : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                    "%4, %5, %6}], [%7];" ::"r"(sb),
                    "l"(reinterpret_cast<unsigned long long>(&tmD)), "r"(0), "r"(blk), "r"(0), "r"(oy0 + 2),
                    "r"(img), "r"(fb)
                    : "memory");
            }
            // no copy of this CTA may still be landing when it exits
            const int n = it < 2 ? it : 2;
            for (int k = 0; k < n; ++k) {
                const int q = it - 1 - k;
                mbar_wait_bounded(sm_addr(&bar_full[q & 1]), (q >> 1) & 1);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            const unsigned idesc = umma_idesc(128, NB) | (1u << 15) | (1u << 16);  // A and B MN-major
            int it = 0;
            for (int item = blockIdx.x; item < items; item += gridDim.x, ++it) {
                const int st = it & 1;
                if (!mbar_wait_or_abort(sm_addr(&bar_full[st]), (it >> 1) & 1, &s_abort)) {
                    fail();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned a0 = base + st * G::STAGE, b0 = a0 + G::ABYTES;
                for (int r = 0; r < kWgR; ++r)
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                        for (int j = 0; j < kWgSK / 16; ++j) {
                            // LBO = K-direction core stride (8 pixels), SBO = channel-group stride
                            const unsigned long long ad =
                                umma_desc(a0 + r * G::AROW + (16 * j + kx) * 16, 128, kWgNP * 16);
                            const unsigned long long bd =
                                umma_desc(b0 + r * G::BROW + (16 * j + 2) * 16, 128, kWgNP * 16);
                            mma_acc(taddr + kx * NB, ad, bd, idesc);
                        }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 sm_addr(&bar_empty[st]))
                             : "memory");
            }
            // every MMA issued above has completed once this arrives
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             sm_addr(&bar_done))
                         : "memory");
        }
    }
    // ---- epilogue (all four warps, once the roles are done): warp w reads
    // TMEM lanes 32 w ..: lane m = stacked row m / CA, channel m % CA
    __syncthreads();
    const bool done = mbar_wait_bounded(sm_addr(&bar_done), 0u);
    if (!__all_sync(0xffffffffu, done) && lane == 0) fail();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (!s_abort) {
        const int m = 32 * warp + lane, rr = m / CA, ca = m % CA;
        float *pc = part + (size_t)blockIdx.x * 9 * CA * 32;
        const unsigned tl = taddr + ((unsigned)(32 * warp) << 16);
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            if constexpr (NB == 64) {
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    unsigned hi[16], lo[16];
                    tmem_load<16>(tl + kx * NB + 16 * half, hi);
                    tmem_load<16>(tl + kx * NB + LO + 16 * half, lo);
                    if (rr < 3)
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            pc[((rr * 3 + kx) * CA + ca) * 32 + 16 * half + c] =
                                __uint_as_float(hi[c]) + __uint_as_float(lo[c]);
                }
            } else {
                unsigned v[16];
                tmem_load<16>(tl + kx * NB, v);
                if (rr < 3)
#pragma unroll
                    for (int c = 0; c < LO; ++c)
                        pc[((rr * 3 + kx) * CA + ca) * 32 + c] = __uint_as_float(v[c]) + __uint_as_float(v[c + LO]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(G::TCOLS));
}

// dW (master layout [tap][ci][co]) and db of every layer in one launch
// (blockIdx.y = layer): the per-CTA weight partials part[cta][tap][CA][32] and
// the bias partials dbpart[slot][32] of the layer.  A block takes 32
// consecutive outputs; thread (g, o) sums partials g, g + 32, ... of output
// o, then the 32 sums are added in order (deterministic).
struct ReduceJobs {
    const float *part[kLayers], *dbpart[kLayers];
    float *dw[kLayers], *db[kLayers];
    int ctas[kLayers], CA[kLayers], ci[kLayers], co[kLayers], slots[kLayers];
};

__global__ void __launch_bounds__(1024) grad_reduce_kernel(const __grid_constant__ ReduceJobs J) {
    __shared__ float red[32][33];
    const int l = blockIdx.y;
    const int o = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + o;
    const int ci_real = J.ci[l], co_real = J.co[l], CA = J.CA[l];
    const int nw = 9 * ci_real * co_real;
    if ((int)blockIdx.x * 32 >= nw + co_real) return;  // block-uniform: this layer has fewer outputs
    float acc = 0.0f;
    if (k < nw) {
        const int co = k % co_real, ci = (k / co_real) % ci_real, t = k / (co_real * ci_real);
        const float *p = J.part[l] + ((size_t)t * CA + ci) * 32 + co;
        const size_t stride = (size_t)9 * CA * 32;
#pragma unroll 4
        for (int c = g; c < J.ctas[l]; c += 32) acc += p[c * stride];
    } else if (k < nw + co_real) {
#pragma unroll 4
        for (int q = g; q < J.slots[l]; q += 32) acc += J.dbpart[l][(size_t)q * 32 + (k - nw)];
    }
    red[g][o] = acc;
    __syncthreads();
    if (g == 0 && k < nw + co_real) {
        float sum = 0.0f;
        for (int j = 0; j < 32; ++j) sum += red[j][o];
        if (k < nw)
            J.dw[l][k] = sum;
        else
            J.db[l][k - nw] = sum;
    }
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
__device__ void pack_layer_at(int k, const float *__restrict__ w, const float *__restrict__ b, int ci_real,
                              int co_real, int ci_pad, int co_pad, __nv_bfloat16 *__restrict__ pk,
                              float *__restrict__ bias) {
    const int kc = ci_pad / 16, rows = 3 * co_pad;
    const int total = 3 * kc * 2 * rows * 8;
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

// FP32 master (one layer, ci_real x co_real) -> the packed BF16 operand of its
// data gradient, in the forward kernel's block format with kWidth output
// channels: input channel k is a channel of the split output gradient (k <
// co_real the rounded value of channel k, co_real <= k < 2 co_real the
// remainder of channel k - co_real, zero beyond), output channel n the
// layer's input channel n, tap (ky, kx) the layer's tap (2 - ky, 2 - kx).
__device__ void pack_layer_bwd_at(int k, const float *__restrict__ w, int ci_real, int co_real, int cin_b,
                                  __nv_bfloat16 *__restrict__ pk) {
    const int kc = cin_b / 16, rows = 3 * kWidth;
    const int total = 3 * kc * 2 * rows * 8;
    if (k >= total) return;
    const int e = k % 8, n3 = (k / 8) % rows, j = (k / (8 * rows)) % 2;
    const int c = (k / (16 * rows)) % kc, kx = k / (16 * rows * kc);
    const int ky = 2 - n3 / kWidth, n = n3 % kWidth;
    const int kin = 16 * c + 8 * j + e;
    const int co = kin < co_real ? kin : kin < 2 * co_real ? kin - co_real : -1;
    const int t = 3 * (2 - ky) + (2 - kx);
    float v = 0.0f;
    if (co >= 0 && n < ci_real) v = w[((size_t)t * ci_real + n) * co_real + co];
    pk[k] = __float2bfloat16(v);
}

// every packing of the master weights in one launch: job j < kLayers the
// forward operand and bias of layer j, job kLayers - 1 + l the data-gradient
// operand of layer l (1 <= l < kLayers); one thread per packed value
struct PackJobs {
    const float *w[2 * kLayers - 1], *b[2 * kLayers - 1];
    __nv_bfloat16 *pk[2 * kLayers - 1];
    float *bias[2 * kLayers - 1];
    int ci_real[2 * kLayers - 1], co_real[2 * kLayers - 1], ci_pad[2 * kLayers - 1], co_pad[2 * kLayers - 1];
};

__global__ void pack_all_kernel(const __grid_constant__ PackJobs J) {
    const int j = blockIdx.y, k = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < kLayers)
        pack_layer_at(k, J.w[j], J.b[j], J.ci_real[j], J.co_real[j], J.ci_pad[j], J.co_pad[j], J.pk[j], J.bias[j]);
    else
        pack_layer_bwd_at(k, J.w[j], J.ci_real[j], J.co_real[j], J.ci_pad[j], J.pk[j]);
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
    __nv_bfloat16 *d_wpack_bwd[kLayers] = {};     // packed data-gradient weights (layers 1-4)
    float *d_bias[kLayers] = {};                  // padded FP32 biases per layer
    unsigned *d_err = nullptr;
    double *d_loss = nullptr, *d_partial = nullptr;
    long long adam_t = 0;
    // cached scratch: activations (BF16) and output (FP32)
    size_t cap_pix = 0, cap_partial = 0;
    __nv_bfloat16 *d_a[kLayers] = {};             // inputs of every layer (a[0] packed input)
    float *d_out = nullptr;
    // backward scratch: two padded split-gradient images, per layer the
    // weight-gradient partials of up to part_ctas CTAs and the bias-gradient
    // partials of up to cap_slots slots
    size_t cap_dpad = 0, cap_slots = 0;
    __nv_bfloat16 *d_dpad[2] = {};
    float *d_part = nullptr, *d_dbpart = nullptr;
    int part_ctas = 0;
    int max_ctas = 0;          // CTAs per kernel at most (0: no limit)
    int smem_per_sm = 233472;  // shared memory per SM (bytes)
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

constexpr int kConvMaxPerSM = 3;  // resident convolution CTAs per SM at most

// The dynamic shared-memory limit of a kernel raised to bytes on the current
// device, once per (kernel, device): the kernel's address keys the record.
template <typename K>
cudaError_t set_smem_once(K *kernel, int bytes) {
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &d : done)
        if (d.first == (const void *)kernel && d.second == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.emplace_back((const void *)kernel, dev);
    return e;
}

// one implicit-GEMM convolution of B x H x W images x (CIN channels) into y
// (act, dbpart: the data-gradient epilogue's mask and partials; grid_out: the
// CTAs launched, each leaving 4 bias-gradient slots in that epilogue)
template <int CIN, int COUT, int MODE>
cudaError_t launch_conv(const fp_surrogate *s, const __nv_bfloat16 *wpack, const float *bias,
                        const __nv_bfloat16 *x, int B, int H, int W, void *y, const __nv_bfloat16 *act,
                        float *dbpart, int *grid_out, cudaStream_t st) {
    using G = ConvGeom<CIN, COUT>;
    {
        cudaError_t e = set_smem_once(conv3x3_tc_kernel<CIN, COUT, MODE>, G::SMEM);
        if (e != cudaSuccess) return e;
    }
    // resident CTAs per SM: shared memory (the dynamic part plus 2 KB of static
    // and reserved per CTA), TMEM (512 / TCOLS columns), at most three
    const int per_sm =
        std::max(1, std::min(std::min(kConvMaxPerSM, s->smem_per_sm / (G::SMEM + 2048)), 512 / G::TCOLS));
    CUtensorMap m;
    cudaError_t e = encode_act_map<CIN>(&m, x, B, H, W);
    if (e != cudaSuccess) return e;
    // strip height 32, 16 or 8 output rows: a CTA's time ~ its items x
    // (strip + the two halo rows staged per item), so the fewest waves of
    // items x (strip + 2), the taller strip on ties (small images get short
    // strips and use more SMs)
    const long long segs = ((W - 2) + kSeg - 1) / kSeg;
    const long long resident = s->max_ctas > 0 ? std::min<long long>(s->max_ctas, (long long)s->sms * per_sm)
                                               : (long long)s->sms * per_sm;
    int strip = kStripRows;
    long long best = -1;
    for (int sr = kStripRows; sr >= 8; sr /= 2) {
        const long long n = (long long)B * segs * (((H - 2) + sr - 1) / sr);
        const long long cost = (n + resident - 1) / resident * (sr + 2);
        if (best < 0 || cost < best) {
            best = cost;
            strip = sr;
        }
    }
    const long long items = (long long)B * segs * (((H - 2) + strip - 1) / strip);
    int grid = (int)std::min<long long>(items, resident);
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = grid;
    conv3x3_tc_kernel<CIN, COUT, MODE><<<grid, kConvWarps * 32, G::SMEM, st>>>(m, B, H, W, strip, wpack, bias, y,
                                                                              act, dbpart, s->d_err);
    return cudaGetLastError();
}

// 5-D view (256 elements = 32 pixels x 8 channels, 32-pixel block, channel
// group, row, image) of a BF16 image batch of `rows` rows, row pitch P pixels
// and C channels in groups of 8, with boxes of (256, blocks, C / 8, box_rows, 1)
cudaError_t encode_rows_map(CUtensorMap *m, const __nv_bfloat16 *x, int B, int rows, int P, int C, int blocks,
                            int box_rows) {
    auto enc = tmap_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[5] = {256, (cuuint64_t)(P / 32), (cuuint64_t)(C / 8), (cuuint64_t)rows, (cuuint64_t)B};
    const cuuint64_t strides[4] = {512, (cuuint64_t)P * 16, (cuuint64_t)P * C * 2, (cuuint64_t)rows * P * C * 2};
    const cuuint32_t box[5] = {256, (cuuint32_t)blocks, (cuuint32_t)(C / 8), (cuuint32_t)box_rows, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(x), dims, strides,
                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// the weight gradient of a layer with input X (B x H x W, CA channels) and
// split output gradient D (NB channels, padded); partials of *ctas CTAs in part
template <int CA, int NB>
cudaError_t launch_wgrad(const fp_surrogate *s, const __nv_bfloat16 *X, const __nv_bfloat16 *D, int B, int H, int W,
                         float *part, int *ctas, cudaStream_t st) {
    using G = WgGeom<CA, NB>;
    {
        cudaError_t e = set_smem_once(conv_wgrad_tc_kernel<CA, NB>, G::SMEM);
        if (e != cudaSuccess) return e;
    }
    CUtensorMap mx, md;
    cudaError_t e = encode_rows_map(&mx, X, B, H, fp_sur_pitch(W), CA, kWgBlocks, G::AROWS);
    if (e == cudaSuccess) e = encode_rows_map(&md, D, B, H - 2 + 4, fp_sur_pitch(W - 2 + 4), NB, kWgBlocks, kWgR);
    if (e != cudaSuccess) return e;
    const long long items = (long long)B * ((H - 2 + kWgR - 1) / kWgR) * ((W - 2 + kWgSK - 1) / kWgSK);
    const int cap = s->max_ctas > 0 ? std::min(s->max_ctas, s->part_ctas) : s->part_ctas;
    int grid = (int)std::min<long long>(items, (long long)cap);
    if (grid < 1) grid = 1;
    *ctas = grid;
    conv_wgrad_tc_kernel<CA, NB><<<grid, kWgThreads, G::SMEM, st>>>(mx, md, B, H, W, part, s->d_err);
    return cudaGetLastError();
}

size_t param_count() {
    size_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += (size_t)9 * kCh[l] * kCh[l + 1] + kCh[l + 1];
    return n;
}

// FP32 master -> packed BF16 operand blocks and padded biases, and the
// data-gradient operands (on the device, one launch)
cudaError_t repack(fp_surrogate *s, cudaStream_t st) {
    PackJobs J{};
    int most = 0;
    for (int j = 0; j < 2 * kLayers - 1; ++j) {
        const int l = j < kLayers ? j : j - kLayers + 1;
        J.w[j] = s->d_master + s->w_off[l];
        J.b[j] = s->d_master + s->b_off[l];
        J.ci_real[j] = kCh[l];
        J.co_real[j] = kCh[l + 1];
        int total;
        if (j < kLayers) {
            J.ci_pad[j] = l == 0 ? kCin0 : kWidth;  // input channels of the operand
            J.co_pad[j] = l == kLayers - 1 ? kCout4 : kWidth;
            J.pk[j] = s->d_wpack[l];
            J.bias[j] = s->d_bias[l];
            total = 9 * (J.ci_pad[j] / 16) * 2 * J.co_pad[j] * 8;
        } else {
            J.ci_pad[j] = l == kLayers - 1 ? 16 : 2 * kWidth;  // split gradient channels
            J.pk[j] = s->d_wpack_bwd[l];
            total = 3 * (J.ci_pad[j] / 16) * 2 * 3 * kWidth * 8;
        }
        most = std::max(most, total);
    }
    pack_all_kernel<<<dim3((most + 255) / 256, 2 * kLayers - 1), 256, 0, st>>>(J);
    return cudaGetLastError();
}

// pix: images x rows x row pitch (pixels) of the largest input
bool ensure_scratch(fp_surrogate *s, size_t pix) {
    if (pix <= s->cap_pix) return true;
    for (int l = 0; l < kLayers; ++l) cudaFree(s->d_a[l]);
    cudaFree(s->d_out); cudaFree(s->d_partial);
    s->cap_pix = 0;
    bool ok = cudaMalloc(&s->d_a[0], pix * kCin0 * sizeof(__nv_bfloat16)) == cudaSuccess;
    for (int l = 1; l < kLayers; ++l) ok &= cudaMalloc(&s->d_a[l], pix * kWidth * sizeof(__nv_bfloat16)) == cudaSuccess;
    ok &= cudaMalloc(&s->d_out, pix * 3 * sizeof(float)) == cudaSuccess;
    s->cap_partial = (pix * 3 + 255) / 256 + 1;
    ok &= cudaMalloc(&s->d_partial, s->cap_partial * sizeof(double)) == cudaSuccess;
    // activation rows are padded to 32 pixels: keep the padding finite
    for (int l = 0; l < kLayers && ok; ++l)
        ok = cudaMemset(s->d_a[l], 0, pix * (l == 0 ? kCin0 : kWidth) * sizeof(__nv_bfloat16)) == cudaSuccess;
    if (ok) s->cap_pix = pix;
    return ok;
}

// backward scratch for B x H x W inputs: padded split gradients up to
// (H + 2) x (W + 2) x 64 channels; per layer, bias-gradient slots for the loss
// blocks or four per convolution CTA
bool ensure_bwd(fp_surrogate *s, int B, int H, int W) {
    const size_t dpad = (size_t)B * (H + 2) * fp_sur_pitch(W + 2) * 2 * kWidth;
    const size_t slots = std::max<size_t>(((size_t)B * H * W + 255) / 256 + 1,
                                          (size_t)4 * kConvMaxPerSM * s->sms);
    if (dpad <= s->cap_dpad && slots <= s->cap_slots) return true;
    cudaFree(s->d_dpad[0]); cudaFree(s->d_dpad[1]); cudaFree(s->d_dbpart);
    s->cap_dpad = s->cap_slots = 0;
    bool ok = cudaMalloc(&s->d_dpad[0], dpad * sizeof(__nv_bfloat16)) == cudaSuccess;
    ok &= cudaMalloc(&s->d_dpad[1], dpad * sizeof(__nv_bfloat16)) == cudaSuccess;
    ok &= cudaMalloc(&s->d_dbpart, (size_t)kLayers * slots * 32 * sizeof(float)) == cudaSuccess;
    if (ok) {
        s->cap_dpad = dpad;
        s->cap_slots = slots;
    }
    return ok;
}

// the five layers from a packed BF16 input in0 [B][H][W][16]; every later
// layer's input stays in d_a; output to out
cudaError_t forward_layers(fp_surrogate *s, const __nv_bfloat16 *in0, int B, int H, int W, float *out,
                           cudaStream_t st) {
    cudaError_t e = launch_conv<kCin0, kWidth, kHidden>(s, s->d_wpack[0], s->d_bias[0], in0, B, H, W, s->d_a[1],
                                                        nullptr, nullptr, nullptr, st);
    int h = H - 2, w = W - 2;
    for (int l = 1; l < kLayers - 1 && e == cudaSuccess; ++l) {
        e = launch_conv<kWidth, kWidth, kHidden>(s, s->d_wpack[l], s->d_bias[l], s->d_a[l], B, h, w, s->d_a[l + 1],
                                                 nullptr, nullptr, nullptr, st);
        h -= 2; w -= 2;
    }
    if (e == cudaSuccess)
        e = launch_conv<kWidth, kCout4, kLast>(s, s->d_wpack[kLayers - 1], s->d_bias[kLayers - 1],
                                               s->d_a[kLayers - 1], B, h, w, out, nullptr, nullptr, nullptr, st);
    return e;
}

// forward of B images x [B][H][W][4] keeping every layer's input in d_a; output to out
cudaError_t forward_keep(fp_surrogate *s, const float *x, int B, int H, int W, float *out, cudaStream_t st) {
    const size_t npix0 = (size_t)B * H * W;
    pack_input_kernel<<<(unsigned)((npix0 + 255) / 256), 256, 0, st>>>(x, B, H, W, s->d_a[0]);
    return forward_layers(s, s->d_a[0], B, H, W, out, st);
}

// loss and gradients (into d_grad, master layout) of the last forward_keep.
// Layer l (input H - 2l x W - 2l): weight-gradient partials from its input and
// split output gradient; then (l > 0) the data gradient into the other padded
// image, whose epilogue leaves the bias partials of layer l - 1.  Every
// layer's partials have buffers of their own, reduced in one launch at the end.
cudaError_t backward(fp_surrogate *s, const float *target, int B, int H, int W, cudaStream_t st) {
    const int H5 = H - 2 * kLayers, W5 = W - 2 * kLayers;
    const size_t npix = (size_t)B * H5 * W5, n_out = npix * 3;
    const unsigned nb = (unsigned)((npix + 255) / 256);
    const size_t part_stride = (size_t)s->part_ctas * 9 * kWidth * 32, slot_stride = s->cap_slots * 32;
    ReduceJobs J{};
    __nv_bfloat16 *cur = s->d_dpad[0], *nxt = s->d_dpad[1];
    cudaError_t e = cudaMemsetAsync(cur, 0, (size_t)B * (H5 + 4) * fp_sur_pitch(W5 + 4) * 16 * sizeof(__nv_bfloat16),
                                    st);
    if (e != cudaSuccess) return e;
    loss_grad_kernel<<<nb, 256, 0, st>>>(s->d_out, target, B, H5, W5, n_out, cur, s->d_partial,
                                         s->d_dbpart + (kLayers - 1) * slot_stride);
    sum_partials_kernel<<<1, 256, 0, st>>>(s->d_partial, (int)nb, 1.0 / (double)n_out, s->d_loss);
    J.slots[kLayers - 1] = (int)nb;
    int most = 0;  // blocks of the largest layer's reduction
    for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
        const int Hl = H - 2 * l, Wl = W - 2 * l;
        float *part = s->d_part + l * part_stride;
        if (l == kLayers - 1)
            e = launch_wgrad<kWidth, 16>(s, s->d_a[l], cur, B, Hl, Wl, part, &J.ctas[l], st);
        else if (l > 0)
            e = launch_wgrad<kWidth, 2 * kWidth>(s, s->d_a[l], cur, B, Hl, Wl, part, &J.ctas[l], st);
        else
            e = launch_wgrad<kCin0, 2 * kWidth>(s, s->d_a[0], cur, B, Hl, Wl, part, &J.ctas[l], st);
        if (e != cudaSuccess) break;
        J.part[l] = part;
        J.dbpart[l] = s->d_dbpart + l * slot_stride;
        J.dw[l] = s->d_grad + s->w_off[l];
        J.db[l] = s->d_grad + s->b_off[l];
        J.CA[l] = l == 0 ? kCin0 : kWidth;
        J.ci[l] = kCh[l];
        J.co[l] = kCh[l + 1];
        most = std::max(most, (9 * kCh[l] * kCh[l + 1] + kCh[l + 1] + 31) / 32);
        if (l == 0) break;
        e = cudaMemsetAsync(nxt, 0, (size_t)B * (Hl + 4) * fp_sur_pitch(Wl + 4) * 2 * kWidth * sizeof(__nv_bfloat16),
                            st);
        if (e != cudaSuccess) break;
        int grid = 0;
        float *dbp = s->d_dbpart + (l - 1) * slot_stride;
        if (l == kLayers - 1)
            e = launch_conv<16, kWidth, kBwdData>(s, s->d_wpack_bwd[l], nullptr, cur, B, Hl + 2, Wl + 2, nxt,
                                                  s->d_a[l], dbp, &grid, st);
        else
            e = launch_conv<2 * kWidth, kWidth, kBwdData>(s, s->d_wpack_bwd[l], nullptr, cur, B, Hl + 2, Wl + 2, nxt,
                                                          s->d_a[l], dbp, &grid, st);
        J.slots[l - 1] = 4 * grid;
        std::swap(cur, nxt);
    }
    if (e == cudaSuccess) {
        grad_reduce_kernel<<<dim3(most, kLayers), 1024, 0, st>>>(J);
        e = cudaGetLastError();
    }
    return e;
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
    cudaDeviceGetAttribute(&s->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
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
        if (l > 0) {
            const size_t cin_b = l == kLayers - 1 ? 16 : 2 * kWidth;
            ok &= (s->d_wpack_bwd[l] = static_cast<__nv_bfloat16 *>(alloc(9 * cin_b * kWidth * 2))) != nullptr;
        }
    }
    s->part_ctas = s->sms;  // one weight-gradient CTA per SM
    ok &= (s->d_part = static_cast<float *>(alloc((size_t)kLayers * s->part_ctas * 9 * kWidth * 32 * sizeof(float)))) !=
          nullptr;
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
    cudaFree(s->d_out); cudaFree(s->d_partial);
    cudaFree(s->d_dpad[0]); cudaFree(s->d_dpad[1]); cudaFree(s->d_dbpart);
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
    if (!ensure_scratch(s, (size_t)B * H * fp_sur_pitch(W)) || !ensure_bwd(s, B, H, W)) {
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

int fp_surrogate_set_max_ctas(fp_surrogate *s, int32_t ctas) {
    if (!s || ctas < 0) return FP_EINVAL;
    s->max_ctas = ctas;
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
