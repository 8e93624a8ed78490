// surrogate.cu -- the learned flood surrogate (build-added; the paper has no
// surrogate): a 5-layer 3x3 convolutional net 4 -> 32 -> 32 -> 32 -> 32 -> 3
// (ReLU between layers) mapping (h, hu, hv, z) around a cell to the change of
// (h, hu, hv) over 8 fixed time steps.
//
// Forward (inference and training): each layer is an implicit GEMM on the
// 5th-generation tensor cores -- tcgen05.mma, kind::f16 with BF16 operands in
// shared memory and an FP32 accumulator in tensor memory (TMEM):
//   M = 128 output pixels of one row, N = 32 output channels (16 for the last
//   layer, 3 used), K = 9 taps x input channels in steps of 16.
// A CTA (128 threads) is persistent over output row segments.  It keeps the
// layer's weights in shared memory in the canonical no-swizzle K-major layout
// (core matrices of 8 rows x 16 bytes; k-cores LBO apart, 8-row groups SBO
// apart) and stages the three input rows of a segment as
// [k-core][pixel][8 channels]: the three horizontal taps of an input row are
// then the same operand shifted by 16 bytes.  One thread issues the MMAs and
// commits them to an mbarrier (bounded wait); the four warps read their 32
// TMEM lanes with tcgen05.ld for the bias / ReLU / BF16 epilogue.  TMEM is
// freed on every exit path.
//
// Training (A13): the backward pass (data and weight gradients of every
// layer, FP32 on the CUDA cores, deterministic reductions), the loss and Adam
// with FP32 master weights.
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
constexpr int kCin0 = 16;   // first layer: 4 real input channels padded to 16
constexpr int kCout4 = 16;  // last layer: 3 real output channels padded to 16
constexpr int kSeg = 128;   // output pixels per MMA (M)
constexpr int kConvThreads = 128;
constexpr float kOutScale = 0.1f;  // the net predicts delta U / 0.1
constexpr int kCh[kLayers + 1] = {4, kWidth, kWidth, kWidth, kWidth, 3};

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

template <int CIN, int COUT>
struct ConvGeom {
    static constexpr int KC = CIN / 16;            // K chunks of 16 channels
    static constexpr int NKC = CIN / 8;            // 16-byte k-cores per pixel
    static constexpr int NPIX = kSeg + 2;          // staged input pixels per row
    static constexpr int ROWB = NKC * NPIX * 16;   // bytes per staged input row
    static constexpr int WBLK = 2 * COUT * 16;     // bytes per (tap, chunk) weight block
    static constexpr int WB = 9 * KC * WBLK;       // weight bytes
    // guard region after the operands (a descriptor-field error reads garbage inside the allocation)
    static constexpr int SMEM = ((WB + 3 * ROWB + 16 * NPIX * 16 + 2048) + 1023) / 1024 * 1024;
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

template <int N>
__device__ __forceinline__ void tmem_load(unsigned taddr, unsigned (&r)[N]);

template <>
__device__ __forceinline__ void tmem_load<32>(unsigned taddr, unsigned (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
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

// One 3x3 valid convolution of B images (NHWC, BF16, CIN channels) with the
// packed weights (9 taps x CIN/16 chunks of [2 k-cores][COUT rows][8] BF16).
// Hidden layers: bias + ReLU, BF16 output with COUT channels.  Last layer
// (LAST): bias, FP32 output with 3 channels, times kOutScale.
template <int CIN, int COUT, bool LAST>
__global__ void __launch_bounds__(kConvThreads) conv3x3_tc_kernel(const __nv_bfloat16 *__restrict__ x, int B, int H,
                                                                  int W, const __nv_bfloat16 *__restrict__ wpack,
                                                                  const float *__restrict__ bias, void *__restrict__ y,
                                                                  unsigned *err) {
    using G = ConvGeom<CIN, COUT>;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *s_w = sm;
    unsigned char *s_x = sm + G::WB;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned s_taddr;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Ho = H - 2, Wo = W - 2;
    const int segs_per_row = (Wo + kSeg - 1) / kSeg;
    const int nseg = B * Ho * segs_per_row;
    constexpr unsigned IDESC = umma_idesc(kSeg, COUT);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(sm_addr(&s_taddr)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    for (int i = tid; i < G::WB / 16; i += kConvThreads)
        reinterpret_cast<uint4 *>(s_w)[i] = reinterpret_cast<const uint4 *>(wpack)[i];
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned taddr = s_taddr;
    unsigned phase = 0;

    for (int seg = blockIdx.x; seg < nseg; seg += gridDim.x) {
        const int img = seg / (Ho * segs_per_row);
        const int rem = seg % (Ho * segs_per_row);
        const int oy = rem / segs_per_row, ox0 = (rem % segs_per_row) * kSeg;
        const __nv_bfloat16 *xin = x + (size_t)img * H * W * CIN;
        // stage input rows oy .. oy+2, pixels ox0 .. ox0+129, as [row][k-core][pixel][8 channels]
        for (int u = tid; u < 3 * G::NKC * G::NPIX; u += kConvThreads) {
            const int r = u / (G::NKC * G::NPIX), q = u % (G::NKC * G::NPIX);
            const int j = q / G::NPIX, p = q % G::NPIX;
            const int ix = ox0 + p;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (ix < W) v = *reinterpret_cast<const uint4 *>(xin + ((size_t)(oy + r) * W + ix) * CIN + j * 8);
            *reinterpret_cast<uint4 *>(s_x + r * G::ROWB + (j * G::NPIX + p) * 16) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const unsigned xs = sm_addr(s_x), ws = sm_addr(s_w);
#pragma unroll 1
            for (int t = 0; t < 9; ++t) {
                const int ky = t / 3, kx = t % 3;
#pragma unroll
                for (int c = 0; c < G::KC; ++c) {
                    const unsigned a = xs + ky * G::ROWB + (2 * c) * (G::NPIX * 16) + kx * 16;
                    const unsigned b = ws + (t * G::KC + c) * G::WBLK;
                    const unsigned long long ad = umma_desc(a, G::NPIX * 16, 128);
                    const unsigned long long bd = umma_desc(b, COUT * 16, 128);
                    const unsigned acc = (t | c) != 0 ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
                        "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             sm_addr(&mbar))
                         : "memory");
        }
        const bool done = mbar_wait_bounded(sm_addr(&mbar), phase);
        phase ^= 1u;
        if (!done) {
            if (lane == 0) atomicOr(err, FP_ERR_TIMEOUT);
            s_ok = 0;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (!s_ok) break;
        // epilogue: warp w owns TMEM lanes (output pixels) 32w .. 32w+31
        const int m = 32 * warp + lane;
        const int ox = ox0 + m;
        unsigned r[COUT];
        tmem_load<COUT>(taddr + ((unsigned)(32 * warp) << 16), r);
        if (ox < Wo) {
            const size_t pix = ((size_t)img * Ho + oy) * Wo + ox;
            if constexpr (LAST) {
                float *yo = static_cast<float *>(y) + pix * 3;
#pragma unroll
                for (int co = 0; co < 3; ++co) yo[co] = (__uint_as_float(r[co]) + bias[co]) * kOutScale;
            } else {
                __nv_bfloat16 *yo = static_cast<__nv_bfloat16 *>(y) + pix * COUT;
#pragma unroll
                for (int q = 0; q < COUT / 8; ++q) {
                    __nv_bfloat162 v[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float a0 = fmaxf(__uint_as_float(r[8 * q + 2 * e]) + bias[8 * q + 2 * e], 0.0f);
                        const float a1 = fmaxf(__uint_as_float(r[8 * q + 2 * e + 1]) + bias[8 * q + 2 * e + 1], 0.0f);
                        v[e] = __floats2bfloat162_rn(a0, a1);
                    }
                    *reinterpret_cast<uint4 *>(yo + 8 * q) = *reinterpret_cast<const uint4 *>(v);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(taddr));
}

// FP32 (h, hu, hv, z) images -> BF16 NHWC with 16 channels (4 used)
__global__ void pack_input_kernel(const float *__restrict__ x4, size_t npix, __nv_bfloat16 *__restrict__ out) {
    const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const float4 v = reinterpret_cast<const float4 *>(x4)[p];
    __nv_bfloat162 o[8];
    o[0] = __floats2bfloat162_rn(v.x, v.y);
    o[1] = __floats2bfloat162_rn(v.z, v.w);
#pragma unroll
    for (int k = 2; k < 8; ++k) o[k] = __floats2bfloat162_rn(0.f, 0.f);
    uint4 *dst = reinterpret_cast<uint4 *>(out + p * 16);
    dst[0] = reinterpret_cast<const uint4 *>(o)[0];
    dst[1] = reinterpret_cast<const uint4 *>(o)[1];
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct fp_surrogate {
    std::vector<float> master;                    // FP32 parameters, per layer w[3][3][ci][co] then b[co]
    std::vector<size_t> w_off, b_off;             // offsets into master
    __nv_bfloat16 *d_wpack[kLayers] = {};         // packed BF16 weights per layer
    float *d_bias[kLayers] = {};                  // padded FP32 biases per layer
    unsigned *d_err = nullptr;
    std::vector<void *> allocs;
    int sms = 148;
    std::string err;
};

namespace {

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
    const long long nseg = (long long)B * (H - 2) * (((W - 2) + kSeg - 1) / kSeg);
    int grid = (int)std::min<long long>(nseg, (long long)s->sms * 3);
    if (grid < 1) grid = 1;
    conv3x3_tc_kernel<CIN, COUT, LAST><<<grid, kConvThreads, G::SMEM, st>>>(x, B, H, W, s->d_wpack[layer],
                                                                             s->d_bias[layer], y, s->d_err);
    return cudaGetLastError();
}

size_t param_count() {
    size_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += (size_t)9 * kCh[l] * kCh[l + 1] + kCh[l + 1];
    return n;
}

// master FP32 -> packed BF16 operand blocks [tap][chunk][k-core][co][8] and padded biases
cudaError_t upload_packed(fp_surrogate *s) {
    for (int l = 0; l < kLayers; ++l) {
        const int ci_pad = l == 0 ? kCin0 : kWidth, co_pad = l == kLayers - 1 ? kCout4 : kWidth;
        const int kc = ci_pad / 16;
        std::vector<__nv_bfloat16> pk((size_t)9 * kc * 2 * co_pad * 8, __float2bfloat16(0.0f));
        const float *w = s->master.data() + s->w_off[l];
        for (int t = 0; t < 9; ++t)
            for (int c = 0; c < kc; ++c)
                for (int j = 0; j < 2; ++j)
                    for (int n = 0; n < co_pad; ++n)
                        for (int e = 0; e < 8; ++e) {
                            const int ci = 16 * c + 8 * j + e;
                            float v = 0.0f;
                            if (ci < kCh[l] && n < kCh[l + 1]) v = w[((size_t)t * kCh[l] + ci) * kCh[l + 1] + n];
                            pk[((((size_t)t * kc + c) * 2 + j) * co_pad + n) * 8 + e] = __float2bfloat16(v);
                        }
        std::vector<float> b(co_pad, 0.0f);
        for (int n = 0; n < kCh[l + 1]; ++n) b[n] = s->master[s->b_off[l] + n];
        cudaError_t e = cudaMemcpy(s->d_wpack[l], pk.data(), pk.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(s->d_bias[l], b.data(), b.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    return cudaDeviceSynchronize();
}

}  // namespace

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
    s->master.assign(o, 0.0f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < kLayers; ++l) {
        std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / (9.0f * kCh[l])));
        for (size_t k = 0; k < (size_t)9 * kCh[l] * kCh[l + 1]; ++k) s->master[s->w_off[l] + k] = nd(rng);
        if (l == kLayers - 1)
            for (size_t k = 0; k < (size_t)9 * kCh[l] * kCh[l + 1]; ++k) s->master[s->w_off[l] + k] *= 0.1f;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    bool ok = true;
    for (int l = 0; l < kLayers; ++l) {
        const int ci_pad = l == 0 ? kCin0 : kWidth, co_pad = l == kLayers - 1 ? kCout4 : kWidth;
        void *p = nullptr, *q = nullptr;
        ok &= cudaMalloc(&p, (size_t)9 * ci_pad * co_pad * sizeof(__nv_bfloat16)) == cudaSuccess;
        ok &= cudaMalloc(&q, (size_t)co_pad * sizeof(float)) == cudaSuccess;
        s->allocs.push_back(p);
        s->allocs.push_back(q);
        s->d_wpack[l] = static_cast<__nv_bfloat16 *>(p);
        s->d_bias[l] = static_cast<float *>(q);
    }
    void *e = nullptr;
    ok &= cudaMalloc(&e, sizeof(unsigned)) == cudaSuccess;
    s->allocs.push_back(e);
    s->d_err = static_cast<unsigned *>(e);
    if (ok) ok = cudaMemset(s->d_err, 0, sizeof(unsigned)) == cudaSuccess;
    if (!ok || upload_packed(s) != cudaSuccess) {
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
    for (void *p : s->allocs) cudaFree(p);
    delete s;
    return FP_OK;
}

int fp_surrogate_get_params(fp_surrogate *s, float *dst, size_t n) {
    if (!s || !dst || n < s->master.size()) return FP_EINVAL;
    memcpy(dst, s->master.data(), s->master.size() * sizeof(float));
    return FP_OK;
}

int fp_surrogate_set_params(fp_surrogate *s, const float *src, size_t n) {
    if (!s || !src || n < s->master.size()) return FP_EINVAL;
    memcpy(s->master.data(), src, s->master.size() * sizeof(float));
    return upload_packed(s) == cudaSuccess ? FP_OK : FP_ECUDA;
}

// x: device FP32 [B][H][W][4]; y: device FP32 [B][H-10][W-10][3] (delta U); H, W >= 11.
// Scratch activations are allocated per call (internal use: tests and training).
int fp_surrogate_forward(fp_surrogate *s, const float *x, int32_t B, int32_t H, int32_t W, float *y) {
    if (!s || !x || !y || B < 1 || H < 11 || W < 11) return FP_EINVAL;
    const size_t npix0 = (size_t)B * H * W;
    __nv_bfloat16 *a0 = nullptr, *a1 = nullptr, *a2 = nullptr;
    cudaError_t e = cudaMalloc(&a0, npix0 * kCin0 * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&a1, npix0 * kWidth * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&a2, npix0 * kWidth * sizeof(__nv_bfloat16));
    if (e != cudaSuccess) {
        cudaFree(a0); cudaFree(a1); cudaFree(a2);
        fp_note_error("fp_surrogate_forward: allocation failed");
        return FP_ENOMEM;
    }
    cudaStream_t st = 0;
    pack_input_kernel<<<(unsigned)((npix0 + 255) / 256), 256, 0, st>>>(x, npix0, a0);
    int h = H, w = W;
    e = launch_conv<kCin0, kWidth, false>(s, 0, a0, B, h, w, a1, st);
    h -= 2; w -= 2;
    __nv_bfloat16 *src = a1, *dst = a2;
    for (int l = 1; l < kLayers - 1 && e == cudaSuccess; ++l) {
        e = launch_conv<kWidth, kWidth, false>(s, l, src, B, h, w, dst, st);
        h -= 2; w -= 2;
        std::swap(src, dst);
    }
    if (e == cudaSuccess) e = launch_conv<kWidth, kCout4, true>(s, kLayers - 1, src, B, h, w, y, st);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned herr = 0;
    cudaMemcpy(&herr, s->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(a0); cudaFree(a1); cudaFree(a2);
    if (e != cudaSuccess) {
        fp_note_error(cudaGetErrorString(e));
        return FP_ECUDA;
    }
    if (herr & FP_ERR_TIMEOUT) {
        fp_note_error("fp_surrogate_forward: tensor-core completion wait timed out");
        return FP_ETIMEOUT;
    }
    return FP_OK;
}

}  // extern "C"
