// noalloc.cu -- water volume of a caller's depth grid without any device allocation.
//
// Same quantity as the mass read of a simulation (sum of h dx^2 in FP64), for a
// caller who owns the depth grid and cannot let this library allocate device
// memory.  The scratch lives in one file-scope device array that every GPU
// which loads the library holds until the process exits:
//   g_volume_scratch[0]        -- completion counter of the CTAs of one call
//   g_volume_scratch[32 + r]   -- FP64 sum of row r (r < FP_NOALLOC_MAX_ROWS)
// Host code never uses the array's name as an address: the first call on each
// device looks the device address up with cudaGetSymbolAddress and passes it to
// the kernel.
#include <mutex>

#include "floodped.h"
#include "fp_common.cuh"

namespace {

constexpr int kRowBase = 32;  // first row slot (keeps rows 256-byte aligned)
static __device__ __align__(256) double g_volume_scratch[kRowBase + FP_NOALLOC_MAX_ROWS];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// One CTA per row (grid-stride over rows): row sums in FP64 in a fixed tree
// order, then the last CTA to finish adds the rows (thread t rows t, t + 256,
// ... in index order, then the same fixed tree), writes the volume and
// re-arms the counter for the next call.
__global__ void __launch_bounds__(256) volume_rows_kernel(const float *__restrict__ h, int nx, int ny,
                                                          long long pitch, double dx2, double *out,
                                                          double *scratch) {
    __shared__ double red[8];
    __shared__ bool last;
    for (int row = blockIdx.x; row < ny; row += gridDim.x) {
        double acc = 0.0;
        const float *hr = h + (size_t)row * (size_t)pitch;
        for (int i = threadIdx.x; i < nx; i += blockDim.x) acc += (double)hr[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
            scratch[kRowBase + row] = s;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long *counter = reinterpret_cast<unsigned long long *>(scratch);
        last = atomicAdd(counter, 1ull) == (unsigned long long)(gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
        __threadfence();
        const volatile double *rows = scratch + kRowBase;
        double acc = 0.0;
        for (int r = threadIdx.x; r < ny; r += blockDim.x) acc += rows[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
            *out = s * dx2;
            *reinterpret_cast<unsigned long long *>(scratch) = 0ull;
            __threadfence();
        }
    }
}

}  // namespace

extern "C" int fp_water_volume_noalloc(const float *h, int32_t nx, int32_t ny, int64_t row_pitch, float dx,
                                       double *out, void *cuda_stream) {
    if (!h || !out) {
        fp_note_error("fp_water_volume_noalloc: null depth grid or output");
        return FP_EINVAL;
    }
    if (nx < 1 || ny < 1 || row_pitch < nx || !(dx > 0.0f)) {
        fp_note_error("fp_water_volume_noalloc: need nx, ny >= 1, row_pitch >= nx and dx > 0");
        return FP_EINVAL;
    }
    if (ny > FP_NOALLOC_MAX_ROWS) {
        fp_note_error("fp_water_volume_noalloc: ny exceeds FP_NOALLOC_MAX_ROWS (65536), the size of its "
                      "fixed device scratch");
        return FP_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        fp_note_error("fp_water_volume_noalloc: no usable current CUDA device");
        return FP_ECUDA;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_volume_scratch);
            if (e != cudaSuccess || !p) {
                fp_note_error("fp_water_volume_noalloc: cudaGetSymbolAddress of the scratch array failed");
                return FP_ECUDA;
            }
            g_scratch_ptr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    const int grid = ny < 148 * 8 ? ny : 148 * 8;
    const double dx2 = (double)dx * (double)dx;
    volume_rows_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(h, nx, ny, (long long)row_pitch,
                                                                                 dx2, out, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        fp_note_error("fp_water_volume_noalloc: kernel launch failed");
        return FP_ECUDA;
    }
    return FP_OK;
}
