// grid_sync.cuh -- the bounded grid barrier of the persistent kernels (one
// simulation, or a batch of them): every CTA resident (cooperative launch).
#pragma once
#include "fp_common.cuh"

namespace fpdev {

// Grid barrier on one word: every CTA adds 1 except CTA 0, which adds
// 2^31 - (gridDim.x - 1), so the word's top bit flips exactly when the last
// CTA has arrived (and the low bits are back to zero); each CTA spins until
// the top bit differs from the value it saw on arrival.  The spin is bounded
// by S.barrier_polls polls; past 2^10 polls it also watches the error word, so
// that CTAs leave soon after another CTA failed; on timeout the error flag is
// set and the CTA returns (those still waiting time out in turn).  No
// asynchronous copy is in flight at a barrier: the kernel makes none.
__device__ __forceinline__ bool grid_sync(unsigned *bar, const FpSim &S) {
    __shared__ int s_fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(bar, add);
        volatile unsigned *vb = bar;
        int fail = 0;
        const int limit = S.barrier_polls;
        for (int it = 0; ((*vb ^ old) & 0x80000000u) == 0u; ++it) {
            if (it >= limit) {
                fail = 1;
                break;
            }
            if (it >= (1 << 10)) {
                if ((*(volatile unsigned *)&S.cnt->err & FP_ERR_TIMEOUT) != 0u) {
                    fail = 1;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();  // the other CTAs' writes of the phase are seen by this CTA's loads after it
        if (fail) fp_set_err(S, FP_ERR_TIMEOUT);
        s_fail = fail;
    }
    __syncthreads();
    return !s_fail;
}

}  // namespace fpdev
