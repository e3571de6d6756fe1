// gc_barrier.cuh -- a grid-wide barrier for cooperative launches (every block
// of the grid resident at once), bounded in time.
//
// Thread 0 of each block reads the barrier generation, counts its block in,
// and either (last block) resets the count and releases the next generation,
// or polls the generation with acquire loads and short sleeps.  A wait that
// exceeds `limit_ns` of %globaltimer sets kErrBarrierTimeout in the control
// block and reports failure, so a kernel whose peers never arrive returns
// with an error status instead of spinning forever.
#pragma once
#include "gc_internal.cuh"

namespace gc {

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Release/acquire fence at GPU scope.  Issued by thread 0 after a block-wide
// barrier it orders the whole block's earlier writes (the pattern of a
// cooperative-groups grid sync); readers of data written by other SMs within
// the same launch load through L2 (ld.global.cg).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// `expected` blocks must arrive (gridDim.x in normal use).  Every thread of
// every block must call it; returns false for the whole block on timeout.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned *gen, int *error, unsigned expected,
                                             unsigned long long limit_ns, int *s_ok) {
    __syncthreads();  // the block's writes before thread 0's release
    if (threadIdx.x == 0) {
        fence_acq_rel_gpu();
        const unsigned g = ld_acquire_gpu(gen);
        int ok = 1;
        if (atomicAdd(count, 1u) == expected - 1) {
            *count = 0u;                 // ordered before the release below
            st_release_gpu(gen, g + 1u);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            while (ld_acquire_gpu(gen) == g) {
                if (globaltimer_ns() - t0 > limit_ns) {
                    atomicOr(error, kErrBarrierTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        *s_ok = ok;
    }
    __syncthreads();  // thread 0's acquire covers the block from here on
    return *s_ok != 0;
}

}  // namespace gc
