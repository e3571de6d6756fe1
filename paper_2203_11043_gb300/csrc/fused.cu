// fused.cu -- the fused small-workload step (Fig. 2 loop body while few holes
// are active): one persistent pair kernel that also integrates each i-tile
// as soon as its last j-chunk is summed (templates in gc_pair.cuh), followed
// by the one-block small_tail kernel of step.cu (compaction and bookkeeping).
// Two launches per step instead of four: small steps are bound by launch
// latency, not by arithmetic.  The arithmetic is the same as in the unfused
// kernels (same items, same partial sums, same per-carrier code), so both
// paths give the same bits.
#include "gc_pair.cuh"
#include "gc_launch.h"

namespace gc {

typedef void (*PairKernel)(Dev);

const void *fused_pair_kernel_ptr(int precision, int R) {
    if (precision == 0) return (const void *)pair_fp64_kernel<true>;
#define GC_PICK(RR)                                                                      \
    if (R == RR) {                                                                       \
        if (precision == 1) return (const void *)pair_fp32_kernel<RR, false, false, false, false, true>; \
        if (precision == 2) return (const void *)pair_fp32_kernel<RR, true, false, false, false, true>;  \
        if (precision == 3) return (const void *)pair_fp32_kernel<RR, true, false, true, false, true>;   \
    }
    GC_PICK(2)
    GC_PICK(4)
    GC_PICK(8)
#undef GC_PICK
    return nullptr;
}

int fused_pair_occupancy(int precision, int R) {
    const void *k = fused_pair_kernel_ptr(precision, R);
    if (!k) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kPairThreads, 0) != cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t launch_fused_pair(const Dev &d, int precision, int grid, cudaStream_t st) {
    const void *k = fused_pair_kernel_ptr(precision, d.shape.R);
    if (!k || grid < 1) return cudaErrorInvalidValue;
    ((PairKernel)k)<<<grid, kPairThreads, 0, st>>>(d);
    return cudaGetLastError();
}

}  // namespace gc
