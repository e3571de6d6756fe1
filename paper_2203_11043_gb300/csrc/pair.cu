// pair.cu -- instantiation and launch of the Eq. 6 pair kernels of one time
// step (templates in gc_pair.cuh).
#include "gc_pair.cuh"
#include "gc_launch.h"

namespace gc {

// ---------------------------------------------------------------------------
// Host-side launch table.
typedef void (*PairKernel)(Dev);

template <bool TF>
static PairKernel fp32_kernel(int R, bool kahan, bool newton, bool h16, int V) {
#define GC_PICK(RR)                                                                                \
    if (R == RR) {                                                                                 \
        if (h16) return pair_fp32_kernel<RR, true, false, true, TF, false>; /* no Newton step */  \
        if (newton) return kahan ? pair_fp32_kernel<RR, true, true, false, TF, false>             \
                                 : pair_fp32_kernel<RR, false, true, false, TF, false>;           \
        if (TF || V == 0) return kahan ? pair_fp32_kernel<RR, true, false, false, TF, false>      \
                                       : pair_fp32_kernel<RR, false, false, false, TF, false>;    \
        if (V == 1) return kahan ? pair_fp32_kernel<RR, true, false, false, false, false, 1>      \
                                 : pair_fp32_kernel<RR, false, false, false, false, false, 1>;    \
        if (V == 2 && RR <= 4) return kahan ? pair_fp32_kernel<RR, true, false, false, false, false, 2> \
                                            : pair_fp32_kernel<RR, false, false, false, false, false, 2>; \
    }
    GC_PICK(2)
    GC_PICK(4)
    GC_PICK(8)
#undef GC_PICK
    return nullptr;
}

// precision: 0 = FP64 form, 1 = FP32, 2 = FP32 + Kahan, 3 = FP16x2.  V: the
// autotuner variant (FP32 and FP32 + Kahan in the event frame without the
// Newton step; other forms have variant 0 only).
const void *pair_kernel_ptr(int precision, int R, int newton, int tile_frames, int V) {
    if (precision == 0) return V == 0 ? (const void *)pair_fp64_kernel<false> : nullptr;
    if (precision >= 1 && precision <= 3) {
        const bool kahan = precision >= 2, h16 = precision == 3;
        if (V != 0 && (h16 || newton || tile_frames)) return nullptr;
        return tile_frames ? (const void *)fp32_kernel<true>(R, kahan, newton != 0, h16, V)
                           : (const void *)fp32_kernel<false>(R, kahan, newton != 0, h16, V);
    }
    return nullptr;
}

int pair_kernel_occupancy(int precision, int R, int newton, int tile_frames, int V) {
    const void *k = pair_kernel_ptr(precision, R, newton, tile_frames, V);
    if (!k) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kPairThreads, 0) != cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t launch_pair(const Dev &d, int precision, int newton, cudaStream_t st) {
    const void *k = pair_kernel_ptr(precision, d.shape.R, newton, d.tile_frames, d.shape.V);
    if (!k) return cudaErrorInvalidValue;
    ((PairKernel)k)<<<d.shape.n_blocks, kPairThreads, 0, st>>>(d);
    return cudaGetLastError();
}

}  // namespace gc
