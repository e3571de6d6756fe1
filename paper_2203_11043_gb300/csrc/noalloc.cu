// noalloc.cu -- gc_coulomb_field_noalloc: the Eq. 6 field without any device
// allocation, for callers that cannot call cudaMalloc (for example code that
// runs inside a memory pool or allocator it must not re-enter, inside an
// embedding framework that owns all device memory, or where allocation is
// forbidden after start-up).
//
// All scratch -- the control block, the one-event offsets, the position
// shadow and the per-chunk partial sums -- lives in one file-scope device
// array of fixed size.  Every GPU that loads the library holds it until the
// process exits.  Every call shares it and it keeps the last call's contents,
// so calls whose work overlaps on the GPU (different streams, or different
// host threads) race with each other and must be serialised by the caller.
#include <mutex>

#include "gcoreccd.h"
#include "gc_internal.cuh"
#include "gc_launch.h"

namespace gc {
namespace {

constexpr int kMaxN = GC_NOALLOC_MAX_CARRIERS;
constexpr int kChunksAtMaxN = 8;               // j-chunks the partial area holds at n = kMaxN
constexpr size_t kHeader = 4096;               // Ctrl, offsets, item bases, origin, FP16x2 extent
constexpr size_t kShadowBytes = (size_t)kMaxN * 32;            // float4 or double4_32a
constexpr size_t kPartialBytes = (size_t)kChunksAtMaxN * 3 * kMaxN * 8;
constexpr size_t kScratchBytes = kHeader + kShadowBytes + kPartialBytes;
static_assert(sizeof(Ctrl) <= 256, "control block must fit its slot");

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_dev[kMaxDevices] = {};  // device address of g_scratch, per device

// Resets the control block, the single-event bookkeeping and the FP16x2
// extent for one call; the event origin is the first carrier's position.
__global__ void noalloc_setup_kernel(Dev d, const double *__restrict__ xyz, int n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        Ctrl c{};
        c.step = 0;
        c.step_limit = 1;
        c.n_active = n;
        *d.ctrl = c;
        d.ev_off[0][0] = 0;
        d.ev_off[0][1] = n;
        d.ev_origin[0] = xyz[0];
        d.ev_origin[1] = xyz[1];
        d.ev_origin[2] = xyz[2];
        if (d.ev_ext[0]) d.ev_ext[0][0] = 0u;  // FP16x2 form only
    }
}

}  // namespace
}  // namespace gc

using namespace gc;

extern "C" gc_status gc_coulomb_field_noalloc(const double *xyz_dev, int64_t n, double softening_um,
                                              double eps_si_rel, int32_t precision, double *E_dev,
                                              void *cuda_stream) {
    if (n < 0 || n > kMaxN) return GC_ERR_PARAM;
    if (!(softening_um > 0) || !(softening_um < 1e300) || !(eps_si_rel > 0) || !(eps_si_rel < 1e300))
        return GC_ERR_PARAM;
    if (precision < GC_FP64 || precision > GC_FP16X2) return GC_ERR_PARAM;
    if (n > 0 && (!xyz_dev || !E_dev)) return GC_ERR_PARAM;
    int cnt = 0;
    cudaError_t e = cudaGetDeviceCount(&cnt);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cnt == 0) return GC_ERR_NO_DEVICE;
    if (n == 0) return GC_OK;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kMaxDevices) return GC_ERR_PARAM;

    // Once per device, with that device current: the scratch's device address.
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_dev[dev]) {
            void *p = nullptr;
            if ((e = cudaGetSymbolAddress(&p, g_scratch)) != cudaSuccess) return cuda_fail(e);
            if (!p) return GC_ERR_CUDA;
            g_scratch_dev[dev] = p;
        }
        base = g_scratch_dev[dev];
    }
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e);

    unsigned char *b = (unsigned char *)base;
    Dev d{};
    d.ctrl = (Ctrl *)b;
    d.ev_off[0] = d.ev_off[1] = (int *)(b + 256);
    d.item_base = (int *)(b + 264);
    d.ev_origin = (double *)(b + 272);
    if (precision == GC_FP16X2) d.ev_ext[0] = d.ev_ext[1] = (unsigned *)(b + 320);
    d.sh32 = (float4 *)(b + kHeader);
    d.sh64 = (double4_32a *)(b + kHeader);
    d.partial = (double *)(b + kHeader + kShadowBytes);
    d.part_stride = n;
    d.n_total = (int)n;
    d.n_events = 1;
    // Eq. 6 constant K = q / (4 pi eps0 eps_r), in V/cm um^2 (CODATA 2018).
    d.phys.K = 1.602176634e-19 / (4.0 * 3.14159265358979323846 * 8.8541878128e-12 * eps_si_rel) * 1e10;
    d.phys.eps2 = softening_um * softening_um;
    d.phys.coulomb = 1;
    const bool f64 = precision == GC_FP64;
    // the allocating entry point's shape, with j-chunks lengthened if the
    // partial-sum area holds fewer of them
    d.shape = field_shape(precision, sms, n, (long long)(kPartialBytes / (24 * (size_t)n)));

    cudaStream_t st = (cudaStream_t)cuda_stream;
    noalloc_setup_kernel<<<1, 32, 0, st>>>(d, xyz_dev, (int)n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_field_prepare(d, xyz_dev, (int)n, f64, st);
    if (e == cudaSuccess) e = launch_build_items(d, st);
    if (e == cudaSuccess) e = launch_pair(d, precision, 0, st);
    if (e == cudaSuccess) e = launch_field_finish(d, (int)n, E_dev, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? GC_OK : cuda_fail(e);
}
