// api.cu -- the C ABI of libgcoreccd (declared in include/gcoreccd.h).
//
// Host orchestration only: parameter validation, the load-time layout
// (events ordered largest first so that pair work items come out in
// longest-processing-time order), the step-0 pass, the pair-kernel
// autotuner, CUDA-graph capture of the step loop, and copies in and out.
// Every step of the transport itself runs in the kernels of pair.cu and
// step.cu.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gcoreccd.h"
#include "gc_internal.cuh"
#include "gc_launch.h"
#include "gc_barrier.cuh"

using namespace gc;

namespace {
thread_local char g_cuda_err[256] = "";
}  // namespace

namespace gc {
gc_status cuda_fail(cudaError_t e) {
    std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e),
                  cudaGetErrorString(e));
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return GC_ERR_NO_DEVICE;
    if (e == cudaErrorMemoryAllocation) return GC_ERR_ALLOC;
    return GC_ERR_CUDA;
}
}  // namespace gc

namespace {

#define GC_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_);   \
    } while (0)

// One FP32 / FP32 + Kahan event of at most this many active holes takes the
// grid-resident kernel by default.  Measured per step to completion (clouds at
// 300 um, FP32 + Kahan): 256 holes 3.2 us there, 4.7 us in the cluster kernel,
// 7.9 us in the persistent kernel; 1573 holes 5.5 us against 15.6 and 11.9 us;
// 4096 holes 12.8 us against 26.5 us in the persistent kernel.
constexpr int kResidentPathMax = 4096;

// Longest a device-side wait (a grid barrier of the persistent kernel, a
// grid-resident kernel's wait for step-tagged words) may take before the
// kernel gives up with an error status.
constexpr double kDeviceWaitLimitS = 1.0;

// CODATA 2018 exact SI values and eps0.
constexpr double kQ = 1.602176634e-19;
constexpr double kKB = 1.380649e-23;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;

bool is_finite(double v) { return std::isfinite(v); }

gc_status validate(const gc_params *p) {
    if (!p || p->abi_version != GC_ABI_VERSION) return GC_ERR_PARAM;
    if (p->precision < GC_FP64 || p->precision > GC_FP16X2) return GC_ERR_PARAM;
    if (p->precision == GC_FP16X2 && p->newton) return GC_ERR_PARAM;
    const double v[] = {p->thickness_um, p->z_well_um, p->a1_V_cm_um, p->a2_V_cm, p->T_K,
                        p->eps_si_rel, p->softening_um, p->dt_s, p->pixel_um, p->stored_z_um};
    for (double x : v)
        if (!is_finite(x)) return GC_ERR_PARAM;
    if (!(p->thickness_um > 0) || !(p->T_K > 0) || !(p->dt_s > 0) || !(p->pixel_um > 0))
        return GC_ERR_PARAM;
    if (p->z_well_um >= p->thickness_um) return GC_ERR_PARAM;
    if (p->max_steps < 0 || p->max_steps > INT_MAX) return GC_ERR_PARAM;
    if (p->img_w <= 0 || p->img_h <= 0 || (int64_t)p->img_w * p->img_h > (1 << 26))
        return GC_ERR_PARAM;
    if ((p->coulomb || p->stored_charge) && (!(p->softening_um > 0) || !(p->eps_si_rel > 0)))
        return GC_ERR_PARAM;
    if (p->graph_steps < 0 || p->graph_steps > 4096) return GC_ERR_PARAM;
    if (p->jchunk < 0) return GC_ERR_PARAM;
    if ((p->coulomb | p->diffusion | p->reflect_back | p->autotune | p->newton | p->timing |
         p->stored_charge | p->tile_frames) & ~1)
        return GC_ERR_PARAM;
    if (p->fuse_small < 0 || p->fuse_small > 5) return GC_ERR_PARAM;
    if (p->resident_ctas < 0) return GC_ERR_PARAM;
    if (p->pair_R != 0 && p->pair_R != 2 && p->pair_R != 4 && p->pair_R != 8) return GC_ERR_PARAM;
    return GC_OK;
}

Phys make_phys(const gc_params &p) {
    Phys ph{};
    ph.a1 = p.a1_V_cm_um;
    ph.a2 = p.a2_V_cm;
    ph.thickness = p.thickness_um;
    ph.z_well = p.z_well_um;
    ph.dt = p.dt_s;
    // Eq. 6: K = q / (4 pi eps0 eps_r) [V m]; 1/um^2 = 1e12/m^2 and 1 V/m = 1e-2 V/cm.
    ph.K = kQ / (4.0 * kPi * kEps0 * p.eps_si_rel) * 1e10;
    ph.eps2 = p.softening_um * p.softening_um;
    // Eq. 2 constants.
    ph.mu0 = 1.31e8 * std::pow(p.T_K, -2.2);
    ph.inv_Ec = 1.0 / (1.24 * std::pow(p.T_K, 1.68));
    ph.beta = 0.46 * std::pow(p.T_K, 0.17);
    ph.inv_beta = 1.0 / ph.beta;
    ph.Vth = kKB * p.T_K / kQ;  // Eq. 4
    ph.pixel = p.pixel_um;
    ph.img_w = p.img_w;
    ph.img_h = p.img_h;
    ph.coulomb = p.coulomb;
    ph.diffusion = p.diffusion;
    ph.reflect = p.reflect_back;
    ph.stored = p.stored_charge;
    ph.stored_z = p.stored_z_um;
    ph.f_a1 = (float)ph.a1;
    ph.f_dt = (float)ph.dt;
    ph.f_K = (float)ph.K;
    ph.f_mu0 = (float)ph.mu0;
    ph.f_inv_Ec = (float)ph.inv_Ec;
    ph.f_beta = (float)ph.beta;
    ph.f_inv_beta = (float)ph.inv_beta;
    ph.f_Vth = (float)ph.Vth;
    return ph;
}

struct DevAllocs {
    std::vector<void *> ptrs;
    cudaError_t alloc(void **p, size_t bytes) {
        *p = nullptr;
        cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release() {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

int round_up(long long v, int m) { return (int)((v + m - 1) / m * m); }

// Spread the low 21 bits of v so that bit k lands on bit 3k (for a 3-D
// Morton / Z-order key): each step doubles the gap between bit groups.
uint64_t spread_bits3(uint64_t v) {
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x001F00000000FFFFull;
    v = (v | (v << 16)) & 0x001F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Reorder ids[0..n) (one event) by the Morton key of their positions on a
// 2^21 grid over the event's bounding box (ties by id), so that consecutive
// slots are spatial neighbours.
void morton_order(const double *xyz, int *ids, int n) {
    if (n < 2) return;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int k = 0; k < n; ++k)
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], xyz[3LL * ids[k] + c]);
            hi[c] = std::max(hi[c], xyz[3LL * ids[k] + c]);
        }
    const double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-30});
    const double scale = 2097151.0 / ext;
    std::vector<std::pair<uint64_t, int>> key(n);
    for (int k = 0; k < n; ++k) {
        uint64_t m = 0;
        for (int c = 0; c < 3; ++c) {
            const double q = std::min(2097151.0, std::max(0.0, (xyz[3LL * ids[k] + c] - lo[c]) * scale));
            m |= spread_bits3((uint64_t)q) << c;
        }
        key[k] = {m, ids[k]};
    }
    std::sort(key.begin(), key.end());
    for (int k = 0; k < n; ++k) ids[k] = key[k].second;
}

}  // namespace

// j-chunk length: one chunk per event when the i-tiles alone give every
// resident block >= 32 items; otherwise split j so that they do (at most 32
// chunks), keeping dynamic-scheduling tail loss near 1/64 of a step.
int gc::choose_jchunk(const std::vector<long long> &sizes, const PairShape &sh, int user, int gran) {
    long long n_max = 1;
    for (long long n : sizes) n_max = std::max(n_max, n);
    if (user > 0) return round_up(user, gran);
    long long tiles = 0;
    for (long long n : sizes)
        if (n > 0) {
            const int it = itile_for(sh.R, lanes_for(sh, (int)n));
            tiles += (n + it - 1) / it;
        }
    const long long want = 32LL * std::max(sh.n_blocks, 1);
    long long js = tiles >= want ? 1 : std::min<long long>(32, (want + tiles - 1) / std::max(tiles, 1LL));
    return round_up((n_max + js - 1) / js, gran);
}

struct gc_sim {
    gc_params p;
    Phys phys;
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool loaded = false;
    int64_t n = 0, E = 0;
    std::vector<int64_t> user_off;   // caller's event offsets
    DevAllocs mem;
    Dev dev{};
    Ctrl *h_ctrl = nullptr;          // pinned mirror of the device control block
    long long *h_limit = nullptr;    // pinned staging for step_limit, loop_last and stop_below
    cudaGraphExec_t graph = nullptr;
    bool graph_loops = false;        // the graph holds a device-side WHILE loop over K-step passes
    // fused small-workload path: two launches per step while at most kFusedMax
    // holes are active (its own graph; the unfused graph hands over to it)
    bool fused_ok = false;
    int fused_grid = 0;
    int fused_ran = 0;               // small-workload path of the last gc_run (gc_stats.fused_path)
    bool se_ok = false;              // the persistent single-event kernel applies
    bool cluster_ok = false;         // the cluster-resident kernel may apply (FP32 forms, small event)
    bool resident_ok = false;        // the grid-resident kernel may apply (FP32 forms, one event)
    int se_grid = 0;
    unsigned *h_probe = nullptr;     // pinned: items_total, work_counter of an autotuner probe
    int device_error = 0;            // Ctrl::error bits seen after the last load or run
    int inject = 0;                  // GC_DEBUG builds: fault to plant at the next load (gc_debug_inject)
    double tune_ms = 0.0;            // autotuner: host time spent at the last load
    int tune_candidates = 0;         //   shapes timed
    int tune_cached = 0;             //   1: the shape came from the in-process cache
    cudaGraphExec_t graph_small = nullptr;
    bool small_loops = false;
    int integ_grid = 1;
    int launches_per_step = 0;
    long long part_cap_chunks = 1;   // j-chunks the partial buffer can hold
    // timing: before the pair kernel, after it, after integrate, after compact
    std::vector<int> load_act;       // the active list at load (event order, in-event order)
    std::vector<int> load_off;       // its event offsets
    std::vector<cudaEvent_t> ev_a, ev_b, ev_c, ev_d;
    double pair_ms = 0.0, integ_ms = 0.0, compact_ms = 0.0;
    long long pair_launches = 0, timed_steps = 0;
};

namespace {

bool fp64_mode(const gc_sim *s) { return s->p.precision == GC_FP64; }

// The status of a failed device-side check (Ctrl::error bits); the state of
// the simulation is undefined afterwards.
gc_status device_error_status(int bits) {
    return (bits & kErrBarrierTimeout) ? GC_ERR_DEVICE_TIMEOUT : GC_ERR_DEVICE_CHECK;
}
// Timing mode launches eagerly: events recorded by captured graph nodes
// cannot be used with cudaEventElapsedTime.
bool use_graph(const gc_sim *s) { return s->p.graph_steps > 0 && !s->p.timing; }

void free_state(gc_sim *s) {
    for (cudaGraphExec_t *g : {&s->graph, &s->graph_small})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
    s->fused_ok = false;
    s->fused_ran = 0;
    s->se_ok = false;
    s->cluster_ok = false;
    s->resident_ok = false;
    for (auto *v : {&s->ev_a, &s->ev_b, &s->ev_c, &s->ev_d}) {
        for (cudaEvent_t e : *v) cudaEventDestroy(e);
        v->clear();
    }
    s->pair_ms = s->integ_ms = s->compact_ms = 0.0;
    s->pair_launches = s->timed_steps = 0;
    s->mem.release();
    s->loaded = false;
    s->dev = Dev{};
}

// One time step; k indexes the step inside a captured graph (timing events).
// fused: the two-launch small-workload step.
gc_status enqueue_step(gc_sim *s, int k, bool fused) {
    const bool f64 = fp64_mode(s);
    if (fused) {
        GC_CUDA(launch_fused_pair(s->dev, s->p.precision, s->fused_grid, s->stream));
        GC_CUDA(launch_small_tail(s->dev, f64, s->stream));
        return GC_OK;
    }
    const bool timed = s->p.timing && k < (int)s->ev_a.size();
    if (timed) GC_CUDA(cudaEventRecord(s->ev_a[k], s->stream));
    if (s->phys.coulomb) GC_CUDA(launch_pair(s->dev, s->p.precision, s->p.newton, s->stream));
    if (timed) GC_CUDA(cudaEventRecord(s->ev_b[k], s->stream));
    if (s->phys.stored) GC_CUDA(launch_occupied_pixels(s->dev, s->stream));
    GC_CUDA(launch_integrate(s->dev, f64, false, s->integ_grid, s->stream));
    if (timed) GC_CUDA(cudaEventRecord(s->ev_c[k], s->stream));
    GC_CUDA(launch_compact(s->dev, f64, s->integ_grid, s->stream));
    if (timed) GC_CUDA(cudaEventRecord(s->ev_d[k], s->stream));
    GC_CUDA(launch_finalize(s->dev, false, s->stream));
    if (s->dev.tile_frames) GC_CUDA(launch_shadow(s->dev, s->sm_count, s->stream));
    return GC_OK;
}

gc_status read_ctrl(gc_sim *s) {
    GC_CUDA(cudaMemcpyAsync(s->h_ctrl, s->dev.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream));
    GC_CUDA(cudaStreamSynchronize(s->stream));
    return GC_OK;
}

gc_status set_limit(gc_sim *s, long long limit) {
    s->h_limit[0] = limit;
    s->h_limit[1] = -1;  // loop_last: the next device-side loop starts afresh
    s->h_limit[2] = s->resident_ok ? kResidentPathMax : 0;  // the other paths hand over to it there
    GC_CUDA(cudaMemcpyAsync(&s->dev.ctrl->step_limit, s->h_limit, 3 * sizeof(long long),
                            cudaMemcpyHostToDevice, s->stream));
    GC_CUDA(cudaStreamSynchronize(s->stream));
    return GC_OK;
}

// A graph of K time steps.  Preferred form: one WHILE conditional node whose
// body is K steps plus the loop-condition kernel, so a whole gc_run is one
// graph launch with no host round trip; otherwise a plain graph of K steps
// that gc_run launches repeatedly.
gc_status capture_plain_graph(gc_sim *s, bool fused, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    GC_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    gc_status st = GC_OK;
    for (int k = 0; k < s->p.graph_steps && st == GC_OK; ++k) st = enqueue_step(s, k, fused);
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (st != GC_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e);
    return GC_OK;
}

// The unfused loop stops once the fused graph can take over.
bool capture_loop_graph(gc_sim *s, bool fused, cudaGraphExec_t *outg) {
    cudaGraphExec_t &graph = *outg;
    cudaGraph_t g = nullptr, body = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    bool ok = false;
    do {
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) break;
        body = np.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(s->stream, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            break;
        gc_status st = GC_OK;
        for (int k = 0; k < s->p.graph_steps && st == GC_OK; ++k) st = enqueue_step(s, k, fused);
        const int switch_below = (!fused && s->fused_ok) ? kFusedMax : 0;
        const cudaError_t le =
            st == GC_OK ? launch_loop_cond(s->dev, h, switch_below, s->stream) : cudaErrorUnknown;
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(s->stream, &out);
        if (st != GC_OK || le != cudaSuccess || ee != cudaSuccess) break;
        if (cudaGraphInstantiate(&graph, g, 0) != cudaSuccess) break;
        ok = true;
    } while (0);
    cudaGraphDestroy(g);
    if (!ok) {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        cudaGetLastError();  // clear a failed attempt; the plain graph is used instead
    }
    return ok;
}

// The graphs a gc_run launches: the unfused step loop (unless every step is
// small enough for the fused path) and the fused one (when available).
gc_status capture_graph(gc_sim *s) {
    for (cudaGraphExec_t *g : {&s->graph, &s->graph_small})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
    s->graph_loops = s->small_loops = false;
    if (!use_graph(s)) return GC_OK;
    if (!s->fused_ok || s->h_ctrl->n_active > kFusedMax) {
        if (capture_loop_graph(s, false, &s->graph)) {
            s->graph_loops = true;
        } else {
            gc_status r = capture_plain_graph(s, false, &s->graph);
            if (r != GC_OK) return r;
        }
    }
    if (s->fused_ok) {
        if (capture_loop_graph(s, true, &s->graph_small)) {
            s->small_loops = true;
        } else {
            gc_status r = capture_plain_graph(s, true, &s->graph_small);
            if (r != GC_OK) return r;
        }
    }
    return GC_OK;
}

// Shapes of the pair kernels.  FP64 form: one carrier per thread, 16 lanes
// per carrier for small events, j-chunks of kTileJ64 granularity chosen like
// the FP32 ones, lengthened if the partial buffer holds fewer chunks.
PairShape fp64_shape(int sm_count, const std::vector<long long> &sizes, int user_jchunk, long long cap) {
    PairShape sh{};
    sh.R = 1;
    sh.small_n = kSmallEvent;
    sh.small_lanes = 16;
    sh.n_blocks = sm_count * std::max(1, pair_kernel_occupancy(GC_FP64, 1, 0, 0));
    sh.jchunk = choose_jchunk(sizes, sh, user_jchunk, kTileJ64);
    long long n_max = 1;
    for (long long n : sizes) n_max = std::max(n_max, n);
    if (cap > 0 && (n_max + sh.jchunk - 1) / sh.jchunk > cap)
        sh.jchunk = round_up((n_max + cap - 1) / cap, kTileJ64);
    return sh;
}
PairShape fp32_shape(int R, int sm_count, int precision, int newton, int tile_frames) {
    PairShape sh{};
    sh.R = R;
    sh.small_n = kSmallEvent;
    sh.small_lanes = 4;
    sh.n_blocks = sm_count * std::max(1, pair_kernel_occupancy(precision, R, newton, tile_frames));
    return sh;
}

}  // namespace

// Shape of the standalone Eq. 6 evaluation of one event of n carriers; with
// max_chunks > 0 the j-chunks are lengthened so that at most that many fit.
PairShape gc::field_shape(int precision, int sm_count, long long n, long long max_chunks) {
    const std::vector<long long> sizes{n};
    if (precision == GC_FP64) return fp64_shape(sm_count, sizes, 0, max_chunks);
    PairShape sh = fp32_shape(4, sm_count, precision, 0, 0);
    sh.jchunk = choose_jchunk(sizes, sh, 0, kTileJ);
    if (max_chunks > 0 && (n + sh.jchunk - 1) / sh.jchunk > max_chunks)
        sh.jchunk = round_up((n + max_chunks - 1) / max_chunks, kTileJ);
    return sh;
}

namespace {

// ---- autotuner ----------------------------------------------------------------
// Knobs of the FP32 pair kernel: R (carriers per thread), the kernel variant V
// (loads in flight, register budget), resident blocks per SM, the j-chunk
// target (work items per resident block) and the 4-lane threshold.  R, V and
// the blocks per SM do not change any result; the j-chunk and the threshold
// change the order of the FP32 partial sums (within the same error bound).
struct TuneKnobs {
    int R = 4, V = 0, bps = 0, small_n = kSmallEvent, target = 32;
};

struct TuneResult {
    TuneKnobs k;
    bool valid = false;
};

std::mutex g_tune_mutex;
std::map<std::string, TuneKnobs> g_tune_cache;  // in-process: device, form and workload shape -> knobs

// Cache key: device, form, user overrides and the workload's event-size
// histogram in powers of two (event count, largest event, sum of n^2, events
// below each lane threshold candidate).
std::string tune_key(const gc_sim *s, const std::vector<long long> &sizes) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, s->device);
    long long n_max = 1, ev = 0, small1 = 0, small2 = 0, small4 = 0;
    double pairs = 0.0;
    for (long long n : sizes) {
        if (n <= 0) continue;
        ++ev;
        n_max = std::max(n_max, n);
        pairs += (double)n * (double)n;
        small1 += n < 1024;
        small2 += n < 2048;
        small4 += n < 4096;
    }
    auto lg = [](double v) { return v > 0 ? (int)std::floor(std::log2(v)) : -1; };
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s|%d|p%d|n%d|t%d|R%d|j%d|E%d|N%d|P%d|s%d.%d.%d", prop.name,
                  prop.multiProcessorCount, s->p.precision, s->p.newton, s->dev.tile_frames, s->p.pair_R,
                  s->p.jchunk, lg((double)ev), lg((double)n_max), lg(pairs), lg((double)small1),
                  lg((double)small2), lg((double)small4));
    return buf;
}

// The pair shape of a set of knobs; n_blocks = 0 when the kernel is not built
// or cannot hold that many blocks per SM.
PairShape shape_of(const gc_sim *s, const std::vector<long long> &sizes, const TuneKnobs &k) {
    PairShape sh{};
    sh.R = k.R;
    sh.V = k.V;
    sh.small_n = k.small_n;
    sh.small_lanes = 4;
    const int occ = pair_kernel_occupancy(s->p.precision, k.R, s->p.newton, s->dev.tile_frames, k.V);
    const int bps = k.bps > 0 ? k.bps : occ;
    sh.n_blocks = (occ > 0 && bps <= occ) ? s->sm_count * bps : 0;
    PairShape ref = sh;
    ref.n_blocks = std::max(1, std::max(1, sh.n_blocks) * k.target / 32);  // items per block = target
    sh.jchunk = choose_jchunk(sizes, ref, s->p.jchunk, kTileJ);
    return sh;
}

// Work items of shape sh for the active event sizes (internal event order),
// and the pair terms of items [a, b).
long long items_of(const PairShape &sh, const std::vector<int> &act_sizes) {
    long long t = 0;
    for (int n : act_sizes)
        if (n > 0) t += (long long)ceil_div(n, itile_for(sh.R, lanes_for(sh, n))) * ceil_div(n, sh.jchunk);
    return t;
}
double pairs_of_items(const PairShape &sh, const std::vector<int> &act_sizes, long long a, long long b) {
    double pairs = 0.0;
    long long base = 0;
    for (int n : act_sizes) {
        if (n <= 0) continue;
        const int itile = itile_for(sh.R, lanes_for(sh, n));
        const int js = ceil_div(n, sh.jchunk);
        const long long cnt = (long long)ceil_div(n, itile) * js;
        for (long long it = std::max(a, base); it < std::min(b, base + cnt); ++it) {
            const long long local = it - base;
            const int ti = (int)(local / js), jc = (int)(local % js);
            pairs += (double)std::min(itile, n - ti * itile) * (double)std::min(sh.jchunk, n - jc * sh.jchunk);
        }
        base += cnt;
        if (base >= b) break;
    }
    return pairs;
}

// Pair terms per second of shape sh, timed on up to three windows of its work
// items (near the start, the middle and the end of the item range, so that
// large and small events are both sampled); 0 if the shape is not usable.
gc_status time_shape(gc_sim *s, const PairShape &sh, const std::vector<int> &act_sizes, cudaEvent_t ea,
                     cudaEvent_t eb, double *rate) {
    *rate = 0.0;
    if (sh.n_blocks <= 0) return GC_OK;
    long long n_max = 1;
    for (int n : act_sizes) n_max = std::max<long long>(n_max, n);
    if ((n_max + sh.jchunk - 1) / sh.jchunk > s->part_cap_chunks) return GC_OK;
    const long long items = items_of(sh, act_sizes);
    if (items <= 0) return GC_OK;
    const long long K = std::min<long long>(items, 2LL * sh.n_blocks);  // two waves per window
    double total_pairs = 0.0;
    for (int n : act_sizes) total_pairs += (double)n * (double)n;
    std::vector<long long> starts;
    // whole launches while they are short (~30 ms): they include the tail of
    // a launch and the real mix of event sizes; sampled windows beyond that
    if (items <= 3 * K || total_pairs < 1e11) starts = {0};
    else if (act_sizes.size() == 1) starts = {(items - K) / 2};  // one event: uniform items
    else for (double f : {0.05, 0.5, 0.9}) starts.push_back(std::min(items - K, (long long)(f * items)));
    const long long len = starts.size() == 1 && starts[0] == 0 ? items : K;
    s->dev.shape = sh;
    GC_CUDA(launch_build_items(s->dev, s->stream));
    double pairs = 0.0, secs = 0.0;
    for (long long st : starts) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up; short windows are repeated
            if (rep >= 2 && best > 2.0f) break;
            s->h_probe[0] = (unsigned)(st + len);  // items_total, then work_counter
            s->h_probe[1] = (unsigned)st;
            GC_CUDA(cudaMemcpyAsync(&s->dev.ctrl->items_total, s->h_probe, 2 * sizeof(unsigned),
                                    cudaMemcpyHostToDevice, s->stream));
            GC_CUDA(cudaEventRecord(ea, s->stream));
            GC_CUDA(launch_pair(s->dev, s->p.precision, s->p.newton, s->stream));
            GC_CUDA(cudaEventRecord(eb, s->stream));
            GC_CUDA(cudaEventSynchronize(eb));
            float ms = 0.f;
            GC_CUDA(cudaEventElapsedTime(&ms, ea, eb));
            if (rep > 0) best = std::min(best, ms);
        }
        pairs += pairs_of_items(sh, act_sizes, st, st + len);
        secs += best * 1e-3;
    }
    *rate = secs > 0 ? pairs / secs : 0.0;
    ++s->tune_candidates;
    return GC_OK;
}

// Pick the FP32 pair kernel's knobs.  autotune = 0: the default knobs (R = 4
// or pair_R).  autotune = 1: the cached choice for this device, form and
// workload histogram, else a staged search timed on the loaded carriers:
// R x V, then blocks per SM, then the j-chunk target, then (when some events
// lie between 1024 and 4096 holes) the 4-lane threshold.
gc_status choose_shape(gc_sim *s, const std::vector<long long> &sizes) {
    s->tune_ms = 0.0;
    s->tune_candidates = 0;
    s->tune_cached = 0;
    if (fp64_mode(s)) {
        s->dev.shape = fp64_shape(s->sm_count, sizes, s->p.jchunk, s->part_cap_chunks);
        GC_CUDA(launch_build_items(s->dev, s->stream));
        return GC_OK;
    }
    long long n_max = 1;
    for (long long n : sizes) n_max = std::max(n_max, n);
    TuneKnobs def;
    if (s->p.pair_R) def.R = s->p.pair_R;
    // one FP32 event small enough for the grid-resident kernel runs every step
    // there, and that kernel does not use the pair kernel's shape: no search
    const bool resident_only = s->resident_ok && s->n <= kResidentPathMax;
    const bool tune = s->p.autotune && s->phys.coulomb && s->n > 0 && !resident_only;
    auto fits = [&](const PairShape &sh) {
        return sh.n_blocks > 0 && (n_max + sh.jchunk - 1) / sh.jchunk <= s->part_cap_chunks;
    };
    TuneKnobs best = def;
    if (!fits(shape_of(s, sizes, best)))  // the default does not fit the partial buffer: try the others
        for (int R : {2, 4, 8}) {
            TuneKnobs k = def;
            k.R = s->p.pair_R ? s->p.pair_R : R;
            if (fits(shape_of(s, sizes, k))) {
                best = k;
                break;
            }
        }
    if (tune) {
        const std::string key = tune_key(s, sizes);
        bool hit = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                best = it->second;
                hit = true;
            }
        }
        if (hit && fits(shape_of(s, sizes, best))) {
            s->tune_cached = 1;
        } else {
            const auto t0 = std::chrono::steady_clock::now();
            // active sizes after the step-0 pass, in internal event order
            std::vector<int> off(s->E + 1), act(s->E);
            GC_CUDA(cudaMemcpyAsync(off.data(), s->dev.ev_off[s->h_ctrl->cur], (s->E + 1) * sizeof(int),
                                    cudaMemcpyDeviceToHost, s->stream));
            GC_CUDA(cudaStreamSynchronize(s->stream));
            for (int64_t e = 0; e < s->E; ++e) act[e] = off[e + 1] - off[e];
            cudaEvent_t ea = nullptr, eb = nullptr;
            GC_CUDA(cudaEventCreate(&ea));
            GC_CUDA(cudaEventCreate(&eb));
            double best_rate = 0.0;
            gc_status st = GC_OK;
            auto trial = [&](const TuneKnobs &k) {
                if (st != GC_OK) return;
                double r = 0.0;
                st = time_shape(s, shape_of(s, sizes, k), act, ea, eb, &r);
                if (st == GC_OK && r > best_rate) {
                    best_rate = r;
                    best = k;
                }
            };
            for (int R : {2, 4, 8}) {  // stage 1: R x V
                if (s->p.pair_R && R != s->p.pair_R) continue;
                for (int V : {0, 1, 2}) {
                    TuneKnobs k = def;
                    k.R = R;
                    k.V = V;
                    trial(k);
                }
            }
            const TuneKnobs b1 = best;  // stage 2: fewer resident blocks per SM
            const int occ = pair_kernel_occupancy(s->p.precision, b1.R, s->p.newton, s->dev.tile_frames, b1.V);
            for (int bps = 1; bps < occ; ++bps) {
                TuneKnobs k = b1;
                k.bps = bps;
                trial(k);
            }
            if (!s->p.jchunk) {  // stage 3: j-chunk target
                const TuneKnobs b2 = best;
                for (int t : {16, 64}) {
                    TuneKnobs k = b2;
                    k.target = t;
                    trial(k);
                }
            }
            bool mid = false;  // stage 4: the 4-lane threshold, if it matters here
            for (int n : act) mid = mid || (n >= 1024 && n < 4096);
            if (mid) {
                const TuneKnobs b3 = best;
                for (int sn : {1024, 4096}) {
                    TuneKnobs k = b3;
                    k.small_n = sn;
                    trial(k);
                }
            }
            cudaEventDestroy(ea);
            cudaEventDestroy(eb);
            if (st != GC_OK) return st;
            {
                std::lock_guard<std::mutex> lock(g_tune_mutex);
                g_tune_cache[key] = best;
            }
            s->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
    }
    s->dev.shape = shape_of(s, sizes, best);
    GC_CUDA(launch_build_items(s->dev, s->stream));
    return GC_OK;
}

}  // namespace

extern "C" {

void gc_default_params(gc_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->abi_version = GC_ABI_VERSION;
    p->precision = GC_FP32_KAHAN;
    p->thickness_um = 675.0;
    p->z_well_um = 0.0;
    p->a1_V_cm_um = 2.0;
    p->a2_V_cm = 1500.0;
    p->T_K = 140.0;
    p->eps_si_rel = 11.7;
    p->softening_um = 0.01;
    p->dt_s = 1e-11;
    p->max_steps = 100000;
    p->coulomb = 1;
    p->diffusion = 1;
    p->reflect_back = 1;
    p->img_w = 64;
    p->img_h = 64;
    p->pixel_um = 15.0;
    p->graph_steps = 32;
    p->autotune = 1;
    p->newton = 0;
    p->jchunk = 0;
    p->fuse_small = 1;
}

const char *gc_status_string(gc_status st) {
    switch (st) {
        case GC_OK: return "GC_OK";
        case GC_INCOMPLETE: return "GC_INCOMPLETE: max_steps reached with carriers still active";
        case GC_ERR_PARAM: return "GC_ERR_PARAM: invalid argument or parameter";
        case GC_ERR_ALLOC: return "GC_ERR_ALLOC: allocation failed";
        case GC_ERR_CUDA: return "GC_ERR_CUDA: CUDA runtime error";
        case GC_ERR_STATE: return "GC_ERR_STATE: call out of order";
        case GC_ERR_DEVICE_TIMEOUT: return "GC_ERR_DEVICE_TIMEOUT: bounded device wait expired";
        case GC_ERR_NO_DEVICE: return "GC_ERR_NO_DEVICE: no CUDA device";
        case GC_ERR_DEVICE_CHECK: return "GC_ERR_DEVICE_CHECK: a device-side consistency check failed";
    }
    return "unknown gc_status";
}

const char *gc_last_cuda_error(void) { return g_cuda_err; }

gc_status gc_device_info(int32_t *sm_count, int32_t *cc_major, int32_t *cc_minor) {
    int dev = 0, cnt = 0;
    cudaError_t e = cudaGetDeviceCount(&cnt);
    if (e != cudaSuccess || cnt == 0) {
        if (e != cudaSuccess) cuda_fail(e);
        return GC_ERR_NO_DEVICE;
    }
    GC_CUDA(cudaGetDevice(&dev));
    int v = 0;
    if (sm_count) {
        GC_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        *sm_count = v;
    }
    if (cc_major) {
        GC_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMajor, dev));
        *cc_major = v;
    }
    if (cc_minor) {
        GC_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMinor, dev));
        *cc_minor = v;
    }
    return GC_OK;
}

gc_status gc_create(const gc_params *p, void *cuda_stream, gc_sim **out) {
    if (!out) return GC_ERR_PARAM;
    *out = nullptr;
    gc_status v = validate(p);
    if (v != GC_OK) return v;
    int cnt = 0;
    cudaError_t e = cudaGetDeviceCount(&cnt);
    if (e != cudaSuccess || cnt == 0) {
        if (e != cudaSuccess) cuda_fail(e);
        return GC_ERR_NO_DEVICE;
    }
    gc_sim *s = new (std::nothrow) gc_sim();
    if (!s) return GC_ERR_ALLOC;
    s->p = *p;
    s->phys = make_phys(*p);
    gc_status st = GC_OK;
    do {
        if ((e = cudaGetDevice(&s->device)) != cudaSuccess) { st = cuda_fail(e); break; }
        if ((e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device)) != cudaSuccess) {
            st = cuda_fail(e);
            break;
        }
        if (cuda_stream) {
            s->stream = (cudaStream_t)cuda_stream;
        } else {
            if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) {
                st = cuda_fail(e);
                break;
            }
            s->own_stream = true;
        }
        if ((e = cudaMallocHost((void **)&s->h_ctrl, sizeof(Ctrl))) != cudaSuccess) { st = cuda_fail(e); break; }
        if ((e = cudaMallocHost((void **)&s->h_limit, 3 * sizeof(long long))) != cudaSuccess) { st = cuda_fail(e); break; }
        if ((e = cudaMallocHost((void **)&s->h_probe, 2 * sizeof(unsigned))) != cudaSuccess) { st = cuda_fail(e); break; }
        std::memset(s->h_ctrl, 0, sizeof(Ctrl));
    } while (0);
    if (st != GC_OK) {
        gc_destroy(s);
        return st;
    }
    *out = s;
    return GC_OK;
}

gc_status gc_load_carriers(gc_sim *s, const double *xyz, int64_t n, const int64_t *event_offsets,
                           int64_t n_events, const uint64_t *seeds, const double *img_origin_xy) {
    if (!s) return GC_ERR_PARAM;
    if (n < 0 || n > (1LL << 30) || (n > 0 && !xyz)) return GC_ERR_PARAM;
    // caller's events
    std::vector<int64_t> uoff;
    if (event_offsets) {
        if (n_events < 1 || n_events > (1LL << 24)) return GC_ERR_PARAM;
        uoff.assign(event_offsets, event_offsets + n_events + 1);
        if (uoff[0] != 0 || uoff[n_events] != n) return GC_ERR_PARAM;
        for (int64_t e = 0; e < n_events; ++e)
            if (uoff[e + 1] < uoff[e]) return GC_ERR_PARAM;
    } else {
        if (n_events > 1) return GC_ERR_PARAM;
        n_events = 1;
        uoff = {0, n};
    }
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!is_finite(xyz[i])) return GC_ERR_PARAM;
    if (img_origin_xy)
        for (int64_t i = 0; i < 2 * n_events; ++i)
            if (!is_finite(img_origin_xy[i])) return GC_ERR_PARAM;
    GC_CUDA(cudaSetDevice(s->device));
    GC_CUDA(cudaStreamSynchronize(s->stream));
    free_state(s);
    const int64_t E = n_events;
    s->n = n;
    s->E = E;
    s->user_off = uoff;

    // internal event order: descending size (stable), i.e. largest work first
    std::vector<int> order(E);
    for (int64_t e = 0; e < E; ++e) order[e] = (int)e;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return uoff[a + 1] - uoff[a] > uoff[b + 1] - uoff[b];
    });
    std::vector<int> act(std::max<int64_t>(n, 1)), ev_of_id(std::max<int64_t>(n, 1)), ioff(E + 1);
    std::vector<unsigned long long> eseed(E);
    std::vector<double> eorig(3 * E), iorig(2 * E);
    std::vector<long long> sizes(E);
    int pos = 0;
    for (int64_t ie = 0; ie < E; ++ie) {
        const int ue = order[ie];
        ioff[ie] = pos;
        sizes[ie] = uoff[ue + 1] - uoff[ue];
        double cx = 0, cy = 0, cz = 0;
        for (int64_t id = uoff[ue]; id < uoff[ue + 1]; ++id) {
            act[pos++] = (int)id;
            ev_of_id[id] = (int)ie;
            cx += xyz[3 * id];
            cy += xyz[3 * id + 1];
            cz += xyz[3 * id + 2];
        }
        const double cnt = (double)std::max<int64_t>(sizes[ie], 1);
        eorig[3 * ie] = cx / cnt;
        eorig[3 * ie + 1] = cy / cnt;
        eorig[3 * ie + 2] = cz / cnt;
        eseed[ie] = seeds ? (unsigned long long)seeds[ue] : 1ull;
        if (img_origin_xy) {
            iorig[2 * ie] = img_origin_xy[2 * ue];
            iorig[2 * ie + 1] = img_origin_xy[2 * ue + 1];
        } else {
            iorig[2 * ie] = eorig[3 * ie] - 0.5 * s->p.img_w * s->p.pixel_um;
            iorig[2 * ie + 1] = eorig[3 * ie + 1] - 0.5 * s->p.img_h * s->p.pixel_um;
        }
    }
    ioff[E] = pos;
#ifdef GC_DEBUG
    if (s->inject == 1) {
        ioff[E] = pos + 7;  // planted: the offsets no longer match the carriers
        s->inject = 0;
    }
#endif
    // tile frames (FP32 forms, on request, when some event has >= small_n
    // holes): the large events in spatial (Morton) order
    const int small_n = kSmallEvent;
    long long n_max = 1;
    for (long long v : sizes) n_max = std::max(n_max, v);
    const bool frames = s->p.tile_frames && !fp64_mode(s) && (s->phys.coulomb || s->phys.stored) &&
                        n_max >= small_n;
    if (frames)
        for (int64_t ie = 0; ie < E; ++ie)
            if (sizes[ie] >= small_n) morton_order(xyz, act.data() + ioff[ie], (int)sizes[ie]);
    s->load_act.assign(act.begin(), act.begin() + pos);
    s->load_off.assign(ioff.begin(), ioff.end());
    std::vector<int> ev_user(order.begin(), order.end()), ev_first(E);
    for (int64_t ie = 0; ie < E; ++ie) ev_first[ie] = (int)uoff[order[ie]];
    std::vector<double> hx(std::max<int64_t>(n, 1)), hy(hx.size()), hz(hx.size());
    for (int64_t i = 0; i < n; ++i) {
        hx[i] = xyz[3 * i];
        hy[i] = xyz[3 * i + 1];
        hz[i] = xyz[3 * i + 2];
    }

    // partial-sum capacity: enough j-chunks for every autotune candidate
    long long cap = 1;
    if (fp64_mode(s) && s->phys.coulomb) {
        const PairShape sh = fp64_shape(s->sm_count, sizes, s->p.jchunk, 0);
        cap = (n_max + sh.jchunk - 1) / sh.jchunk;
    } else if (s->phys.coulomb) {
        for (int R : {2, 4, 8})  // every j-chunk the autotuner may try (up to 64 items per block)
            for (int target : {32, 64}) {
                PairShape sh = fp32_shape(R, s->sm_count, s->p.precision, s->p.newton, frames);
                sh.n_blocks = sh.n_blocks * target / 32;
                const int jc = choose_jchunk(sizes, sh, s->p.jchunk, kTileJ);
                cap = std::max(cap, (n_max + jc - 1) / jc);
            }
    }
    s->part_cap_chunks = cap;

    // the fused two-launch step for small workloads (not with the Newton
    // step, tile frames, stored charge or per-kernel timing)
    s->fused_ok = s->p.fuse_small && s->phys.coulomb && !s->phys.stored && !s->p.newton && !frames &&
                  !s->p.timing && n > 0;
    Dev &d = s->dev;
    const size_t N = (size_t)std::max<int64_t>(n, 1);
    const size_t nchunk = (size_t)ceil_div((int)N, kChunk);
    const size_t img = (size_t)E * s->p.img_w * s->p.img_h;
    DevAllocs &m = s->mem;
    cudaError_t e = cudaSuccess;
#define GC_ALLOC(ptr, bytes)                                                  \
    if ((e = m.alloc((void **)&(ptr), (bytes))) != cudaSuccess) {             \
        free_state(s);                                                        \
        return cuda_fail(e);                                                  \
    }
    GC_ALLOC(d.px, N * 8) GC_ALLOC(d.py, N * 8) GC_ALLOC(d.pz, N * 8)
    GC_ALLOC(d.ev_of_id, N * 4) GC_ALLOC(d.collect_step, N * 4)
    GC_ALLOC(d.act[0], N * 4) GC_ALLOC(d.act[1], N * 4)
    if (fp64_mode(s)) {
        GC_ALLOC(d.sh64, N * sizeof(double4_32a))
    } else {
        GC_ALLOC(d.sh32, N * sizeof(float4))
    }
    if (s->phys.coulomb) {
        GC_ALLOC(d.partial, (size_t)cap * 3 * N * 8)
    }
    if (s->p.precision == GC_FP16X2) {
        GC_ALLOC(d.ev_ext[0], E * 4) GC_ALLOC(d.ev_ext[1], E * 4)
    }
    if (frames) {
        GC_ALLOC(d.frame_hi, N * sizeof(float4)) GC_ALLOC(d.frame_lo, N * sizeof(float4))
    }
    std::vector<int> occ_off(E + 1, 0);  // stored charge: per-event occupied-pixel capacity
    for (int64_t ie = 0; ie < E; ++ie)
        occ_off[ie + 1] = occ_off[ie] + (int)std::min<long long>((long long)s->p.img_w * s->p.img_h, sizes[ie]);
    if (s->phys.stored) {
        GC_ALLOC(d.occ_pix, (size_t)std::max(occ_off[E], 1) * 4)
        GC_ALLOC(d.occ_q, (size_t)std::max(occ_off[E], 1) * 4)
        GC_ALLOC(d.occ_f4, (size_t)std::max(occ_off[E], 1) * 16)
        GC_ALLOC(d.occ_off, (E + 1) * 4) GC_ALLOC(d.occ_cnt, E * 4)
    }
    GC_ALLOC(d.keepmask, nchunk * (kChunk / 32) * 4) GC_ALLOC(d.chunk_cnt, nchunk * 4)
    GC_ALLOC(d.ev_off[0], (E + 1) * 4) GC_ALLOC(d.ev_off[1], (E + 1) * 4)
    GC_ALLOC(d.ev_collected_now, E * 4) GC_ALLOC(d.item_base, (E + 1) * 4)
    GC_ALLOC(d.ev_seed, E * 8) GC_ALLOC(d.ev_origin, E * 24) GC_ALLOC(d.img_origin, E * 16)
    GC_ALLOC(d.ev_user, E * 4) GC_ALLOC(d.ev_first, E * 4) GC_ALLOC(d.image, img * 4)
    GC_ALLOC(d.off_image, E * 8)
    if (s->fused_ok) {  // i-tiles are at least 8 carriers long
        GC_ALLOC(d.tile_base, (E + 1) * 4)
        GC_ALLOC(d.tile_ticket, (N / 8 + E + 1) * 4)
        GC_ALLOC(d.keep8, N)
    }
    // the persistent single-event kernel: one event, FP64 or FP32 without FP16x2;
    // its shadows and keep bytes (keep bytes by slot, shadows by hole id)
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
    s->se_ok = s->fused_ok && (s->p.fuse_small == 1 || s->p.fuse_small == 3) && E == 1 &&
               s->p.precision != GC_FP16X2 && coop;
    const bool fp32 = s->p.precision == GC_FP32 || s->p.precision == GC_FP32_KAHAN;
    s->cluster_ok = s->fused_ok && s->p.fuse_small == 5 && E == 1 && fp32;
    s->resident_ok = s->fused_ok && (s->p.fuse_small == 1 || s->p.fuse_small == 4) && E == 1 && fp32 && coop &&
                     resident_path_available(s->p.precision, kResidentPathMax, s->sm_count);
    if (s->resident_ok) {
        GC_ALLOC(d.rs_rec, resident_words_bytes())
    }
    if (s->se_ok) {
        const size_t M = N;  // indexed by hole id
        for (int b = 0; b < 2; ++b) {
            if (fp64_mode(s)) {
                GC_ALLOC(d.se_sh64[b], M * sizeof(double4_32a))
            } else {
                GC_ALLOC(d.se_sh32[b], M * sizeof(float4))
            }
            GC_ALLOC(d.se_keep[b], (M + 15) / 16 * 16)  // whole 16-byte words (vector loads)
        }
    }
    GC_ALLOC(d.ctrl, sizeof(Ctrl))
#undef GC_ALLOC
    d.part_stride = (long long)N;
    d.n_total = (int)n;
    d.n_events = (int)E;
    d.phys = s->phys;
    d.shape.R = fp64_mode(s) ? 1 : 4;
    d.shape.small_n = small_n;
    d.shape.small_lanes = fp64_mode(s) ? 16 : 4;
    d.tile_frames = frames ? 1 : 0;
    d.shape.jchunk = round_up(n_max, kTileJ);
    d.shape.n_blocks = s->sm_count;

    cudaStream_t st = s->stream;
    GC_CUDA(cudaMemcpyAsync(d.px, hx.data(), n * 8, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d.py, hy.data(), n * 8, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d.pz, hz.data(), n * 8, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d.ev_of_id, ev_of_id.data(), n * 4, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d.act[0], act.data(), n * 4, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d.ev_off[0], ioff.data(), (E + 1) * 4, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d.ev_seed, eseed.data(), E * 8, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d.ev_origin, eorig.data(), E * 24, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d.img_origin, iorig.data(), E * 16, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d.ev_user, ev_user.data(), E * 4, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d.ev_first, ev_first.data(), E * 4, cudaMemcpyHostToDevice, st));
    if (d.occ_off) {
        GC_CUDA(cudaMemcpyAsync(d.occ_off, occ_off.data(), (E + 1) * 4, cudaMemcpyHostToDevice, st));
        GC_CUDA(cudaMemsetAsync(d.occ_cnt, 0, E * 4, st));
    }
    GC_CUDA(cudaMemsetAsync(d.collect_step, 0xFF, N * 4, st));
    GC_CUDA(cudaMemsetAsync(d.chunk_cnt, 0, nchunk * 4, st));  // the step-0 pass may accumulate
    GC_CUDA(cudaMemsetAsync(d.ev_collected_now, 0, E * 4, st));
    GC_CUDA(cudaMemsetAsync(d.image, 0, img * 4, st));
    GC_CUDA(cudaMemsetAsync(d.off_image, 0, E * 8, st));
    if (d.tile_ticket) GC_CUDA(cudaMemsetAsync(d.tile_ticket, 0, (N / 8 + E + 1) * 4, st));
    if (d.ev_ext[0]) {
        GC_CUDA(cudaMemsetAsync(d.ev_ext[0], 0, E * 4, st));
        GC_CUDA(cudaMemsetAsync(d.ev_ext[1], 0, E * 4, st));
    }
    std::memset(s->h_ctrl, 0, sizeof(Ctrl));
    s->h_ctrl->step_limit = LLONG_MAX;  // open for the step-0 pass
    s->h_ctrl->n_active = (int)n;
    GC_CUDA(cudaMemcpyAsync(d.ctrl, s->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, st));

    // integrate/compact grid: one block per chunk (per 256-slot unit while few chunks
    // are active), at most two waves of blocks
    const int units0 = (int)nchunk * (fine_units((int)n) ? kChunk / kFineUnit : 1);
    s->integ_grid = std::max(1, std::min(units0, 2 * s->sm_count));
    const bool f64 = fp64_mode(s);
    if (n > 0) {
        // step 0: reflect at the back surface, collect what is already in the well
        GC_CUDA(launch_integrate(d, f64, true, s->integ_grid, st));
        GC_CUDA(launch_compact(d, f64, s->integ_grid, st));
        GC_CUDA(launch_finalize(d, true, st));
        if (d.tile_frames) GC_CUDA(launch_shadow(d, s->sm_count, st));
    }
    GC_CUDA(cudaStreamSynchronize(st));
    gc_status r = read_ctrl(s);
    if (r != GC_OK) return r;
    s->device_error = s->h_ctrl->error;
    if (s->device_error) {  // the step-0 pass found the input inconsistent: gc_run reports it
        s->loaded = true;
        return GC_OK;
    }
    if (s->phys.coulomb && n > 0) {
        r = choose_shape(s, sizes);  // the sizes the partial buffer was sized for
        if (r != GC_OK) return r;
    }
    if (s->fused_ok) {
        s->fused_grid = s->sm_count * std::max(1, fused_pair_occupancy(s->p.precision, s->dev.shape.R));
        if (!fused_pair_kernel_ptr(s->p.precision, s->dev.shape.R)) s->fused_ok = s->se_ok = false;
    }
    if (s->se_ok) {
        const int occ = se_occupancy(s->p.precision, s->dev.shape.R);
        s->se_grid = s->sm_count * occ;
        if (occ < 1 || !se_kernel_ptr(s->p.precision, s->dev.shape.R)) s->se_ok = false;
    }
    r = set_limit(s, 0);
    if (r != GC_OK) return r;
    r = read_ctrl(s);
    if (r != GC_OK) return r;
    s->launches_per_step = (s->fused_ok && s->h_ctrl->n_active <= kFusedMax)
                               ? ((s->se_ok || s->resident_ok || s->cluster_ok) ? 0 : 2)
                               : (s->phys.coulomb ? 1 : 0) + (s->phys.stored ? 1 : 0) + (frames ? 1 : 0) + 3;
    if (s->p.timing) {
        for (auto *v : {&s->ev_a, &s->ev_b, &s->ev_c, &s->ev_d}) {
            v->resize(1);
            GC_CUDA(cudaEventCreate(&(*v)[0]));
        }
    }
    s->loaded = true;
    r = capture_graph(s);
    if (r != GC_OK) {
        s->loaded = false;
        return r;
    }
    return GC_OK;
}

gc_status gc_run(gc_sim *s, int64_t steps, int64_t *steps_done) {
    if (steps_done) *steps_done = 0;
    if (!s) return GC_ERR_PARAM;
    if (!s->loaded) return GC_ERR_STATE;
    if (s->device_error) return device_error_status(s->device_error);
    GC_CUDA(cudaSetDevice(s->device));
    const long long step0 = s->h_ctrl->step;
    const long long max_steps = s->p.max_steps;
    const long long limit = steps < 0 ? max_steps : std::min<long long>(max_steps, step0 + steps);
    if (s->h_ctrl->n_active > 0 && step0 < limit) {
        gc_status r = set_limit(s, limit);
        if (r != GC_OK) return r;
        const int K = use_graph(s) ? s->p.graph_steps : 1;
        s->fused_ran = false;
        // Up to three phases: the unfused step while more than kFusedMax holes
        // are active, then (when available) a small-workload path: the
        // persistent kernel until at most kResidentPathMax holes are active
        // and the grid-resident kernel from there (one FP32 event), or one of
        // the others.
        for (int phase = 0; phase < 3; ++phase) {
            const bool fz = s->fused_ok && s->h_ctrl->n_active <= kFusedMax;
            const int na0 = s->h_ctrl->n_active;
            if (fz && s->resident_ok && na0 <= kResidentPathMax &&
                resident_path_available(s->p.precision, na0, s->sm_count)) {
                // one event: the whole remaining loop on every SM, each CTA owning
                // a fixed set of holes, no grid barrier between steps
                s->fused_ran = 4;
                Dev dd = s->dev;
#ifdef GC_DEBUG
                dd.dbg_withhold = s->inject == 2;  // planted: one CTA withholds its first words
                if (s->inject == 2) s->inject = 0;
#endif
                GC_CUDA(launch_resident_event(dd, s->p.precision, na0, s->sm_count, s->p.resident_ctas,
                                              kDeviceWaitLimitS, s->stream));
                r = read_ctrl(s);
                if (r != GC_OK) return r;
                if (s->h_ctrl->error) {
                    s->device_error = s->h_ctrl->error;
                    return device_error_status(s->device_error);
                }
                GC_CUDA(launch_build_items(s->dev, s->stream));  // items in the other paths' layout
                break;
            }
            if (fz && s->cluster_ok && cluster_path_available(s->p.precision, na0)) {
                // one event of at most 2048 holes: the whole remaining loop in one
                // cluster, its state in shared memory
                s->fused_ran = 3;
                GC_CUDA(launch_cluster_event(s->dev, s->p.precision, na0, s->stream));
                r = read_ctrl(s);
                if (r != GC_OK) return r;
                if (s->h_ctrl->error) {
                    s->device_error = s->h_ctrl->error;
                    return device_error_status(s->device_error);
                }
                GC_CUDA(launch_build_items(s->dev, s->stream));  // items in the other paths' layout
                break;
            }
            if (fz && s->se_ok) {
                // one event, few holes: the whole remaining loop in one cooperative launch
                s->fused_ran = 2;
                // at most one block per work item of the first step (fewer arrivals per barrier)
                const int na = s->h_ctrl->n_active;
                const PairShape &sh = s->dev.shape;
                const long long items = (long long)ceil_div(na, itile_for(sh.R, lanes_for(sh, na))) *
                                        ceil_div(na, sh.jchunk);
                const int grid = (int)std::max(1LL, std::min<long long>(s->se_grid, items));
                GC_CUDA(launch_se_loop(s->dev, s->p.precision, grid, kDeviceWaitLimitS, s->stream));
                r = read_ctrl(s);
                if (r != GC_OK) return r;
                if (s->h_ctrl->error) {  // the state is undefined after a failed check or wait
                    s->device_error = s->h_ctrl->error;
                    return device_error_status(s->device_error);
                }
                GC_CUDA(launch_build_items(s->dev, s->stream));  // items in the other paths' layout
                if (s->resident_ok && s->h_ctrl->n_active > 0 && s->h_ctrl->step < limit) continue;
                break;
            }
            if (fz) s->fused_ran = 1;
            cudaGraphExec_t g = fz ? s->graph_small : s->graph;
            const bool loops = fz ? s->small_loops : s->graph_loops;
            if (use_graph(s) && !g) return GC_ERR_STATE;
            const long long want = limit - s->h_ctrl->step;
            // one launch = one captured graph of K steps, or one eager step
            auto launch_one = [&]() -> gc_status {
                const long long before = s->h_ctrl->step;
                if (use_graph(s)) {
                    GC_CUDA(cudaGraphLaunch(g, s->stream));
                } else {
                    gc_status q = enqueue_step(s, 0, fz);
                    if (q != GC_OK) return q;
                }
                if (s->p.timing) {  // read this launch's events before they are re-recorded
                    gc_status q = read_ctrl(s);
                    if (q != GC_OK) return q;
                    const long long did = std::min<long long>(K, s->h_ctrl->step - before);
                    for (long long k = 0; k < did; ++k) {
                        float ms = 0.f;
                        if (s->phys.coulomb) {
                            GC_CUDA(cudaEventElapsedTime(&ms, s->ev_a[k], s->ev_b[k]));
                            s->pair_ms += ms;
                            s->pair_launches += 1;
                        }
                        GC_CUDA(cudaEventElapsedTime(&ms, s->ev_b[k], s->ev_c[k]));
                        s->integ_ms += ms;
                        GC_CUDA(cudaEventElapsedTime(&ms, s->ev_c[k], s->ev_d[k]));
                        s->compact_ms += ms;
                        s->timed_steps += 1;
                    }
                }
                return GC_OK;
            };
            if (use_graph(s) && loops) {
                // the device-side loop runs to the limit, to completion or (the
                // unfused loop) to the hand-over, in one launch
                GC_CUDA(cudaGraphLaunch(g, s->stream));
                r = read_ctrl(s);
                if (r != GC_OK) return r;
            } else if (steps >= 0) {
                // known step count: enqueue everything, synchronise once
                for (long long k = 0; k < (want + K - 1) / K; ++k) {
                    r = launch_one();
                    if (r != GC_OK) return r;
                }
                r = read_ctrl(s);
                if (r != GC_OK) return r;
            } else {
                // until every carrier is collected: poll between batches of steps
                const long long batch = std::max(1, 256 / K);
                for (;;) {
                    const long long before = s->h_ctrl->step;
                    for (long long k = 0; k < batch; ++k) {
                        r = launch_one();
                        if (r != GC_OK) return r;
                    }
                    r = read_ctrl(s);
                    if (r != GC_OK) return r;
                    if (s->h_ctrl->n_active <= 0 || s->h_ctrl->step >= limit) break;
                    if (!fz && s->fused_ok && s->h_ctrl->n_active <= kFusedMax) break;  // hand over
                    if (s->resident_ok && s->h_ctrl->n_active <= kResidentPathMax) break;  // hand over
                    if (s->h_ctrl->step == before) return GC_ERR_STATE;  // no progress: never spin
                }
            }
            if (s->h_ctrl->n_active <= 0 || s->h_ctrl->step >= limit) break;
            // the next phase: a small-workload path below kFusedMax, the grid-resident
            // kernel below kResidentPathMax
            if (fz ? !(s->resident_ok && s->h_ctrl->n_active <= kResidentPathMax)
                   : !(s->fused_ok && s->h_ctrl->n_active <= kFusedMax))
                break;
        }
        if (s->h_ctrl->error) {
            s->device_error = s->h_ctrl->error;
            return device_error_status(s->device_error);
        }
        r = set_limit(s, s->h_ctrl->step);  // closed until the next gc_run
        if (r != GC_OK) return r;
    }
    if (steps_done) *steps_done = s->h_ctrl->step - step0;
    if (s->h_ctrl->n_active > 0 && s->h_ctrl->step >= max_steps) return GC_INCOMPLETE;
    return GC_OK;
}

gc_status gc_collect(gc_sim *s, double *final_xy, int32_t *collect_step, int64_t *n_collected,
                     int64_t *n_offimage, int64_t *n_active) {
    if (!s) return GC_ERR_PARAM;
    if (!s->loaded) return GC_ERR_STATE;
    GC_CUDA(cudaSetDevice(s->device));
    const int64_t n = s->n, E = s->E;
    std::vector<int32_t> cs(std::max<int64_t>(n, 1));
    GC_CUDA(cudaMemcpyAsync(cs.data(), s->dev.collect_step, n * 4, cudaMemcpyDeviceToHost, s->stream));
    std::vector<double> hx, hy;
    if (final_xy) {
        hx.resize(std::max<int64_t>(n, 1));
        hy.resize(std::max<int64_t>(n, 1));
        GC_CUDA(cudaMemcpyAsync(hx.data(), s->dev.px, n * 8, cudaMemcpyDeviceToHost, s->stream));
        GC_CUDA(cudaMemcpyAsync(hy.data(), s->dev.py, n * 8, cudaMemcpyDeviceToHost, s->stream));
    }
    std::vector<unsigned long long> off(std::max<int64_t>(E, 1));
    GC_CUDA(cudaMemcpyAsync(off.data(), s->dev.off_image, E * 8, cudaMemcpyDeviceToHost, s->stream));
    GC_CUDA(cudaStreamSynchronize(s->stream));
    if (collect_step) std::memcpy(collect_step, cs.data(), n * 4);
    if (final_xy)
        for (int64_t i = 0; i < n; ++i) {
            final_xy[2 * i] = hx[i];
            final_xy[2 * i + 1] = hy[i];
        }
    for (int64_t e = 0; e < E; ++e) {
        int64_t col = 0;
        for (int64_t i = s->user_off[e]; i < s->user_off[e + 1]; ++i) col += cs[i] >= 0;
        if (n_collected) n_collected[e] = col;
        if (n_active) n_active[e] = (s->user_off[e + 1] - s->user_off[e]) - col;
        if (n_offimage) n_offimage[e] = (int64_t)off[e];
    }
    return GC_OK;
}

gc_status gc_image(gc_sim *s, uint32_t *img, int is_device) {
    if (!s || !img) return GC_ERR_PARAM;
    if (!s->loaded) return GC_ERR_STATE;
    GC_CUDA(cudaSetDevice(s->device));
    const size_t bytes = (size_t)s->E * s->p.img_w * s->p.img_h * 4;
    GC_CUDA(cudaMemcpyAsync(img, s->dev.image, bytes,
                            is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
    GC_CUDA(cudaStreamSynchronize(s->stream));
    return GC_OK;
}

gc_status gc_positions(gc_sim *s, double *xyz) {
    if (!s || !xyz) return GC_ERR_PARAM;
    if (!s->loaded) return GC_ERR_STATE;
    GC_CUDA(cudaSetDevice(s->device));
    const int64_t n = s->n;
    std::vector<double> hx(std::max<int64_t>(n, 1)), hy(hx.size()), hz(hx.size());
    GC_CUDA(cudaMemcpyAsync(hx.data(), s->dev.px, n * 8, cudaMemcpyDeviceToHost, s->stream));
    GC_CUDA(cudaMemcpyAsync(hy.data(), s->dev.py, n * 8, cudaMemcpyDeviceToHost, s->stream));
    GC_CUDA(cudaMemcpyAsync(hz.data(), s->dev.pz, n * 8, cudaMemcpyDeviceToHost, s->stream));
    GC_CUDA(cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < n; ++i) {
        xyz[3 * i] = hx[i];
        xyz[3 * i + 1] = hy[i];
        xyz[3 * i + 2] = hz[i];
    }
    return GC_OK;
}

gc_status gc_get_stats(gc_sim *s, gc_stats *out) {
    if (!s || !out) return GC_ERR_PARAM;
    if (!s->loaded) return GC_ERR_STATE;
    GC_CUDA(cudaSetDevice(s->device));
    gc_status r = read_ctrl(s);
    if (r != GC_OK) return r;
    std::memset(out, 0, sizeof(*out));
    out->steps = s->h_ctrl->step;
    out->n_active = s->h_ctrl->n_active;
    out->n_collected = s->n - s->h_ctrl->n_active;
    out->pair_interactions = (double)s->h_ctrl->pair_interactions;
    out->carrier_steps = (double)s->h_ctrl->carrier_steps;
    out->pair_variant = s->dev.shape.R;
    out->pair_blocks = s->dev.shape.n_blocks;
    out->jchunk = s->dev.shape.jchunk;
    out->launches_per_step = s->launches_per_step;
    out->pair_kernel_ms = s->pair_ms;
    out->pair_kernel_launches = s->pair_launches;
    out->integrate_kernel_ms = s->integ_ms;
    out->compact_kernel_ms = s->compact_ms;
    out->timed_steps = s->timed_steps;
    out->device_loop = use_graph(s) && (!s->graph || s->graph_loops) && (!s->graph_small || s->small_loops);
    out->fused_path = s->fused_ran;
    out->tune_ms = s->tune_ms;
    out->tune_candidates = s->tune_candidates;
    out->tune_cached = s->tune_cached;
    out->pair_kernel_variant = s->dev.shape.V;
    out->small_n = s->dev.shape.small_n;
    return GC_OK;
}

gc_status gc_save_state(gc_sim *s, gc_state *st) {
    if (!s || !st || (s->n > 0 && (!st->xyz || !st->collect_step)) || !st->image || !st->off_image)
        return GC_ERR_PARAM;
    if (!s->loaded) return GC_ERR_STATE;
    gc_status r = gc_positions(s, st->xyz);
    if (r != GC_OK) return r;
    r = gc_collect(s, nullptr, st->collect_step, nullptr, st->off_image, nullptr);
    if (r != GC_OK) return r;
    r = gc_image(s, st->image, 0);
    if (r != GC_OK) return r;
    r = read_ctrl(s);
    if (r != GC_OK) return r;
    st->step = s->h_ctrl->step;
    st->pair_interactions = (double)s->h_ctrl->pair_interactions;
    st->carrier_steps = (double)s->h_ctrl->carrier_steps;
    return GC_OK;
}

gc_status gc_restore_state(gc_sim *s, const gc_state *st) {
    if (!s || !st || (s->n > 0 && (!st->xyz || !st->collect_step)) || !st->image || !st->off_image)
        return GC_ERR_PARAM;
    if (!s->loaded) return GC_ERR_STATE;
    if (st->step < 0 || st->step > s->p.max_steps) return GC_ERR_PARAM;
    const int64_t n = s->n, E = s->E;
    for (int64_t i = 0; i < n; ++i) {
        const double z = st->xyz[3 * i + 2];
        if (!is_finite(st->xyz[3 * i]) || !is_finite(st->xyz[3 * i + 1]) || !is_finite(z)) return GC_ERR_PARAM;
        if (st->collect_step[i] < -1 || st->collect_step[i] > st->step) return GC_ERR_PARAM;
        if (st->collect_step[i] < 0 && (z <= s->p.z_well_um || (s->p.reflect_back && z > s->p.thickness_um)))
            return GC_ERR_PARAM;
    }
    GC_CUDA(cudaSetDevice(s->device));
    Dev &d = s->dev;
    cudaStream_t q = s->stream;
    // the active list in the load order (what stable compaction has kept)
    std::vector<int> act(std::max<int64_t>(n, 1)), ioff(E + 1);
    int pos = 0;
    for (int64_t ie = 0; ie < E; ++ie) {
        ioff[ie] = pos;
        for (int k = s->load_off[ie]; k < s->load_off[ie + 1]; ++k)
            if (st->collect_step[s->load_act[k]] < 0) act[pos++] = s->load_act[k];
    }
    ioff[E] = pos;
    std::vector<double> hx(std::max<int64_t>(n, 1)), hy(hx.size()), hz(hx.size());
    for (int64_t i = 0; i < n; ++i) {
        hx[i] = st->xyz[3 * i];
        hy[i] = st->xyz[3 * i + 1];
        hz[i] = st->xyz[3 * i + 2];
    }
    std::vector<unsigned long long> off(std::max<int64_t>(E, 1));
    for (int64_t e = 0; e < E; ++e) off[e] = (unsigned long long)st->off_image[e];
    const size_t img = (size_t)E * s->p.img_w * s->p.img_h;
    GC_CUDA(cudaMemcpyAsync(d.px, hx.data(), n * 8, cudaMemcpyHostToDevice, q));
    GC_CUDA(cudaMemcpyAsync(d.py, hy.data(), n * 8, cudaMemcpyHostToDevice, q));
    GC_CUDA(cudaMemcpyAsync(d.pz, hz.data(), n * 8, cudaMemcpyHostToDevice, q));
    GC_CUDA(cudaMemcpyAsync(d.collect_step, st->collect_step, n * 4, cudaMemcpyHostToDevice, q));
    GC_CUDA(cudaMemcpyAsync(d.image, st->image, img * 4, cudaMemcpyHostToDevice, q));
    GC_CUDA(cudaMemcpyAsync(d.off_image, off.data(), E * 8, cudaMemcpyHostToDevice, q));
    GC_CUDA(cudaMemcpyAsync(d.act[0], act.data(), (size_t)pos * 4, cudaMemcpyHostToDevice, q));
    GC_CUDA(cudaMemcpyAsync(d.ev_off[0], ioff.data(), (E + 1) * 4, cudaMemcpyHostToDevice, q));
    GC_CUDA(cudaMemsetAsync(d.ev_collected_now, 0, E * 4, q));
    GC_CUDA(cudaMemsetAsync(d.chunk_cnt, 0, (size_t)ceil_div((int)std::max<int64_t>(n, 1), kChunk) * 4, q));
    if (d.tile_ticket)
        GC_CUDA(cudaMemsetAsync(d.tile_ticket, 0, ((size_t)std::max<int64_t>(n, 1) / 8 + E + 1) * 4, q));
    GC_CUDA(cudaStreamSynchronize(q));
    Ctrl c{};
    c.step = st->step;
    c.step_limit = LLONG_MAX;  // open for the rebuild pass
    c.n_active = pos;
    c.cur = 0;
    c.pair_interactions = (unsigned long long)st->pair_interactions;
    c.carrier_steps = (unsigned long long)st->carrier_steps;
    *s->h_ctrl = c;
    GC_CUDA(cudaMemcpyAsync(d.ctrl, s->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, q));
    if (pos > 0) {
        // the step-0 pass keeps every (consistent) active carrier and rebuilds
        // the shadow, the event offsets and the pair work items
        const bool f64 = fp64_mode(s);
        GC_CUDA(launch_integrate(d, f64, true, s->integ_grid, q));
        GC_CUDA(launch_compact(d, f64, s->integ_grid, q));
        GC_CUDA(launch_finalize(d, true, q));
        if (d.tile_frames) GC_CUDA(launch_shadow(d, s->sm_count, q));
    }
    gc_status r = set_limit(s, st->step);
    if (r != GC_OK) return r;
    return read_ctrl(s);
}

gc_status gc_coulomb_field(const double *xyz_dev, int64_t n, double softening_um, double eps_si_rel,
                           int32_t precision, double *E_dev, void *cuda_stream) {
    if (n < 0 || n > (1LL << 30)) return GC_ERR_PARAM;
    if (!(softening_um > 0) || !is_finite(softening_um) || !(eps_si_rel > 0) || !is_finite(eps_si_rel))
        return GC_ERR_PARAM;
    if (precision < GC_FP64 || precision > GC_FP16X2) return GC_ERR_PARAM;
    if (n > 0 && (!xyz_dev || !E_dev)) return GC_ERR_PARAM;
    int cnt = 0;
    cudaError_t e = cudaGetDeviceCount(&cnt);
    if (e != cudaSuccess || cnt == 0) {
        if (e != cudaSuccess) cuda_fail(e);
        return GC_ERR_NO_DEVICE;
    }
    if (n == 0) return GC_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    GC_CUDA(cudaGetDevice(&dev));
    GC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    gc_params p;
    gc_default_params(&p);
    p.softening_um = softening_um;
    p.eps_si_rel = eps_si_rel;
    Dev d{};
    d.phys = make_phys(p);
    const bool f64 = precision == GC_FP64;
    d.shape = field_shape(precision, sms, n, 0);
    const long long S = (n + d.shape.jchunk - 1) / d.shape.jchunk;
    DevAllocs m;
    gc_status status = GC_OK;
    do {
        if ((e = m.alloc(f64 ? (void **)&d.sh64 : (void **)&d.sh32, (size_t)n * (f64 ? 32 : 16))) ||
            (e = m.alloc((void **)&d.partial, (size_t)S * 3 * n * 8)) ||
            (e = m.alloc((void **)&d.ev_off[0], 8)) || (e = m.alloc((void **)&d.item_base, 8)) ||
            (e = m.alloc((void **)&d.ev_origin, 24)) || (e = m.alloc((void **)&d.ctrl, sizeof(Ctrl))) ||
            (precision == GC_FP16X2 && (e = m.alloc((void **)&d.ev_ext[0], 4)))) {
            status = cuda_fail(e);
            break;
        }
        d.ev_off[1] = d.ev_off[0];
        d.part_stride = n;
        d.n_total = (int)n;
        d.n_events = 1;
        Ctrl c{};
        c.step_limit = 1;
        c.n_active = (int)n;
        const int off[2] = {0, (int)n};
        if ((e = cudaMemcpyAsync(d.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(d.ev_off[0], off, 8, cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(d.ev_origin, xyz_dev, 24, cudaMemcpyDeviceToDevice, st)) ||
            (d.ev_ext[0] && (e = cudaMemsetAsync(d.ev_ext[0], 0, 4, st))) ||
            (e = launch_field_prepare(d, xyz_dev, (int)n, f64, st)) || (e = launch_build_items(d, st)) ||
            (e = launch_pair(d, precision, 0, st)) || (e = launch_field_finish(d, (int)n, E_dev, st)) ||
            (e = cudaStreamSynchronize(st))) {
            status = cuda_fail(e);
            break;
        }
    } while (0);
    cudaStreamSynchronize(st);
    m.release();
    return status;
}

gc_status gc_debug_inject(gc_sim *s, int32_t what) {
    if (!s || what < 0 || what > 2) return GC_ERR_PARAM;
#ifdef GC_DEBUG
    s->inject = what;
    return GC_OK;
#else
    return GC_ERR_STATE;  // only builds with GC_DEBUG plant faults
#endif
}

gc_status gc_selftest_barrier_timeout(double limit_s) {
    if (!(limit_s > 0) || !(limit_s <= 10.0)) return GC_ERR_PARAM;
    int cnt = 0;
    cudaError_t e = cudaGetDeviceCount(&cnt);
    if (e != cudaSuccess || cnt == 0) {
        if (e != cudaSuccess) cuda_fail(e);
        return GC_ERR_NO_DEVICE;
    }
    int dev = 0, sms = 0, coop = 0;
    GC_CUDA(cudaGetDevice(&dev));
    GC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GC_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return GC_ERR_NO_DEVICE;
    int bits = 0;
    GC_CUDA(selftest_barrier_timeout(sms, limit_s, &bits, nullptr));
    return (bits & kErrBarrierTimeout) ? GC_ERR_DEVICE_TIMEOUT : GC_OK;
}

void gc_destroy(gc_sim *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    free_state(s);
    if (s->h_ctrl) cudaFreeHost(s->h_ctrl);
    if (s->h_limit) cudaFreeHost(s->h_limit);
    if (s->h_probe) cudaFreeHost(s->h_probe);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
