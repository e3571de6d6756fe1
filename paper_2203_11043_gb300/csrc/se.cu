// se.cu -- the persistent single-event kernel: the whole Fig. 2 loop of one
// small event (at most kFusedMax active holes) in one cooperative launch.
//
// A small event's step is a few microseconds of arithmetic but a chain of
// dependent memory round trips per kernel; a launch per stage (or two, in
// the fused path) pays that chain again and again.  Here every block stays
// resident for all steps:
//   0. (once per launch) the shadow is copied into a buffer indexed by hole
//      id, then one grid barrier;
//   1. pair + integrate: blocks take the step's pair work items (the same
//      items, partial sums and per-carrier arithmetic as the other paths);
//      the item that completes an i-tile's j-chunks integrates that i-tile
//      and writes each kept hole's next shadow at the hole's id;
//   2. one grid barrier (bounded in time, gc_barrier.cuh);
//   3. every block compacts its own copy of the active list (hole ids, in
//      shared memory) from the step's keep bytes, so no data moves between
//      steps.
// Slot numbering, j order and partial sums are those of the compacted active
// list of the four-launch step, so the results are the same bits.  At the end
// block 0 writes the state back in the layout of the other paths.
#include <type_traits>

#include "gc_barrier.cuh"
#include "gc_pair.cuh"
#include "gc_launch.h"

namespace gc {

constexpr int kSEListBytes = kFusedMax * 4;  // dynamic shared memory: the active list (hole ids)

// After one pair item (slots of event 0 numbered by the current list): the
// item that completes its i-tile integrates the tile's holes.
// (x, y, z): the position of this thread's hole of the i-tile (preloaded).
template <bool F64, typename Shadow>
__device__ __forceinline__ void se_tile_done(const Dev &d, int n, int local, int js, int itile, long long step,
                                             const int *list, unsigned char *keep, Shadow *wr, int *s_flag,
                                             double x, double y, double z) {
    const int it = local / js;
    __syncthreads();  // the block's partial sums before thread 0's release (or own use)
    if (js == 1) {
        // one j-chunk: this item completes its i-tile
    } else if (threadIdx.x == 0) {
        fence_acq_rel_gpu();
        unsigned *t = d.tile_ticket + it;
        const unsigned done = atomicAdd(t, 1u);
        const int last = done == (unsigned)(js - 1);
        if (last) {
            *t = 0u;
            fence_acq_rel_gpu();  // acquire: the other items' partial sums (read through L2)
        }
        *s_flag = last;
    }
    if (js > 1) {
        __syncthreads();
        if (!*s_flag) return;
    }
    const double ox = d.ev_origin[0], oy = d.ev_origin[1], oz = d.ev_origin[2];
    const int i1 = min(n, (it + 1) * itile);
    bool first = true;  // the first hole's position was preloaded; larger i-tiles load the rest here
    for (int q = it * itile + (int)threadIdx.x; q < i1; q += blockDim.x, first = false) {
        const int id = list[q];
        if (!first) {
            x = __ldcg(d.px + id);
            y = __ldcg(d.py + id);
            z = __ldcg(d.pz + id);
        }
        const bool kept = advance_hole<F64, false, true>(d, id, 0, n, q, step, x, y, z);
        if (kept) {  // the shadow of the next step, as the compaction writes it
            if constexpr (F64)
                wr[id] = make_double4_32a(x - ox, y - oy, z - oz, 0.0);
            else
                wr[id] = make_float4((float)(x - ox), (float)(y - oy), (float)(z - oz), 1.0f);
        }
        keep[q] = kept ? 1 : 0;
    }
}

// Stable in-place compaction of list[0..n) by keep (written by other blocks:
// read through L2), in rounds of 16 slots per thread; returns the new length.
__device__ __forceinline__ int se_compact_list(int *list, const unsigned char *keep, int n, long long *s_warp) {
    constexpr int PER = 16;  // one 16-byte load of keep bytes per thread and round
    int base = 0;
    for (int c0 = 0; c0 < n; c0 += PER * (int)blockDim.x) {
        const int p0 = c0 + (int)threadIdx.x * PER;
        int v[PER];
        unsigned char kb[PER];
        int cnt = 0;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (p0 < n) w = __ldcg(reinterpret_cast<const uint4 *>(keep + p0));  // keep is 16-byte aligned
        const unsigned wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int p = p0 + u;
            kb[u] = p < n ? (unsigned char)((wv[u >> 2] >> (8 * (u & 3))) & 0xffu) : (unsigned char)0;
            v[u] = p < n ? list[p] : 0;
            cnt += kb[u];
        }
        long long tot;
        int q = base + (int)block_exclusive_scan(cnt, s_warp, tot);  // all reads of the round precede its writes
#pragma unroll
        for (int u = 0; u < PER; ++u)
            if (kb[u]) list[q++] = v[u];
        base += (int)tot;
    }
    __syncthreads();
    return base;
}

// FP64: the pair term is FP64-latency bound, so keep 5 blocks (20 warps) per SM.
template <int R, bool KAHAN, bool F64>
__global__ void __launch_bounds__(kPairThreads, F64 ? 5 : 1) se_loop_kernel(Dev d, unsigned long long limit_ns) {
    extern __shared__ int s_list[];  // the active list: kFusedMax hole ids
    __shared__ __align__(16) float s_x[4 * kTileJ], s_y[4 * kTileJ], s_z[4 * kTileJ];
    __shared__ __align__(16) float4 s_raw[4 * kTileJ];
    __shared__ float4 s_fr[1];
    __shared__ long long s_warp[33];
    __shared__ int s_flag, s_ok;
    using Shadow = typename std::conditional<F64, double4_32a, float4>::type;
    Ctrl *c = d.ctrl;
    if (step_skipped(c)) return;  // uniform: nothing changes the control block before the first barrier
    const long long limit = c->step_limit, stop_below = c->stop_below;
    long long step = c->step;
    const int cur = c->cur;
    const int *act0 = d.act[cur];
    int n = c->n_active;
    for (int q = threadIdx.x; q < n; q += blockDim.x) s_list[q] = act0[q];
    // the shadow of the first step, indexed by hole id
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        if constexpr (F64) d.se_sh64[0][act0[q]] = d.sh64[q];
        else d.se_sh32[0][act0[q]] = d.sh32[q];
    }
    if (!grid_barrier(&c->bar_count, &c->bar_gen, &c->error, gridDim.x, limit_ns, &s_ok)) return;
    unsigned long long pairs = 0, csteps = 0;
    int k = 0;
    for (;; ++k) {
        unsigned char *keep = d.se_keep[k & 1];
        const Shadow *rd;
        Shadow *wr;
        if constexpr (F64) {
            rd = d.se_sh64[k & 1];
            wr = d.se_sh64[(k + 1) & 1];
        } else {
            rd = d.se_sh32[k & 1];
            wr = d.se_sh32[(k + 1) & 1];
        }
        const int L = lanes_for(d.shape, n);
        const int itile = itile_for(d.shape.R, L);
        const int js = ceil_div(n, d.shape.jchunk);
        const int items = ceil_div(n, itile) * js;
        // FP32: one or a few items per block, assigned round-robin; FP64: many
        // long items, taken from a counter (reset by block 0 after the step's barrier)
        for (int item = F64 ? -1 : (int)blockIdx.x;; item += gridDim.x) {
            if constexpr (F64) {
                __syncthreads();
                if (threadIdx.x == 0) s_flag = (int)atomicAdd(&c->se_item[k & 1], 1u);
                __syncthreads();
                item = s_flag;
            }
            if (item >= items) break;
            // this thread's hole of the item's i-tile: its position is loaded now, so that
            // the integration after the pair sum waits on no memory but the partial sums
            double hx = 0.0, hy = 0.0, hz = 0.0;
            {
                const int q = (item / js) * itile + (int)threadIdx.x;
                if ((int)threadIdx.x < itile && q < n) {  // the first hole this thread integrates
                    const int id = s_list[q];
                    hx = __ldcg(d.px + id);
                    hy = __ldcg(d.py + id);
                    hz = __ldcg(d.pz + id);
                }
            }
            if constexpr (F64) {
                double *tx = reinterpret_cast<double *>(s_x), *ty = reinterpret_cast<double *>(s_y),
                       *tz = reinterpret_cast<double *>(s_z);
                if (L == 1) pair_item_fp64<1, true>(d, 0, n, item, tx, ty, tz, rd, s_list);
                else pair_item_fp64<16, true>(d, 0, n, item, tx, ty, tz, rd, s_list);
            } else {
                if (L == 1)
                    pair_item_fp32_j<R, KAHAN, false, 1, false, false, true>(d, 0, n, item, 1.0f, s_x, s_y, s_z,
                                                                           s_fr, s_raw, rd, s_list);
                else
                    pair_item_fp32_j<R, KAHAN, false, 4, false, false, true>(d, 0, n, item, 1.0f, s_x, s_y, s_z,
                                                                           s_fr, s_raw, rd, s_list);
            }
            se_tile_done<F64>(d, n, item, js, itile, step + 1, s_list, keep, wr, &s_flag, hx, hy, hz);
            __syncthreads();  // shared tiles and s_flag are reused by the next item
        }
        if (!grid_barrier(&c->bar_count, &c->bar_gen, &c->error, gridDim.x, limit_ns, &s_ok)) return;
        if (F64 && blockIdx.x == 0 && threadIdx.x == 0) c->se_item[k & 1] = 0u;  // every block is past its items
        pairs += (unsigned long long)n * (unsigned long long)n;
        csteps += (unsigned long long)n;
        n = se_compact_list(s_list, keep, n, s_warp);
        ++step;
        if (n <= stop_below || n == 0 || step >= limit) break;  // (stop_below: a hand-over)
    }
    if (blockIdx.x != 0) return;
    // block 0: the state in the layout of the other paths (active list and
    // shadow of the next step, event offsets, counters), as a finalize would
    Shadow *sh;
    if constexpr (F64) sh = d.sh64; else sh = d.sh32;
    const Shadow *last;
    if constexpr (F64) last = d.se_sh64[(k + 1) & 1]; else last = d.se_sh32[(k + 1) & 1];
    int *dst = d.act[cur ^ 1];
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int id = s_list[q];
        dst[q] = id;
        if constexpr (F64) sh[q] = ldcg_shadow64(last + id);  // written by other SMs
        else sh[q] = __ldcg(last + id);
    }
    if (threadIdx.x == 0) {
        d.ev_off[cur ^ 1][0] = 0;
        d.ev_off[cur ^ 1][1] = n;
        d.ev_collected_now[0] = 0;
        c->step = step;
        c->n_active = n;
        c->cur = cur ^ 1;
        c->carrier_steps += csteps;
        c->pair_interactions += pairs;
        c->work_counter = 0u;
    }
}

// ---- launch ------------------------------------------------------------------

const void *se_kernel_ptr(int precision, int R) {
    if (precision == 0) return (const void *)se_loop_kernel<1, false, true>;
#define GC_PICK(RR)                                                                        \
    if (R == RR) {                                                                         \
        if (precision == 1) return (const void *)se_loop_kernel<RR, false, false>;         \
        if (precision == 2) return (const void *)se_loop_kernel<RR, true, false>;          \
    }
    GC_PICK(2)
    GC_PICK(4)
    GC_PICK(8)
#undef GC_PICK
    return nullptr;
}

// The active list (dynamic) plus the static tiles exceed the default 48 KB
// per block: opt in to the larger dynamic size.
static cudaError_t se_prepare(const void *k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSEListBytes);
}

int se_occupancy(int precision, int R) {
    const void *k = se_kernel_ptr(precision, R);
    if (!k || se_prepare(k) != cudaSuccess) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kPairThreads, kSEListBytes) != cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t launch_se_loop(const Dev &d, int precision, int grid, double limit_s, cudaStream_t st) {
    const void *k = se_kernel_ptr(precision, d.shape.R);
    if (!k || grid < 1) return cudaErrorInvalidValue;
    cudaError_t e = se_prepare(k);
    if (e != cudaSuccess) return e;
    Dev dd = d;
    unsigned long long limit_ns = (unsigned long long)(limit_s * 1e9);
    void *args[] = {(void *)&dd, (void *)&limit_ns};
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kPairThreads), args, kSEListBytes, st);
}

// ---- self-test of the bounded barrier --------------------------------------------
// A barrier that waits for one block more than the grid has: nothing ever
// completes it, so every block must give up after limit_ns and report the
// timeout in the control block.
__device__ Ctrl g_selftest_ctrl;

__global__ void barrier_timeout_kernel(unsigned long long limit_ns) {
    __shared__ int s_ok;
    Ctrl *c = &g_selftest_ctrl;
    grid_barrier(&c->bar_count, &c->bar_gen, &c->error, gridDim.x + 1, limit_ns, &s_ok);
}

__global__ void selftest_reset_kernel() {
    g_selftest_ctrl.bar_count = 0u;
    g_selftest_ctrl.error = 0;
}

cudaError_t selftest_barrier_timeout(int grid, double limit_s, int *error_bits, cudaStream_t st) {
    selftest_reset_kernel<<<1, 1, 0, st>>>();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    unsigned long long limit_ns = (unsigned long long)(limit_s * 1e9);
    void *args[] = {(void *)&limit_ns};
    e = cudaLaunchCooperativeKernel((const void *)barrier_timeout_kernel, dim3(grid), dim3(128), args, 0, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyFromSymbolAsync(error_bits, g_selftest_ctrl, sizeof(int), offsetof(Ctrl, error),
                                  cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

}  // namespace gc
