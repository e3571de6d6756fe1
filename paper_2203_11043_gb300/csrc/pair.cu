// pair.cu -- the Eq. 6 all-pairs softened Coulomb sum (Sec. 3.2, Fig. 3).
//
// E_i = K sum_{j in event(i), active} (r_i - r_j) / (|r_i - r_j|^2 + eps^2)^(3/2)
//
// The paper tiles positions through shared memory (GPU Gems 3 ch. 31,
// Fig. 3: one thread per carrier, shPos tiles, __syncthreads between
// tiles).  This file keeps the tiling idea but is shaped for sm_103a:
//  * a persistent grid (one wave of resident blocks) pulls work items
//    (event, i-tile, j-chunk) from an atomic counter; items are ordered by
//    event, events by descending size (largest first), so thousands of
//    uneven events share one launch and one big event splits into
//    equal-cost items;
//  * each thread keeps R i-carriers in registers as R/2 packed FP32 pairs
//    and runs every step of the pair term on the f32x2 pipe path
//    (sub/fma/mul .f32x2), with the reciprocal square root on MUFU;
//  * j positions are staged in shared memory pre-duplicated as {x,x},{y,y},
//    {z,z} so one broadcast load feeds R/2 packed pairs;
//  * per-tile FP32 sums are folded into Kahan-compensated running sums
//    (FP32_KAHAN), and each item writes an FP64 partial per j-chunk; the
//    integrate kernel adds the chunks in a fixed order (deterministic);
//  * events smaller than `small_n` run 4 lanes per i-group that split the
//    j range and combine with warp shuffles, so small events keep the
//    block busy.
#include "gc_internal.cuh"
#include "gc_launch.h"

namespace gc {

// ---------------------------------------------------------------------------
// FP32 work item.  L lanes share one i-group; each thread owns R carriers.
template <int R, bool KAHAN, bool NEWTON, int L>
__device__ __forceinline__ void pair_item_fp32(const Dev &d, int e_start, int n_e, int local,
                                               ulonglong2 *__restrict__ s_xy,
                                               f2 *__restrict__ s_z) {
    constexpr int Q = R / 2;
    constexpr int G = 32 / L;                 // i-groups per warp
    constexpr int STRIDE = kPairThreads / L;  // distance between a thread's carriers
    constexpr int IB = R * STRIDE;            // carriers per i-tile
    constexpr int PER = kTileJ / kPairThreads;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane / L, ph = lane % L;
    const int jchunk = d.shape.jchunk;
    const int js = ceil_div(n_e, jchunk);
    const int it = local / js, jc = local - it * js;
    const int il0 = it * IB + warp * G + g;

    f2 xi[Q], yi[Q], zi[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float4 a = make_float4(kSentinel, kSentinel, kSentinel, 0.f), b = a;
        const int ia = il0 + (2 * q) * STRIDE, ib = il0 + (2 * q + 1) * STRIDE;
        if (ia < n_e) a = d.sh32[e_start + ia];
        if (ib < n_e) b = d.sh32[e_start + ib];
        xi[q] = pack2(a.x, b.x);
        yi[q] = pack2(a.y, b.y);
        zi[q] = pack2(a.z, b.z);
    }
    const float eps2f = (float)d.phys.eps2;
    const f2 EPS2 = pack2(eps2f, eps2f);
    const f2 ZERO = pack2(0.f, 0.f);
    f2 ax[Q], ay[Q], az[Q], sx[Q], sy[Q], sz[Q], cx[Q], cy[Q], cz[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        ax[q] = ay[q] = az[q] = ZERO;
        sx[q] = sy[q] = sz[q] = ZERO;
        cx[q] = cy[q] = cz[q] = ZERO;
    }

    const int j0 = jc * jchunk;
    const int j1 = min(n_e, j0 + jchunk);
    float4 pre[PER];
    auto fetch = [&](int jt) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int j = jt + u * kPairThreads + tid;
            pre[u] = j < j1 ? d.sh32[e_start + j] : make_float4(kSentinel, kSentinel, kSentinel, 0.f);
        }
    };
    fetch(j0);
    for (int jt = j0; jt < j1; jt += kTileJ) {
        __syncthreads();  // the previous tile has been consumed
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int k = u * kPairThreads + tid;
            s_xy[k] = make_ulonglong2(pack2(pre[u].x, pre[u].x), pack2(pre[u].y, pre[u].y));
            s_z[k] = pack2(pre[u].z, pre[u].z);
        }
        __syncthreads();
        const int cnt = min(kTileJ, j1 - jt);
        if (jt + kTileJ < j1) fetch(jt + kTileJ);  // overlaps the loads with this tile's work
        const int kmax = (cnt + 4 * L - 1) / (4 * L) * (4 * L);  // padded with sentinels
        for (int k0 = 0; k0 < kmax; k0 += 4 * L) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + u * L + ph;
                const ulonglong2 xy = s_xy[k];
                const f2 zz = s_z[k];
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const f2 dx = sub2(xi[q], xy.x);
                    const f2 dy = sub2(yi[q], xy.y);
                    const f2 dz = sub2(zi[q], zz);
                    f2 r2 = fma2(dx, dx, EPS2);
                    r2 = fma2(dy, dy, r2);
                    r2 = fma2(dz, dz, r2);
                    float ra, rb;
                    unpack2(r2, ra, rb);
                    f2 inv = pack2(rsqrt_mufu(ra), rsqrt_mufu(rb));
                    if (NEWTON) {  // y <- y (3/2 - r2 y^2 / 2)
                        const f2 nh = mul2(r2, pack2(-0.5f, -0.5f));
                        const f2 t = fma2(nh, mul2(inv, inv), pack2(1.5f, 1.5f));
                        inv = mul2(inv, t);
                    }
                    const f2 inv3 = mul2(mul2(inv, inv), inv);
                    ax[q] = fma2(dx, inv3, ax[q]);
                    ay[q] = fma2(dy, inv3, ay[q]);
                    az[q] = fma2(dz, inv3, az[q]);
                }
            }
        }
        if (KAHAN) {  // fold this tile's sums into the compensated totals
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                f2 y = sub2(ax[q], cx[q]), t = add2(sx[q], y);
                cx[q] = sub2(sub2(t, sx[q]), y); sx[q] = t; ax[q] = ZERO;
                y = sub2(ay[q], cy[q]); t = add2(sy[q], y);
                cy[q] = sub2(sub2(t, sy[q]), y); sy[q] = t; ay[q] = ZERO;
                y = sub2(az[q], cz[q]); t = add2(sz[q], y);
                cz[q] = sub2(sub2(t, sz[q]), y); sz[q] = t; az[q] = ZERO;
            }
        }
    }

    // Combine the L lanes of each i-group and write the chunk's FP64 partial.
    double *P = d.partial + (long long)jc * 3 * d.part_stride;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        double v[2][3];
        float lo, hi, clo, chi;
        if (KAHAN) {
            unpack2(sx[q], lo, hi); unpack2(cx[q], clo, chi);
            v[0][0] = (double)lo - (double)clo; v[1][0] = (double)hi - (double)chi;
            unpack2(sy[q], lo, hi); unpack2(cy[q], clo, chi);
            v[0][1] = (double)lo - (double)clo; v[1][1] = (double)hi - (double)chi;
            unpack2(sz[q], lo, hi); unpack2(cz[q], clo, chi);
            v[0][2] = (double)lo - (double)clo; v[1][2] = (double)hi - (double)chi;
        } else {
            unpack2(ax[q], lo, hi); v[0][0] = lo; v[1][0] = hi;
            unpack2(ay[q], lo, hi); v[0][1] = lo; v[1][1] = hi;
            unpack2(az[q], lo, hi); v[0][2] = lo; v[1][2] = hi;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int o = 1; o < L; o <<= 1) v[h][c] += __shfl_xor_sync(0xffffffffu, v[h][c], o);
            }
            const int il = il0 + (2 * q + h) * STRIDE;
            if (ph == 0 && il < n_e) {
                const long long p = e_start + il;
                P[p] = v[h][0];
                P[d.part_stride + p] = v[h][1];
                P[2 * d.part_stride + p] = v[h][2];
            }
        }
    }
}

// Largest event e with item_base[e] <= item (events without items are skipped
// because their base equals the next event's).
__device__ __forceinline__ int event_of_item(const int *__restrict__ base, int n_events, int item) {
    int lo = 0, hi = n_events;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (base[mid] <= item) lo = mid; else hi = mid;
    }
    return lo;
}

template <int R, bool KAHAN, bool NEWTON>
__global__ void __launch_bounds__(kPairThreads) pair_fp32_kernel(Dev d) {
    __shared__ ulonglong2 s_xy[kTileJ];
    __shared__ f2 s_z[kTileJ];
    __shared__ int s_item;
    Ctrl *c = d.ctrl;
    if (step_skipped(c)) return;
    const int *off = d.ev_off[c->cur];
    const int items = c->items_total;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&c->work_counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= items) break;
        const int e = event_of_item(d.item_base, d.n_events, item);
        const int e_start = off[e], n_e = off[e + 1] - e_start;
        const int local = item - d.item_base[e];
        if (lanes_for(n_e, d.shape.small_n) == 1)
            pair_item_fp32<R, KAHAN, NEWTON, 1>(d, e_start, n_e, local, s_xy, s_z);
        else
            pair_item_fp32<R, KAHAN, NEWTON, 4>(d, e_start, n_e, local, s_xy, s_z);
        __syncthreads();  // s_item and the tiles are reused by the next item
    }
}

// ---------------------------------------------------------------------------
// FP64 form: the plain per-carrier tiled sum in double precision (one
// carrier per thread, shared-memory tiles, j in ascending order inside the
// event), used as the reference form on the GPU.
__global__ void __launch_bounds__(kPairThreads) pair_fp64_kernel(Dev d) {
    constexpr int J = kPairThreads;
    __shared__ double s_x[J], s_y[J], s_z[J];
    __shared__ int s_item;
    Ctrl *c = d.ctrl;
    if (step_skipped(c)) return;
    const int *off = d.ev_off[c->cur];
    const int items = c->items_total;
    const double eps2 = d.phys.eps2;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&c->work_counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= items) break;
        const int e = event_of_item(d.item_base, d.n_events, item);
        const int e_start = off[e], n_e = off[e + 1] - e_start;
        const int local = item - d.item_base[e];
        const int js = ceil_div(n_e, d.shape.jchunk);
        const int it = local / js, jc = local - it * js;
        const int il = it * kPairThreads + threadIdx.x;
        double4_32a me = make_double4_32a(0, 0, 0, 0);
        if (il < n_e) me = d.sh64[e_start + il];
        double ex = 0.0, ey = 0.0, ez = 0.0;
        const int j0 = jc * d.shape.jchunk, j1 = min(n_e, j0 + d.shape.jchunk);
        for (int jt = j0; jt < j1; jt += J) {
            __syncthreads();
            const int j = jt + threadIdx.x;
            if (j < j1) {
                const double4_32a q = d.sh64[e_start + j];
                s_x[threadIdx.x] = q.x; s_y[threadIdx.x] = q.y; s_z[threadIdx.x] = q.z;
            }
            __syncthreads();
            const int cnt = min(J, j1 - jt);
            for (int k = 0; k < cnt; ++k) {
                const double rx = me.x - s_x[k], ry = me.y - s_y[k], rz = me.z - s_z[k];
                const double r2 = rx * rx + ry * ry + rz * rz + eps2;
                const double inv = 1.0 / (r2 * sqrt(r2));
                ex += rx * inv;
                ey += ry * inv;
                ez += rz * inv;
            }
        }
        if (il < n_e) {
            double *P = d.partial + (long long)jc * 3 * d.part_stride;
            const long long p = e_start + il;
            P[p] = ex;
            P[d.part_stride + p] = ey;
            P[2 * d.part_stride + p] = ez;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host-side launch table.
typedef void (*PairKernel)(Dev);

static PairKernel fp32_kernel(int R, bool kahan, bool newton) {
#define GC_PICK(RR)                                                                   \
    if (R == RR) {                                                                    \
        if (kahan) return newton ? pair_fp32_kernel<RR, true, true> : pair_fp32_kernel<RR, true, false>; \
        return newton ? pair_fp32_kernel<RR, false, true> : pair_fp32_kernel<RR, false, false>;         \
    }
    GC_PICK(2)
    GC_PICK(4)
    GC_PICK(8)
#undef GC_PICK
    return nullptr;
}

const void *pair_kernel_ptr(int precision, int R, int newton) {
    if (precision == 0) return (const void *)pair_fp64_kernel;
    if (precision == 1 || precision == 2)
        return (const void *)fp32_kernel(R, precision == 2, newton != 0);
    return nullptr;
}

int pair_kernel_occupancy(int precision, int R, int newton) {
    const void *k = pair_kernel_ptr(precision, R, newton);
    if (!k) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kPairThreads, 0) != cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t launch_pair(const Dev &d, int precision, int newton, cudaStream_t st) {
    const void *k = pair_kernel_ptr(precision, d.shape.R, newton);
    if (!k) return cudaErrorInvalidValue;
    ((PairKernel)k)<<<d.shape.n_blocks, kPairThreads, 0, st>>>(d);
    return cudaGetLastError();
}

}  // namespace gc
