// gc_pair.cuh -- the Eq. 6 all-pairs softened Coulomb sum (Sec. 3.2, Fig. 3):
// pair work items and the persistent pair kernels, included by pair.cu (the
// kernels of every step) and fused.cu (their fused small-workload variants).
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
//  * each thread keeps R i-carriers in registers, each duplicated as a
//    packed FP32 pair {x_i, x_i}, and pairs it with two j's at a time: every
//    step of the pair term runs as packed f32x2 instructions
//    (sub/fma/mul .f32x2) with the reciprocal square root on MUFU;
//  * j positions arrive by cp.async one tile ahead and are staged in shared
//    memory as SoA tiles, so one 16-byte broadcast load per coordinate feeds
//    four j's (two packed pairs) to every i of the thread;
//  * per-tile FP32 sums are folded into Kahan-compensated running sums
//    (FP32_KAHAN), and each item writes an FP64 partial per j-chunk; the
//    integrate kernel adds the chunks in a fixed order (deterministic);
//  * events smaller than `small_n` run 4 lanes per i-group that split the
//    j range and combine with warp shuffles, so small events keep the
//    block busy (16 lanes in the FP64 form).
#pragma once
#include "gc_internal.cuh"
#include "gc_slot.cuh"

namespace gc {

// ---------------------------------------------------------------------------
// FP32 work item, packed over j: each thread owns R i-carriers, each held
// duplicated as {x_i, x_i}; the shared tile is SoA (x[], y[], z[]) so one
// 16-byte load per coordinate brings four consecutive j's as two packed pairs
// {x_j, x_j+1}.  Each packed accumulator holds the even-j and odd-j sums of
// one i; the Kahan state of the cross-tile sums stays in registers.  L lanes
// share an i-group and split the j range.
//
// H16 (the FP16x2 form): coordinates are multiplied by the event's
// power-of-two scale s (exact), the differences are rounded to f16x2 and
// r^2 s^2 is formed with packed half FMAs; the reciprocal square root and the
// accumulation stay FP32 and the sum is multiplied by s^2 at the end.
//
// Tile frames (TF; large events, one lane per i-group): the shadow of a hole
// is relative to the FP64 origin of its 256-slot tile, held as an FP32 hi + lo
// pair.  An item works in the frame I of its first i-tile: each i and, while
// a j-tile is staged, each j is moved into I by adding (hi_t - hi_I) +
// (lo_t - lo_I) for its own tile t.  The i's are shifted once per item (they
// stay loop-invariant, as in the event frame), both sides use the same
// expression, so a hole's self term stays exactly 0, and differences of close
// holes are taken between small FP32 numbers.  The j-tile origins reach
// shared memory (s_fr) by cp.async with the tile before.  s_fr is written by
// other threads, so it is not a restrict pointer.
// LIST (the persistent single-event kernel): the event's shadow `shb` is
// indexed by hole id, list[slot] in shared memory; otherwise shb = sh32 +
// e_start is indexed by slot.
// JUH (one lane per i-group only): 1 halves the 16-byte loads in flight per
// coordinate (an autotuner variant; the per-carrier sum order is unchanged).
template <int R, bool KAHAN, bool NEWTON, int L, bool H16, bool TF, bool LIST = false, int JUH = 0>
__device__ __forceinline__ void pair_item_fp32_j(const Dev &d, int e_start, int n_e, int local,
                                                 float scale, float *__restrict__ sx,
                                                 float *__restrict__ sy, float *__restrict__ sz,
                                                 float4 *s_fr, float4 *s_raw,
                                                 const float4 *__restrict__ shb,
                                                 const int *list = nullptr) {
    constexpr int G = 32 / L;
    constexpr int STRIDE = kPairThreads / L;
    constexpr int IB = R * STRIDE;
    // j positions per shared-memory tile (a multiple of the 256-slot frame
    // tile): tile frames need one frame per staged tile; otherwise longer tiles
    // amortise the barriers (4 lanes split a tile, so the 4-lane path takes 4
    // tiles' worth).  Measured on 4096 X-ray events: +3.4 % for the 4-lane path.
    constexpr int TJ = L == 1 ? (TF ? kTileJ : 2 * kTileJ) : 4 * kTileJ;
    constexpr int PER = TJ / kPairThreads;
    // 16-byte loads (4 j's) per coordinate per iteration: about 16 packed
    // pair chains in flight per lane (R * JU * 2 = 16 on one lane; the 4-lane
    // path measured best at 4 for R = 2, against 2 and 8)
    constexpr int JU0 = L == 1 ? (R >= 8 ? 1 : 8 / R) : 4;
    constexpr int JU = (L == 1 && JUH) ? (JU0 > 1 ? JU0 / 2 : 1) : JU0;
    constexpr int STEP = 4 * JU * L;  // j's consumed per unrolled iteration by the L lanes
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane / L, ph = lane % L;
    const int jchunk = d.shape.jchunk;
    const int js = ceil_div(n_e, jchunk);
    const int it = local / js, jc = local - it * js;
    const int il0 = it * IB + warp * G + g;

    f2 xi[R], yi[R], zi[R], ax[R], ay[R], az[R];
    const f2 ZERO = pack2(0.f, 0.f);
    f2 kreg[KAHAN ? 6 * R : 1];  // Kahan sums and compensations, {even, odd} j
    float4 Ih = make_float4(0.f, 0.f, 0.f, 0.f), Il = Ih;  // tile frames: the item frame I
    if (TF) {
        Ih = d.frame_hi[e_start + it * IB];  // it * IB is a tile start
        Il = d.frame_lo[e_start + it * IB];
        if (tid < 2) s_fr[tid] = tid ? Il : Ih;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float4 a = make_float4(kSentinel, kSentinel, kSentinel, 0.f);
        const int ia = il0 + r * STRIDE;
        if (ia < n_e) {
            a = LIST ? __ldcg(shb + list[ia]) : shb[ia];  // LIST: written by other SMs in this launch
            if (TF) {  // into the item frame
                const int t = e_start + (ia & ~(kTileJ - 1));
                const float4 th = d.frame_hi[t], tl = d.frame_lo[t];
                a.x = a.x + ((th.x - Ih.x) + (tl.x - Il.x));
                a.y = a.y + ((th.y - Ih.y) + (tl.y - Il.y));
                a.z = a.z + ((th.z - Ih.z) + (tl.z - Il.z));
            }
        }
        if (H16) {
            a.x *= scale;
            a.y *= scale;
            a.z *= scale;
        }
        xi[r] = pack2(a.x, a.x);
        yi[r] = pack2(a.y, a.y);
        zi[r] = pack2(a.z, a.z);
        ax[r] = ay[r] = az[r] = ZERO;
        if (KAHAN) {
#pragma unroll
            for (int c = 0; c < 6; ++c) kreg[r * 6 + c] = ZERO;
        }
    }
    const float eps2f = (float)d.phys.eps2 * (H16 ? scale * scale : 1.0f);
    const f2 EPS2 = pack2(eps2f, eps2f);
    const unsigned EPS2H = f2_to_h2(EPS2);

    const int j0 = jc * jchunk;
    const int j1 = min(n_e, j0 + jchunk);
    float4 *s_fj = s_fr + 2;  // j-tile frames (hi, lo), double-buffered by tile parity
    // The next j-tile goes by cp.async into this thread's own landing slots
    // (s_raw[u * 128 + tid], zero-filled past j1); at the tile start each
    // thread moves its own slots into the SoA tile, so s_raw needs no barrier.
    auto fetch = [&](int jt) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int j = jt + u * kPairThreads + tid;
            const int jj = j < j1 ? j : j0;
            cp_async16_zfill(s_raw + u * kPairThreads + tid, shb + (LIST ? (int)list[jj] : jj),
                             j < j1 ? 16u : 0u);
        }
        if (TF && tid < 2)  // jt is a tile start (j-chunks are whole tiles)
            cp_async16(s_fj + 2 * ((jt / TJ) & 1) + tid,
                       (tid ? d.frame_lo : d.frame_hi) + e_start + jt);
    };
    fetch(j0);
    for (int jt = j0; jt < j1; jt += TJ) {
        cp_async_wait_all();  // this thread's slots of the tile (and the tile's frame) have landed
        __syncthreads();      // the previous tile has been consumed
        float ox = 0.f, oy = 0.f, oz = 0.f;
        if (TF) {  // this j-tile's frame relative to the item frame
            const int b = 2 * ((jt / TJ) & 1);
            const float4 th = s_fj[b], tl = s_fj[b + 1], ih = s_fr[0], il = s_fr[1];
            ox = (th.x - ih.x) + (tl.x - il.x);
            oy = (th.y - ih.y) + (tl.y - il.y);
            oz = (th.z - ih.z) + (tl.z - il.z);
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int k = u * kPairThreads + tid;
            const float sc = H16 ? scale : 1.0f;  // exact (power of two)
            float4 v = s_raw[k];
            if (jt + k >= j1) v = make_float4(kSentinel, kSentinel, kSentinel, 0.f);
            if (TF) {
                sx[k] = (v.x + ox) * sc;
                sy[k] = (v.y + oy) * sc;
                sz[k] = (v.z + oz) * sc;
            } else {
                sx[k] = v.x * sc;
                sy[k] = v.y * sc;
                sz[k] = v.z * sc;
            }
        }
        __syncthreads();
        const int cnt = min(TJ, j1 - jt);
        if (jt + TJ < j1) fetch(jt + TJ);  // overlaps the loads with this tile's work
        const int kmax = (cnt + STEP - 1) / STEP * STEP;  // padded with sentinels
        auto j_step = [&](const int k0) {  // 4 * JU j's per lane: two packed pairs per load
#pragma unroll
            for (int u = 0; u < JU; ++u) {
                const int k = k0 + u * 4 * L;
                const ulonglong2 X = *reinterpret_cast<const ulonglong2 *>(sx + k);
                const ulonglong2 Y = *reinterpret_cast<const ulonglong2 *>(sy + k);
                const ulonglong2 Z = *reinterpret_cast<const ulonglong2 *>(sz + k);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const f2 xj = h ? X.y : X.x, yj = h ? Y.y : Y.x, zj = h ? Z.y : Z.x;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const f2 dx = sub2(xi[r], xj);
                        const f2 dy = sub2(yi[r], yj);
                        const f2 dz = sub2(zi[r], zj);
                        float ra, rb;
                        f2 r2;
                        if (H16) {
                            const unsigned hx = f2_to_h2(dx), hy = f2_to_h2(dy), hz = f2_to_h2(dz);
                            unsigned h = hfma2(hx, hx, EPS2H);
                            h = hfma2(hy, hy, h);
                            h = hfma2(hz, hz, h);
                            h2_to_f(h, ra, rb);
                            r2 = pack2(ra, rb);
                        } else {
                            r2 = fma2(dx, dx, EPS2);
                            r2 = fma2(dy, dy, r2);
                            r2 = fma2(dz, dz, r2);
                            unpack2(r2, ra, rb);
                        }
                        f2 inv = pack2(rsqrt_mufu(ra), rsqrt_mufu(rb));
                        if (NEWTON) {  // y <- y (3/2 - r2 y^2 / 2)
                            const f2 nh = mul2(r2, pack2(-0.5f, -0.5f));
                            const f2 t = fma2(nh, mul2(inv, inv), pack2(1.5f, 1.5f));
                            inv = mul2(inv, t);
                        }
                        const f2 inv3 = mul2(mul2(inv, inv), inv);
                        ax[r] = fma2(dx, inv3, ax[r]);
                        ay[r] = fma2(dy, inv3, ay[r]);
                        az[r] = fma2(dz, inv3, az[r]);
                    }
                }
            }
        };
        if (TF) {  // measured: unrolling by 2 suits the tile-frame variant, not the other
#pragma unroll 2
            for (int k0 = 4 * ph; k0 < kmax; k0 += STEP) j_step(k0);
        } else {
            for (int k0 = 4 * ph; k0 < kmax; k0 += STEP) j_step(k0);
        }
        if (KAHAN) {  // fold this tile's sums into the compensated totals
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const f2 acc[3] = {ax[r], ay[r], az[r]};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const f2 s0 = kreg[r * 6 + 2 * c], c0 = kreg[r * 6 + 2 * c + 1];
                    const f2 y = sub2(acc[c], c0), t = add2(s0, y);
                    kreg[r * 6 + 2 * c + 1] = sub2(sub2(t, s0), y);
                    kreg[r * 6 + 2 * c] = t;
                }
                ax[r] = ay[r] = az[r] = ZERO;
            }
        }
    }

    // Combine the even/odd halves and the L lanes of each i-group in FP32 (a few
    // roundings of the item's sum, within the FP32 bound of the Kahan sums: on
    // GB300 an FP64 combination costs more FP64-unit time per item than a small
    // event's pair work), then write the FP64 partial (an exact conversion).
    double *P = d.partial + (long long)jc * 3 * d.part_stride;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float lo, hi;
            if (KAHAN) {
                float clo, chi;
                unpack2(kreg[r * 6 + 2 * c], lo, hi);
                unpack2(kreg[r * 6 + 2 * c + 1], clo, chi);
                v[c] = (lo - clo) + (hi - chi);
            } else {
                unpack2(c == 0 ? ax[r] : (c == 1 ? ay[r] : az[r]), lo, hi);
                v[c] = lo + hi;
            }
            if (H16) v[c] *= scale * scale;  // a power of two: exact
#pragma unroll
            for (int o = 1; o < L; o <<= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
        }
        const int il = il0 + r * STRIDE;
        if (ph == 0 && il < n_e && GC_GUARD(e_start + il < d.n_total)) {
            const long long p = e_start + il;
            P[p] = f2d_exact(v[0]);
            P[d.part_stride + p] = f2d_exact(v[1]);
            P[2 * d.part_stride + p] = f2d_exact(v[2]);
        }
    }
}

// Fused small-workload path, after one pair item: the block's partial-sum
// stores are released by thread 0, which counts the item on its i-tile's ticket, and the
// item that brings the ticket to the number of j-chunks integrates the
// i-tile's carriers (reading the partials through L2) and writes their keep
// bytes.  The ticket is reset for the next step by that item.  No block ever
// waits for another: whichever block finishes an i-tile's last chunk does it.
template <bool F64>
__device__ __forceinline__ void fused_tile_done(const Dev &d, int e, int e_start, int n_e, int local,
                                                int cur, long long step, int *s_flag) {
    const int itile = itile_for(d.shape.R, lanes_for(d.shape, n_e));
    const int js = ceil_div(n_e, d.shape.jchunk);
    const int it = local / js;
    __syncthreads();  // the block's partial sums before thread 0's release
    if (threadIdx.x == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        unsigned *t = d.tile_ticket + d.tile_base[e] + it;
        const unsigned done = atomicAdd(t, 1u);
        const int last = done == (unsigned)(js - 1);
        if (last) {
            *t = 0u;
            asm volatile("fence.acq_rel.gpu;" ::: "memory");  // acquire: the other items' partial sums
        }
        *s_flag = last;
    }
    __syncthreads();
    if (*s_flag) {
        const int i1 = min(n_e, (it + 1) * itile);
        for (int q = it * itile + (int)threadIdx.x; q < i1; q += blockDim.x) {
            const int p = e_start + q;
            d.keep8[p] = advance_slot<F64, false, true>(d, cur, p, step) ? 1 : 0;
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

// Min blocks = 1 lets ptxas keep many independent pair chains in registers
// (R = 4: ~240 registers, 2 blocks per SM); measured faster than letting it
// trade registers for occupancy.
// TF: the tile-frame variant (used when some event is large enough for one
// lane per i-group); its small events still run the event-frame path.
// FUSED (small workloads, FP32 forms without Newton step or tile frames):
// after each item, the item that completes its i-tile's j-chunks integrates
// that i-tile (fused_tile_done), so one launch does the pair sum and the
// per-carrier step; the one-block small_tail kernel then compacts.
// Autotuner variants V of the unfused FP32 kernel (the arithmetic per carrier
// is the same in all of them, so they give the same bits): 0 = the default;
// 1 = half the loads in flight on one lane; 2 = a register budget for one
// more resident block per SM (4 at R = 2, 3 at R = 4).
__host__ __device__ constexpr int pair_min_blocks(int R, int V) { return V == 2 ? (R == 2 ? 4 : 3) : 1; }

template <int R, bool KAHAN, bool NEWTON, bool H16, bool TF, bool FUSED, int V = 0>
__global__ void __launch_bounds__(kPairThreads, pair_min_blocks(R, V)) pair_fp32_kernel(Dev d) {
    __shared__ __align__(16) float s_x[4 * kTileJ], s_y[4 * kTileJ], s_z[4 * kTileJ];
    __shared__ float4 s_fr[TF ? 6 : 1];  // tile frames: the item frame, then two j-tile frames
    __shared__ __align__(16) float4 s_raw[4 * kTileJ];  // cp.async landing slots of the next j-tile
    __shared__ int s_item, s_flag;
    Ctrl *c = d.ctrl;
    if (step_skipped(c)) return;
    const int cur = c->cur;
    const int *off = d.ev_off[cur];
    const unsigned *ext = H16 ? d.ev_ext[cur] : nullptr;
    const int items = c->items_total;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&c->work_counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= items) break;
        const int e = event_of_item(d.item_base, d.n_events, item);
        const int e_start = off[e], n_e = off[e + 1] - e_start;
        const int local = item - d.item_base[e];
        const float scale = H16 ? h2_scale(__uint_as_float(ext[e])) : 1.0f;
        if (lanes_for(d.shape, n_e) == 1)
            pair_item_fp32_j<R, KAHAN, NEWTON, 1, H16, TF, false, V == 1>(d, e_start, n_e, local, scale, s_x,
                                                                          s_y, s_z, s_fr, s_raw, d.sh32 + e_start);
        else
            pair_item_fp32_j<R, KAHAN, NEWTON, 4, H16, false>(d, e_start, n_e, local, scale, s_x, s_y,
                                                              s_z, s_fr, s_raw, d.sh32 + e_start);
        if constexpr (FUSED) fused_tile_done<false>(d, e, e_start, n_e, local, cur, c->step + 1, &s_flag);
        __syncthreads();  // s_item and the tiles are reused by the next item
    }
}

// ---------------------------------------------------------------------------
// FP64 form: the plain tiled sum in double precision (shared-memory j tiles,
// j in ascending order inside a j-chunk), used as the reference form on the
// GPU.  Large events: one carrier per thread.  Small events (FP64 is a small
// fraction of the FP32 rate on this GPU, so a few i-tiles would keep most SMs
// idle): L = 16 lanes per carrier split each j-tile and combine with a fixed
// xor-shuffle tree, 8 carriers per item, so the work spreads over the GPU.
// An FP64 shadow entry read through L2 (two 16-byte loads).
__device__ __forceinline__ double4_32a ldcg_shadow64(const double4_32a *p) {
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    return make_double4_32a(a.x, a.y, b.x, b.y);
}

template <int L, bool LIST = false>
__device__ __forceinline__ void pair_item_fp64(const Dev &d, int e_start, int n_e, int local,
                                               double *__restrict__ s_x, double *__restrict__ s_y,
                                               double *__restrict__ s_z,
                                               const double4_32a *__restrict__ shb,
                                               const int *list = nullptr) {
    constexpr int J = kPairThreads;      // j positions per shared tile
    constexpr int G = kPairThreads / L;  // carriers per item
    const int tid = threadIdx.x;
    const int g = tid / L, ph = tid - g * L;  // the L lanes of a carrier are adjacent in one warp
    const int jchunk = d.shape.jchunk;
    const int js = ceil_div(n_e, jchunk);
    const int it = local / js, jc = local - it * js;
    const int il = it * G + g;
    double4_32a me = make_double4_32a(0, 0, 0, 0);
    if (il < n_e) me = LIST ? ldcg_shadow64(shb + list[il]) : shb[il];
    const double eps2 = d.phys.eps2;
    double ex = 0.0, ey = 0.0, ez = 0.0;
    const int j0 = jc * jchunk, j1 = min(n_e, j0 + jchunk);
    for (int jt = j0; jt < j1; jt += J) {
        __syncthreads();
        const int j = jt + tid;
        if (j < j1) {
            const double4_32a q = LIST ? ldcg_shadow64(shb + list[j]) : shb[j];
            s_x[tid] = q.x; s_y[tid] = q.y; s_z[tid] = q.z;
        }
        __syncthreads();
        const int cnt = min(J, j1 - jt);
        for (int k = ph; k < cnt; k += L) {
            const double rx = me.x - s_x[k], ry = me.y - s_y[k], rz = me.z - s_z[k];
            const double r2 = rx * rx + ry * ry + rz * rz + eps2;
            const double inv = 1.0 / (r2 * sqrt(r2));
            ex += rx * inv;
            ey += ry * inv;
            ez += rz * inv;
        }
    }
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
        ex += __shfl_xor_sync(0xffffffffu, ex, o);
        ey += __shfl_xor_sync(0xffffffffu, ey, o);
        ez += __shfl_xor_sync(0xffffffffu, ez, o);
    }
    if (ph == 0 && il < n_e && GC_GUARD(e_start + il < d.n_total)) {
        double *P = d.partial + (long long)jc * 3 * d.part_stride;
        const long long p = e_start + il;
        P[p] = ex;
        P[d.part_stride + p] = ey;
        P[2 * d.part_stride + p] = ez;
    }
}

template <bool FUSED>
__global__ void __launch_bounds__(kPairThreads) pair_fp64_kernel(Dev d) {
    __shared__ double s_x[kPairThreads], s_y[kPairThreads], s_z[kPairThreads];
    __shared__ int s_item, s_flag;
    Ctrl *c = d.ctrl;
    if (step_skipped(c)) return;
    const int cur = c->cur;
    const int *off = d.ev_off[cur];
    const int items = c->items_total;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&c->work_counter, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= items) break;
        const int e = event_of_item(d.item_base, d.n_events, item);
        const int e_start = off[e], n_e = off[e + 1] - e_start;
        const int local = item - d.item_base[e];
        if (lanes_for(d.shape, n_e) == 1)
            pair_item_fp64<1>(d, e_start, n_e, local, s_x, s_y, s_z, d.sh64 + e_start);
        else
            pair_item_fp64<16>(d, e_start, n_e, local, s_x, s_y, s_z, d.sh64 + e_start);
        if constexpr (FUSED) fused_tile_done<true>(d, e, e_start, n_e, local, cur, c->step + 1, &s_flag);
        __syncthreads();
    }
}

}  // namespace gc
