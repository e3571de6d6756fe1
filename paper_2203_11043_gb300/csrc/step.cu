// step.cu -- everything in one time step after the Eq. 6 pair sum (Fig. 2):
//
//  integrate:  E = E_Coul + (0, 0, a1 z - a2) (Eq. 1), |E|, mu(|E|, T) (Eq. 2),
//              v = mu E, D = mu kT/q (Eq. 4), sigma = sqrt(2 D dt) (Eq. 3),
//              Philox-4x32-10 + Box-Muller normals, r += v dt + sigma n (FP64),
//              reflection at the back surface, the z check (collection at
//              z <= z_well), exact integer binning into the event's image
//              (Fig. 5), and a warp-ballot keep mask per 32 slots.
//  compact:    stable stream compaction of the active list (ballot masks ->
//              popc prefix inside a 4096-slot chunk -> prefix over chunks),
//              writing the next step's id list and FP32 / FP64 shadow.
//  finalize:   one block: per-event active counts, new event offsets,
//              pair work items, step and throughput counters, termination.
//
// No kernel waits on another block: ordering comes from the stream (or the
// captured graph), so nothing here can spin.
#include "gc_internal.cuh"
#include "gc_launch.h"
#include "gc_slot.cuh"

namespace gc {

// ---- FP32 position shadow with tile frames -------------------------------------------------------
// Runs after finalize when tile frames are on (the new active list and event
// offsets are current; without tile frames the compaction writes the shadow).
// Events with at least small_n active holes (the ones whose pair items run
// one lane per i-group) get tile frames: slot q of event e (start e0) is
// stored relative to the FP64 position of the hole in slot
// e0 + ((q - e0) rounded down to 256), so the FP32 coordinates of spatially
// close holes (load-time Morton order) stay small; that origin is stored at
// the tile start as an FP32 hi + lo pair.  Smaller events use the event
// centroid.  It also measures the FP16x2 extents (max |r - centroid|).
// Rebuilding from the current state is idempotent, so it needs no skip flag.
__global__ void __launch_bounds__(256) shadow_kernel(Dev d) {
    Ctrl *c = d.ctrl;
    const int n = c->n_active;
    if (n <= 0 || c->error) return;
    const int cur = c->cur;
    const int *act = d.act[cur];
    const int *off = d.ev_off[cur];
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    const int n_round = (n + 31) / 32 * 32;  // whole warps stay in the loop
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_round; q += stride) {
        const bool valid = q < n;
        int e = -1;
        unsigned ext_bits = 0u;
        if (valid) {
            const int id = act[q];
            e = d.ev_of_id[id];
            const int e0 = off[e], ne = off[e + 1] - e0;
            const double x = d.px[id], y = d.py[id], z = d.pz[id];
            const double cx = d.ev_origin[3 * e], cy = d.ev_origin[3 * e + 1], cz = d.ev_origin[3 * e + 2];
            double ox = cx, oy = cy, oz = cz;
            if (d.tile_frames && ne >= d.shape.small_n) {
                const int rs = e0 + ((q - e0) & ~(kTileJ - 1));
                const int rid = act[rs];
                ox = d.px[rid];
                oy = d.py[rid];
                oz = d.pz[rid];
                if (q == rs) {
                    const float hx = (float)ox, hy = (float)oy, hz = (float)oz;
                    d.frame_hi[q] = make_float4(hx, hy, hz, 0.f);
                    d.frame_lo[q] = make_float4((float)(ox - hx), (float)(oy - hy), (float)(oz - hz), 0.f);
                }
            }
            d.sh32[q] = make_float4(d2f_exact(x - ox), d2f_exact(y - oy), d2f_exact(z - oz), 1.0f);
            if (d.ev_ext[0])
                ext_bits = __float_as_uint(fmaxf(fabsf((float)(x - cx)),
                                                 fmaxf(fabsf((float)(y - cy)), fabsf((float)(z - cz)))));
        }
        if (d.ev_ext[0]) {  // FP16x2 form: per-event max |r - centroid|, warp-aggregated
            unsigned *ext = d.ev_ext[cur];
            const unsigned lead = __ffs(__ballot_sync(0xffffffffu, valid));
            if (lead) {
                const int e0 = __shfl_sync(0xffffffffu, e, lead - 1);
                if (__all_sync(0xffffffffu, !valid || e == e0)) {
                    const unsigned mx = __reduce_max_sync(0xffffffffu, ext_bits);
                    if (lane == 0) atomicMax(&ext[e0], mx);
                } else if (valid) {
                    atomicMax(&ext[e], ext_bits);
                }
            }
        }
    }
}

// One block per event: the occupied pixels of its image in index order, for
// the stored-charge field of this step.  Each thread takes 8 consecutive
// pixels of a 8192-pixel span; one block-wide exclusive scan of the per-thread
// counts places them.
constexpr int kOccPer = 8;
__global__ void __launch_bounds__(kChunkThreads) occupied_pixels_kernel(Dev d) {
    __shared__ long long s_warp[33];
    Ctrl *c = d.ctrl;
    if (step_skipped(c)) return;
    const int npix = d.phys.img_w * d.phys.img_h;
    constexpr int SPAN = kOccPer * kChunkThreads;
    for (int e = blockIdx.x; e < d.n_events; e += gridDim.x) {
        const unsigned *img = d.image + (long long)d.ev_user[e] * npix;
        int *out = d.occ_pix + d.occ_off[e];
        const int cap = d.occ_off[e + 1] - d.occ_off[e];
        long long base = 0;
        for (int b0 = 0; b0 < npix; b0 += SPAN) {
            const int first = b0 + threadIdx.x * kOccPer;
            unsigned bits = 0u;
#pragma unroll
            for (int k = 0; k < kOccPer; ++k)
                if (first + k < npix && img[first + k] != 0u) bits |= 1u << k;
            long long total;
            const long long ex = block_exclusive_scan((long long)__popc(bits), s_warp, total);
            long long k_out = base + ex;
#pragma unroll
            for (int k = 0; k < kOccPer; ++k)
                if ((bits >> k) & 1u) {
                    if (k_out < cap) {
                        const int pidx = first + k;
                        out[k_out] = pidx;
                        d.occ_q[d.occ_off[e] + k_out] = img[pidx];
                        const int iy = pidx / d.phys.img_w, ix = pidx - iy * d.phys.img_w;
                        d.occ_f4[d.occ_off[e] + k_out] = make_float4(
                            (float)(d.img_origin[2 * e] + (ix + 0.5) * d.phys.pixel - d.ev_origin[3 * e]),
                            (float)(d.img_origin[2 * e + 1] + (iy + 0.5) * d.phys.pixel - d.ev_origin[3 * e + 1]),
                            (float)img[pidx], 0.0f);
                    }
                    ++k_out;
                }
            base += total;
        }
        if (threadIdx.x == 0) d.occ_cnt[e] = (int)(base < cap ? base : (long long)cap);
        __syncthreads();
    }
}

// FIELD = false: no Coulomb or stored-charge field (the O(N) path).
template <bool F64, bool INIT, bool FIELD>
__global__ void __launch_bounds__(kChunkThreads) integrate_kernel(Dev d) {
    __shared__ int s_cnt[kChunkThreads / 32];
    Ctrl *c = d.ctrl;
    if (step_skipped(c)) return;
    const int cur = c->cur;
    const int n_act = c->n_active;
    const long long step = INIT ? 0 : c->step + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (d.ev_ext[0]) {  // FP16x2 form: the compaction below measures the new extents
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.n_events; e += gridDim.x * blockDim.x)
            d.ev_ext[cur ^ 1][e] = 0u;
    }
    const int nchunks = ceil_div(n_act, kChunk);
    const bool fine = fine_units(n_act);  // uniform over the grid
    const int per_chunk = fine ? kChunk / kFineUnit : 1;
    for (int u = blockIdx.x; u < nchunks * per_chunk; u += gridDim.x) {
        const int ch = u / per_chunk;
        int kept = 0;
        if (fine) {  // one slot per thread of the first kFineUnit threads
            if (threadIdx.x < kFineUnit) {
                const int p = ch * kChunk + (u - ch * per_chunk) * kFineUnit + threadIdx.x;
                const bool keep = p < n_act ? advance_slot<F64, INIT, false, FIELD>(d, cur, p, step) : false;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (lane == 0) d.keepmask[p >> 5] = m;
                kept = __popc(m);
            }
        } else {
#pragma unroll
            for (int k = 0; k < kChunk / kChunkThreads; ++k) {
                const int p = ch * kChunk + k * kChunkThreads + threadIdx.x;
                const bool keep = p < n_act ? advance_slot<F64, INIT, false, FIELD>(d, cur, p, step) : false;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (lane == 0) d.keepmask[p >> 5] = m;
                kept += __popc(m);
            }
        }
        if (lane == 0) s_cnt[warp] = kept;
        __syncthreads();
        if (warp == 0) {
            int v = s_cnt[lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) {
                if (fine) atomicAdd(&d.chunk_cnt[ch], v);
                else d.chunk_cnt[ch] = v;
            }
        }
        __syncthreads();
    }
}

// ---- compaction ---------------------------------------------------------------------------
template <bool F64>
__global__ void __launch_bounds__(kChunkThreads) compact_kernel(Dev d) {
    constexpr int WORDS = kChunk / 32;  // 128 mask words per chunk
    __shared__ int s_wpre[WORDS];
    __shared__ int s_wtot[WORDS / 32];
    __shared__ int s_red[kChunkThreads / 32];
    __shared__ int s_base;
    Ctrl *c = d.ctrl;
    if (step_skipped(c)) return;
    const int cur = c->cur;
    const int n_act = c->n_active;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int *src = d.act[cur];
    int *dst = d.act[cur ^ 1];
    const int nchunks = ceil_div(n_act, kChunk);
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        // kept slots in all earlier chunks
        int acc = 0;
        for (int k = threadIdx.x; k < ch; k += kChunkThreads) acc += d.chunk_cnt[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_red[warp] = acc;
        // exclusive prefix of the chunk's mask-word popcounts (warps 0..3)
        if (threadIdx.x < WORDS) {
            const int wc = __popc(d.keepmask[(long long)ch * WORDS + threadIdx.x]);
            int incl = wc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            s_wpre[threadIdx.x] = incl - wc;  // exclusive within the warp
            if (lane == 31) s_wtot[warp] = incl;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int b = 0;
            for (int w = 0; w < kChunkThreads / 32; ++w) b += s_red[w];
            s_base = b;
        }
        if (threadIdx.x < WORDS && warp > 0) {
            int add = 0;
            for (int w = 0; w < warp; ++w) add += s_wtot[w];
            s_wpre[threadIdx.x] += add;
        }
        __syncthreads();
        const int base = s_base;
#pragma unroll
        for (int k = 0; k < kChunk / kChunkThreads; ++k) {
            const int p = ch * kChunk + k * kChunkThreads + threadIdx.x;
            const int m = k * (kChunkThreads / 32) + warp;
            const unsigned w = d.keepmask[(long long)ch * WORDS + m];
            const bool keep = (w >> lane) & 1u;
            int e = -1;
            unsigned ext_bits = 0u;
            // ok: kept and (GC_DEBUG) its slot, target slot and id in range;
            // every lane still reaches the warp-wide vote below
            bool ok = keep && GC_GUARD(p < d.n_total);
            const int q = base + s_wpre[m] + __popc(w & ((1u << lane) - 1u));
            const int id = ok ? src[p] : 0;
            ok = ok && GC_GUARD(q >= 0 && q < d.n_total && id >= 0 && id < d.n_total);
            if (ok) {
                dst[q] = id;
                // the shadow in the event frame (with tile frames the FP32 shadow
                // is written by shadow_kernel once the new event offsets are known)
                if (d.phys.coulomb || d.phys.stored) {  // the O(N) path reads no shadow
                    e = d.ev_of_id[id];
                    const double ox = d.ev_origin[3 * e], oy = d.ev_origin[3 * e + 1],
                                 oz = d.ev_origin[3 * e + 2];
                    if (F64) {
                        d.sh64[q] = make_double4_32a(d.px[id] - ox, d.py[id] - oy, d.pz[id] - oz, 0.0);
                    } else if (!d.tile_frames) {
                        const float4 v = make_float4(d2f_exact(d.px[id] - ox), d2f_exact(d.py[id] - oy),
                                                     d2f_exact(d.pz[id] - oz), 1.0f);
                        d.sh32[q] = v;
                        ext_bits = __float_as_uint(fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z))));
                    }
                }
            }
            if (!F64 && !d.tile_frames && d.ev_ext[0] && (d.phys.coulomb || d.phys.stored)) {
                unsigned *ext = d.ev_ext[cur ^ 1];  // FP16x2: max |coordinate|, warp-aggregated
                const unsigned lead = __ffs(__ballot_sync(0xffffffffu, ok));
                if (lead) {
                    const int e0 = __shfl_sync(0xffffffffu, e, lead - 1);
                    if (__all_sync(0xffffffffu, !ok || e == e0)) {
                        const unsigned mx = __reduce_max_sync(0xffffffffu, ext_bits);
                        if (lane == 0) atomicMax(&ext[e0], mx);
                    } else if (ok) {
                        atomicMax(&ext[e], ext_bits);
                    }
                }
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int items_for(const Dev &d, int n) {
    if (n <= 0 || !d.phys.coulomb) return 0;
    const int L = lanes_for(d.shape, n);
    return ceil_div(n, itile_for(d.shape.R, L)) * ceil_div(n, d.shape.jchunk);
}
__device__ __forceinline__ int tiles_for(const Dev &d, int n) {
    if (n <= 0 || !d.phys.coulomb) return 0;
    return ceil_div(n, itile_for(d.shape.R, lanes_for(d.shape, n)));
}

// One block (any multiple of 32 threads): per-event active counts after this
// step's collections, the new event offsets, the pair work items and i-tiles
// of the next step (prefix over events), the step and throughput counters,
// and the flip of the double-buffered lists.
template <bool INIT>
__device__ __forceinline__ void finalize_block(const Dev &d, long long *s_warp) {
    Ctrl *c = d.ctrl;
    const int cur = c->cur;
    const int *off = d.ev_off[cur];
    int *noff = d.ev_off[cur ^ 1];
    // The active event offsets (and this step's collections) are checked as
    // they are read: an inconsistency sets kErrOffsets before anything they
    // size is written (chunk counters, the control block); every later kernel
    // then skips its step.  The prefixes written meanwhile (next buffers,
    // one entry per event) are then never used.
    int bad = 0;
    if (threadIdx.x == 0 && (off[0] != 0 || off[d.n_events] != c->n_active)) bad = 1;
    long long carry_n = 0, carry_items = 0, carry_tiles = 0;
    unsigned long long pairs = 0, cs = 0;
    for (int base = 0; base < d.n_events; base += blockDim.x) {
        const int e = base + threadIdx.x;
        int n_old = 0, n_new = 0;
        if (e < d.n_events) {
            const int a = off[e], b = off[e + 1];
            const int k = d.ev_collected_now[e];
            if (a < 0 || b < a || b > d.n_total || k < 0 || k > b - a) bad = 1;
            n_old = b - a;
            n_new = n_old - k;
            d.ev_collected_now[e] = 0;
        }
        pairs += (unsigned long long)n_old * (unsigned long long)n_old;
        cs += (unsigned long long)n_old;
        long long tn, ti, tt = 0;
        const long long exn = block_exclusive_scan(n_new, s_warp, tn);
        const long long exi = block_exclusive_scan(items_for(d, n_new), s_warp, ti);
        long long ext_ = 0;
        if (d.tile_base) ext_ = block_exclusive_scan(tiles_for(d, n_new), s_warp, tt);
        if (e < d.n_events) {
            noff[e] = (int)(carry_n + exn);
            d.item_base[e] = (int)(carry_items + exi);
            if (d.tile_base) d.tile_base[e] = (int)(carry_tiles + ext_);
        }
        carry_n += tn;
        carry_items += ti;
        carry_tiles += tt;
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) atomicOr(&c->error, kErrOffsets);
        return;
    }
    // reduce the counters
    long long tot_pairs, tot_cs;
    (void)block_exclusive_scan((long long)pairs, s_warp, tot_pairs);
    (void)block_exclusive_scan((long long)cs, s_warp, tot_cs);
    // the next integrate accumulates its chunk counts atomically: zero them
    const int nch = ceil_div((int)carry_n, kChunk);
    if (fine_units((int)carry_n))
        for (int k = threadIdx.x; k < nch; k += blockDim.x) d.chunk_cnt[k] = 0;
    if (threadIdx.x == 0) {
        noff[d.n_events] = (int)carry_n;
        d.item_base[d.n_events] = (int)carry_items;
        if (d.tile_base) d.tile_base[d.n_events] = (int)carry_tiles;
        c->n_active = (int)carry_n;
        c->items_total = (int)carry_items;
        c->tiles_total = (int)carry_tiles;
        c->work_counter = 0u;
        c->cur = cur ^ 1;
        if (!INIT) {
            c->step += 1;
            c->carrier_steps += (unsigned long long)tot_cs;
            if (d.phys.coulomb) c->pair_interactions += (unsigned long long)tot_pairs;
        }
    }
}

template <bool INIT>
__global__ void __launch_bounds__(kChunkThreads) finalize_kernel(Dev d) {
    __shared__ long long s_warp[33];
    if (step_skipped(d.ctrl)) return;
    finalize_block<INIT>(d, s_warp);
}

// Fused small-workload path, after the fused pair kernel has integrated every
// i-tile: one block compacts the active list from the keep bytes (stable,
// thread t owning a contiguous run of slots), writes the next step's shadow
// (and FP16x2 extents) exactly as compact_kernel does, then runs the
// bookkeeping of finalize_kernel.
template <bool F64>
__global__ void __launch_bounds__(kChunkThreads) small_tail_kernel(Dev d) {
    __shared__ long long s_warp[33];
    Ctrl *c = d.ctrl;
    if (step_skipped(c)) return;
    const int cur = c->cur;
    const int n_act = c->n_active;
    const int *src = d.act[cur];
    int *dst = d.act[cur ^ 1];
    unsigned *ext = (!F64 && d.ev_ext[0]) ? d.ev_ext[cur ^ 1] : nullptr;
    if (ext) {
        for (int e = threadIdx.x; e < d.n_events; e += blockDim.x) ext[e] = 0u;
        __syncthreads();
    }
    const int per = ceil_div(n_act, (int)blockDim.x);
    const int p0 = min(n_act, (int)threadIdx.x * per), p1 = min(n_act, p0 + per);
    int kept = 0;
    for (int p = p0; p < p1; ++p) kept += d.keep8[p];
    long long total;
    int q = (int)block_exclusive_scan(kept, s_warp, total);
#pragma unroll 4
    for (int p = p0; p < p1; ++p) {
        if (!d.keep8[p]) continue;
        const int id = src[p];
        if (!GC_GUARD(q < d.n_total && id >= 0 && id < d.n_total)) continue;
        dst[q] = id;
        const int e = d.ev_of_id[id];
        const double ox = d.ev_origin[3 * e], oy = d.ev_origin[3 * e + 1], oz = d.ev_origin[3 * e + 2];
        if (F64) {
            d.sh64[q] = make_double4_32a(d.px[id] - ox, d.py[id] - oy, d.pz[id] - oz, 0.0);
        } else {
            const float4 v = make_float4(d2f_exact(d.px[id] - ox), d2f_exact(d.py[id] - oy),
                                         d2f_exact(d.pz[id] - oz), 1.0f);
            d.sh32[q] = v;
            if (ext) atomicMax(&ext[e], __float_as_uint(fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z)))));
        }
        ++q;
    }
    __syncthreads();
    finalize_block<false>(d, s_warp);
}

// Device-side loop condition: continue while holes are active, the step limit
// is not reached, the last pass advanced the step counter and (when a second,
// fused small-workload graph takes over below it) more than switch_below
// holes are active.
__global__ void loop_cond_kernel(Dev d, cudaGraphConditionalHandle h, int switch_below) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Ctrl *c = d.ctrl;
    const bool go = c->n_active > switch_below && c->n_active > c->stop_below && c->n_active > 0 &&
                    c->step < c->step_limit && c->step != c->loop_last;
    c->loop_last = c->step;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Items only (no counters, no buffer flip): used after the pair shape changes.
__global__ void __launch_bounds__(kChunkThreads) build_items_kernel(Dev d) {
    __shared__ long long s_warp[33];
    Ctrl *c = d.ctrl;
    if (c->error) return;  // the offsets failed a check: they size nothing
    const int *off = d.ev_off[c->cur];
    long long carry = 0, carry_t = 0;
    for (int base = 0; base < d.n_events; base += kChunkThreads) {
        const int e = base + threadIdx.x;
        const int n = e < d.n_events ? off[e + 1] - off[e] : 0;
        long long t, tt = 0;
        const long long ex = block_exclusive_scan(items_for(d, n), s_warp, t);
        long long ext_ = 0;
        if (d.tile_base) ext_ = block_exclusive_scan(tiles_for(d, n), s_warp, tt);
        if (e < d.n_events) {
            d.item_base[e] = (int)(carry + ex);
            if (d.tile_base) d.tile_base[e] = (int)(carry_t + ext_);
        }
        carry += t;
        carry_t += tt;
    }
    if (threadIdx.x == 0) {
        d.item_base[d.n_events] = (int)carry;
        if (d.tile_base) d.tile_base[d.n_events] = (int)carry_t;
        c->items_total = (int)carry;
        c->tiles_total = (int)carry_t;
        c->work_counter = 0u;
    }
}

// ---- standalone Eq. 6 helpers -------------------------------------------------------------------
__global__ void field_prepare_kernel(Dev d, const double *__restrict__ xyz, int n, bool f64) {
    const double ox = d.ev_origin[0], oy = d.ev_origin[1], oz = d.ev_origin[2];
    const int stride = gridDim.x * blockDim.x;
    const int n_round = (n + 31) / 32 * 32;  // whole warps stay in the loop (warp reduction)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        unsigned ext_bits = 0u;
        if (i < n) {
            const double x = xyz[3LL * i] - ox, y = xyz[3LL * i + 1] - oy, z = xyz[3LL * i + 2] - oz;
            if (f64) {
                d.sh64[i] = make_double4_32a(x, y, z, 0.0);
            } else {
                const float4 v = make_float4((float)x, (float)y, (float)z, 1.0f);
                d.sh32[i] = v;
                ext_bits = __float_as_uint(fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z))));
            }
        }
        if (d.ev_ext[0]) {  // FP16x2 form: one event, buffer 0
            const unsigned mx = __reduce_max_sync(0xffffffffu, ext_bits);
            if ((threadIdx.x & 31) == 0) atomicMax(&d.ev_ext[0][0], mx);
        }
    }
}

__global__ void field_finish_kernel(Dev d, int n, double *__restrict__ E) {
    const int js = ceil_div(n, d.shape.jchunk);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double ex = 0.0, ey = 0.0, ez = 0.0;
        const double *P = d.partial + i;
        for (int jc = 0; jc < js; ++jc) {
            ex += P[0];
            ey += P[d.part_stride];
            ez += P[2 * d.part_stride];
            P += 3 * d.part_stride;
        }
        E[3LL * i] = d.phys.K * ex;
        E[3LL * i + 1] = d.phys.K * ey;
        E[3LL * i + 2] = d.phys.K * ez;
    }
}

// ---- launchers ---------------------------------------------------------------------------------------
cudaError_t launch_integrate(const Dev &d, bool fp64, bool init, int grid, cudaStream_t st) {
    const bool field = d.phys.coulomb || d.phys.stored;
    if (fp64) {
        if (init) integrate_kernel<true, true, true><<<grid, kChunkThreads, 0, st>>>(d);
        else if (field) integrate_kernel<true, false, true><<<grid, kChunkThreads, 0, st>>>(d);
        else integrate_kernel<true, false, false><<<grid, kChunkThreads, 0, st>>>(d);
    } else {
        if (init) integrate_kernel<false, true, true><<<grid, kChunkThreads, 0, st>>>(d);
        else if (field) integrate_kernel<false, false, true><<<grid, kChunkThreads, 0, st>>>(d);
        else integrate_kernel<false, false, false><<<grid, kChunkThreads, 0, st>>>(d);
    }
    return cudaGetLastError();
}

cudaError_t launch_compact(const Dev &d, bool fp64, int grid, cudaStream_t st) {
    if (fp64) compact_kernel<true><<<grid, kChunkThreads, 0, st>>>(d);
    else compact_kernel<false><<<grid, kChunkThreads, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Dev &d, bool init, cudaStream_t st) {
    if (init) finalize_kernel<true><<<1, kChunkThreads, 0, st>>>(d);
    else finalize_kernel<false><<<1, kChunkThreads, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_loop_cond(const Dev &d, cudaGraphConditionalHandle h, int switch_below,
                             cudaStream_t st) {
    loop_cond_kernel<<<1, 32, 0, st>>>(d, h, switch_below);
    return cudaGetLastError();
}

cudaError_t launch_small_tail(const Dev &d, bool fp64, cudaStream_t st) {
    if (fp64) small_tail_kernel<true><<<1, kChunkThreads, 0, st>>>(d);
    else small_tail_kernel<false><<<1, kChunkThreads, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_shadow(const Dev &d, int sm_count, cudaStream_t st) {
    const int grid = max(1, min(ceil_div(d.n_total, 256), 8 * max(sm_count, 1)));
    shadow_kernel<<<grid, 256, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_occupied_pixels(const Dev &d, cudaStream_t st) {
    occupied_pixels_kernel<<<min(d.n_events, 8192), kChunkThreads, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_build_items(const Dev &d, cudaStream_t st) {
    build_items_kernel<<<1, kChunkThreads, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_field_prepare(const Dev &d, const double *xyz, int n, bool fp64, cudaStream_t st) {
    const int grid = n > 0 ? min(ceil_div(n, 256), 4096) : 1;
    field_prepare_kernel<<<grid, 256, 0, st>>>(d, xyz, n, fp64);
    return cudaGetLastError();
}

cudaError_t launch_field_finish(const Dev &d, int n, double *E, cudaStream_t st) {
    const int grid = n > 0 ? min(ceil_div(n, 256), 4096) : 1;
    field_finish_kernel<<<grid, 256, 0, st>>>(d, n, E);
    return cudaGetLastError();
}

}  // namespace gc
