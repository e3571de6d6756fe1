// resident.cu -- one small FP32 event resident on every SM: all steps of the
// Fig. 2 loop in one cooperative launch (one CTA per SM), with no grid
// barrier between steps.
//
// Events of one to a few thousand holes fit neither of the other
// single-launch paths well: a thread-block cluster's 16 SMs are bound by the
// pair arithmetic, and the persistent kernel's grid barrier plus its
// partial-sum hand-off are a chain of fences and L2 round trips per step.
// Here:
//   * every CTA keeps the whole active list and its FP32 shadow in shared
//     memory, in list order (as the cluster kernel does);
//   * each CTA owns the holes at slots b, b + G, b + 2G, ... of the list at
//     the launch (G CTAs, at most 32 holes each) for the whole launch: their
//     FP64 positions stay in registers of its first warp, so no position
//     crosses SMs;
//   * per step a CTA sums Eq. 6 for its owned holes (one warp per hole, the
//     32 lanes over j in packed even/odd pairs, FP32 sums folded into
//     Kahan-compensated totals every 1024 j's, lanes combined in FP32 as in
//     the cluster kernel), integrates them in one warp and publishes each
//     hole's keep bit and next FP32 shadow as three 8-byte words.  (Measured
//     against two holes per warp sharing each load, and against the list
//     split into segments for more, shorter work units: both slower at 1573
//     holes, the second at every size, by the fixed cost of each unit's
//     lane reduction);
//   * the integration is a dependent chain, and on GB300 every FP64 step of
//     it (a double operation or conversion) costs ~150-190 cycles, so it
//     forms the field in FP32 (the sum, K and the Eq. 1 field from the FP32
//     shadow; the other FP32 paths round the field to FP32 too) and keeps
//     FP64 for the position update and the z check (advance_hole32); the
//     step's normals, which do not depend on the field, come from the last
//     warp while the others sum Eq. 6;
//   * each word carries the step's tag beside its value and is written and
//     read whole (8-byte relaxed accesses at GPU scope are single-copy
//     atomic), so a reader that sees the tag has the value.  Every CTA reads
//     the words of all holes of the step, re-reading (bounded in time) those
//     without the tag yet, and compacts its own copy of the list.  The data
//     exchange is the synchronisation: no fence, no arrival counter.
// The words are double-buffered by step parity: a CTA cannot finish step
// k + 1 before every live owner has published its step-(k + 1) words, which
// each does only after reading all step-k words, so no CTA gets more than
// one step ahead of a reader.  A CTA whose holes are all collected leaves
// (nobody reads words it would write), except CTA 0, which writes the state
// back at the end: it also publishes a progress word per step, which every
// CTA waits for, so that it too is never overtaken by two steps.  The
// launcher clears the words first (tag 0 is no step).  The result does not
// depend on G: each hole's sum runs over the whole list in list order with
// the same lane split.  At the end CTA 0 writes the state back in the layout
// of the other paths.
#include "gc_barrier.cuh"
#include "gc_slot.cuh"
#include "gc_launch.h"

namespace gc {

constexpr int kRsThreads = 512;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsMaxN = 4096;                    // active holes at the launch
constexpr int kRsOwn = 32;                       // holes owned per CTA: one lane each of warp 0
constexpr int kRsRounds = kRsMaxN / kRsThreads;  // list slots per thread in the exchange
constexpr int kRsFoldGroups = 8;                 // Kahan fold every 8 groups of 128 j's
constexpr size_t kRsProgress = 2 * 3 * (size_t)kRsMaxN;  // words [parity][coordinate][launch slot], then
constexpr size_t kRsWords = kRsProgress + 2;              // CTA 0's progress word [parity]

struct RsSmem {
    int ini[kRsMaxN];                       // list: each entry's launch slot (its word index)
    float sx[kRsMaxN], sy[kRsMaxN], sz[kRsMaxN];  // FP32 shadow, list order, sentinel to a multiple of 128
    float4 own_s[kRsOwn];                   // shadow of each owned hole (the i side)
    float gsum[kRsOwn][3];                  // Eq. 6 sum of each owned hole
    float own_n[kRsOwn][3];                 // the step's normals of each owned hole (Eq. 3)
    int own_id[kRsOwn];                     // hole id of each owned hole
    int act_own[kRsOwn];                    // owned holes still active, in owned order
    int cnt[kRsRounds * kRsWarps];          // kept count per (round, warp)
    int n_own;
};

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
// A published word: the value's bits low, (tag << 1 | keep) high.
__device__ __forceinline__ unsigned long long rs_word(float v, unsigned tagkeep) {
    return ((unsigned long long)tagkeep << 32) | (unsigned long long)__float_as_uint(v);
}
__device__ __forceinline__ bool rs_tagged(unsigned long long w, unsigned tag) {
    return (unsigned)(w >> 33) == tag;
}

// Eq. 6 sum of one hole (FP32 shadow position A) over the list's `groups`
// groups of 128 slots: lane l takes slots 4l .. 4l + 3 of each group as
// packed even/odd pairs; FP32 sums are folded into Kahan-compensated totals
// every kRsFoldGroups groups.  Returns on every lane the sum over the 32
// lanes (even/odd halves first).
template <bool KAHAN>
__device__ __forceinline__ void rs_pair_sum(const RsSmem &S, float4 A, int groups, f2 EPS2, int lane,
                                            float out[3]) {
    const f2 ZERO = pack2(0.f, 0.f);
    const f2 xi = pack2(A.x, A.x), yi = pack2(A.y, A.y), zi = pack2(A.z, A.z);
    f2 acc[3] = {ZERO, ZERO, ZERO}, kreg[6] = {ZERO, ZERO, ZERO, ZERO, ZERO, ZERO};
    for (int t0 = 0; t0 < groups; t0 += kRsFoldGroups) {
        const int t1 = min(groups, t0 + kRsFoldGroups);
#pragma unroll 1
        for (int g = t0; g < t1; ++g) {
            const int j = g * 128 + 4 * lane;
            const float4 X = *reinterpret_cast<const float4 *>(S.sx + j);
            const float4 Y = *reinterpret_cast<const float4 *>(S.sy + j);
            const float4 Z = *reinterpret_cast<const float4 *>(S.sz + j);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const f2 xj = h ? pack2(X.z, X.w) : pack2(X.x, X.y);
                const f2 yj = h ? pack2(Y.z, Y.w) : pack2(Y.x, Y.y);
                const f2 zj = h ? pack2(Z.z, Z.w) : pack2(Z.x, Z.y);
                const f2 dx = sub2(xi, xj), dy = sub2(yi, yj), dz = sub2(zi, zj);
                f2 r2 = fma2(dx, dx, EPS2);
                r2 = fma2(dy, dy, r2);
                r2 = fma2(dz, dz, r2);
                float ra, rb;
                unpack2(r2, ra, rb);
                const f2 inv = pack2(rsqrt_mufu(ra), rsqrt_mufu(rb));
                const f2 inv3 = mul2(mul2(inv, inv), inv);
                acc[0] = fma2(dx, inv3, acc[0]);
                acc[1] = fma2(dy, inv3, acc[1]);
                acc[2] = fma2(dz, inv3, acc[2]);
            }
        }
        if (KAHAN) {  // fold this tile's sums into the compensated totals
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const f2 s0 = kreg[2 * cc], c0 = kreg[2 * cc + 1];
                const f2 yk = sub2(acc[cc], c0), t = add2(s0, yk);
                kreg[2 * cc + 1] = sub2(sub2(t, s0), yk);
                kreg[2 * cc] = t;
                acc[cc] = ZERO;
            }
        }
    }
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        float lo, hi, v;
        if (KAHAN) {
            float clo, chi;
            unpack2(kreg[2 * cc], lo, hi);
            unpack2(kreg[2 * cc + 1], clo, chi);
            v = (lo - clo) + (hi - chi);
        } else {
            unpack2(acc[cc], lo, hi);
            v = lo + hi;
        }
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
        out[cc] = v;
    }
}

template <bool KAHAN>
__global__ void __launch_bounds__(kRsThreads, 1) resident_event_kernel(Dev d, unsigned long long limit_ns) {
    extern __shared__ __align__(16) unsigned char rs_smem_raw[];
    RsSmem &S = *reinterpret_cast<RsSmem *>(rs_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x, b = blockIdx.x;
    Ctrl *c = d.ctrl;
    if (run_over(c)) return;  // uniform: nothing has been written yet (stop_below is for the other paths)
    const long long limit = c->step_limit;
    long long step = c->step;
    const int cur = c->cur;
    const int *act0 = d.act[cur];
    int n = c->n_active;  // at most kRsMaxN and kRsOwn * G (checked by the launcher)
    unsigned long long *const rec = d.rs_rec;
    const double ox = d.ev_origin[0], oy = d.ev_origin[1], oz = d.ev_origin[2];
    const Phys &ph = d.phys;
    const float c0 = (float)(ph.a1 * oz - ph.a2);  // Eq. 1 at the event origin: a1 z - a2 = c0 + a1 (z - oz)
    const unsigned long long seed = d.ev_seed[0];
    const int first = d.ev_first[0];
    {
        const int npad = (n + 127) & ~127;
        for (int q = tid; q < npad; q += kRsThreads) {
            if (q < n) {
                const float4 v = d.sh32[q];
                S.ini[q] = q;
                S.sx[q] = v.x;
                S.sy[q] = v.y;
                S.sz[q] = v.z;
            } else {
                S.sx[q] = S.sy[q] = S.sz[q] = kSentinel;
            }
        }
    }
    // owned holes: lane o of warp 0 holds the hole at launch slot b + o G
    int id = 0;
    bool alive = false;
    double x = 0.0, y = 0.0, z = 0.0;
    if (warp == 0) {
        const int q = b + lane * G;
        alive = q < n;
        if (alive) {
            id = act0[q];
            x = d.px[id];
            y = d.py[id];
            z = d.pz[id];
            S.own_s[lane] = d.sh32[q];
            S.own_id[lane] = id;
        }
        const unsigned m = __ballot_sync(0xffffffffu, alive);
        if (alive) S.act_own[__popc(m & lanemask_lt())] = lane;
        if (lane == 0) S.n_own = __popc(m);
    }
    __syncthreads();
    const float eps2f = (float)d.phys.eps2;
    const f2 EPS2 = pack2(eps2f, eps2f);
    unsigned long long pairs = 0, csteps = 0;
    for (int k = 0;; ++k) {
        const int par = k & 1;
        const unsigned tag = (unsigned)k + 1u;
        unsigned long long *const wbuf = rec + (size_t)par * 3 * kRsMaxN;
        // ---- Eq. 6 for the owned active holes: one warp per hole, lanes over j
        const int K = S.n_own;
        const int groups = (n + 127) >> 7;
        if (warp == kRsWarps - 1 && ph.diffusion && lane < K) {  // the normals of this step (Philox, Box-Muller)
            const int o = S.act_own[lane];
            float nv[3];
            normals32(diffusion_bits(seed, S.own_id[o] - first, step + 1), nv);
            S.own_n[o][0] = nv[0];
            S.own_n[o][1] = nv[1];
            S.own_n[o][2] = nv[2];
        }
        for (int m = warp; m < K; m += kRsWarps) {  // one warp per owned active hole
            const int o = S.act_own[m];
            float out[3];
            rs_pair_sum<KAHAN>(S, S.own_s[o], groups, EPS2, lane, out);
            if (lane == 0) {
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) S.gsum[o][cc] = out[cc];
            }
        }
        __syncthreads();
        // ---- integrate the owned holes (warp 0) and publish their words
        if (warp == 0) {
            if (alive) {
                const float nv[3] = {S.own_n[lane][0], S.own_n[lane][1], S.own_n[lane][2]};
                const bool kept = advance_hole32(d, id, 0, step + 1, x, y, z, S.gsum[lane][0], S.gsum[lane][1],
                                                 S.gsum[lane][2],
                                                 fmaf(ph.f_a1, S.own_s[lane].z, c0), nv);
                const float nx = (float)(x - ox), ny = (float)(y - oy), nz = (float)(z - oz);
                const unsigned tk = (tag << 1) | (kept ? 1u : 0u);
                unsigned long long *w = wbuf + (b + lane * G);
#ifdef GC_DEBUG
                const bool withhold = d.dbg_withhold && b == 1 && k == 0;  // planted: the others' waits run out
#else
                constexpr bool withhold = false;
#endif
                if (!withhold) {
                    st_relaxed_u64(w, rs_word(nx, tk));
                    st_relaxed_u64(w + kRsMaxN, rs_word(ny, tk));
                    st_relaxed_u64(w + 2 * kRsMaxN, rs_word(nz, tk));
                }
                if (kept) S.own_s[lane] = make_float4(nx, ny, nz, 0.0f);
                alive = kept;
            }
            const unsigned m = __ballot_sync(0xffffffffu, alive);
            if (alive) S.act_own[__popc(m & lanemask_lt())] = lane;
            if (lane == 0) {
                S.n_own = __popc(m);
                if (b == 0) st_relaxed_u64(rec + kRsProgress + par, (unsigned long long)tag << 33);
            }
        }
        __syncthreads();  // the other warps wait here rather than spin on words not yet written
        // ---- read every hole's words of this step: all loads first, then the checks
        const int rounds = (n + kRsThreads - 1) / kRsThreads;
        unsigned long long w[kRsRounds][3];
        int rr[kRsRounds];
#pragma unroll
        for (int u = 0; u < kRsRounds; ++u) {
            const int p = u * kRsThreads + tid;
            rr[u] = -1;
            w[u][0] = w[u][1] = w[u][2] = 0ull;
            if (u < rounds && p < n) {
                rr[u] = S.ini[p];
                const unsigned long long *src = wbuf + rr[u];
                w[u][0] = ld_relaxed_u64(src);
                w[u][1] = ld_relaxed_u64(src + kRsMaxN);
                w[u][2] = ld_relaxed_u64(src + 2 * kRsMaxN);
            }
        }
        bool failed = false;
        if (tid == 0) {  // CTA 0 has read every step-(k - 1) word (it may own no hole)
            const unsigned long long *src = rec + kRsProgress + par;
            unsigned long long t0 = 0ull;
            for (int spins = 1; !rs_tagged(ld_relaxed_u64(src), tag); ++spins) {
                if ((spins & 31) == 0) {  // bounded wait
                    const unsigned long long now = globaltimer_ns();
                    if (t0 == 0ull) {
                        t0 = now;
                    } else if (now - t0 > limit_ns) {
                        atomicOr(&c->error, kErrBarrierTimeout);
                        failed = true;
                        break;
                    }
                }
            }
        }
        unsigned bal[kRsRounds];
#pragma unroll
        for (int u = 0; u < kRsRounds; ++u) {
            bal[u] = 0u;
            if (u < rounds) {  // uniform over the block
                bool kept = false;
                if (rr[u] >= 0) {
                    const unsigned long long *src = wbuf + rr[u];
                    unsigned long long t0 = 0ull;
                    int spins = 0;
                    while (!failed && !(rs_tagged(w[u][0], tag) && rs_tagged(w[u][1], tag) &&
                                        rs_tagged(w[u][2], tag))) {
                        if ((++spins & 31) == 0) {  // bounded wait
                            const unsigned long long now = globaltimer_ns();
                            if (t0 == 0ull) {
                                t0 = now;
                            } else if (now - t0 > limit_ns) {
                                atomicOr(&c->error, kErrBarrierTimeout);
                                failed = true;
                            }
                        }
                        w[u][0] = ld_relaxed_u64(src);
                        w[u][1] = ld_relaxed_u64(src + kRsMaxN);
                        w[u][2] = ld_relaxed_u64(src + 2 * kRsMaxN);
                    }
                    kept = ((w[u][2] >> 32) & 1ull) != 0ull;
                }
                bal[u] = __ballot_sync(0xffffffffu, kept);
                if (lane == 0) S.cnt[u * kRsWarps + warp] = __popc(bal[u]);
            }
        }
        if (__syncthreads_or(failed)) return;  // the other CTAs' waits run out in turn
        // ---- each warp: exclusive prefix of the kept counts in list order (round, then
        // warp; at most 128, four per lane), then its entries of the compacted list
        int pre[4], n_new;
        {
            const int nv = rounds * kRsWarps;
            int v[4], s = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int idx = lane * 4 + i;
                v[i] = idx < nv ? S.cnt[idx] : 0;
                s += v[i];
            }
            int incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            pre[0] = incl - s;
#pragma unroll
            for (int i = 1; i < 4; ++i) pre[i] = pre[i - 1] + v[i - 1];
            n_new = __shfl_sync(0xffffffffu, incl, 31);
        }
#pragma unroll
        for (int u = 0; u < kRsRounds; ++u) {
            if (u < rounds) {  // uniform over the block
                const int idx = u * kRsWarps + warp;  // uniform over the warp
                const int w4 = idx & 3;
                const int mine = w4 == 0 ? pre[0] : (w4 == 1 ? pre[1] : (w4 == 2 ? pre[2] : pre[3]));
                const int base = __shfl_sync(0xffffffffu, mine, idx >> 2);
                if ((bal[u] >> lane) & 1u) {
                    const int q = base + __popc(bal[u] & lanemask_lt());
                    S.ini[q] = rr[u];
                    S.sx[q] = __uint_as_float((unsigned)w[u][0]);
                    S.sy[q] = __uint_as_float((unsigned)w[u][1]);
                    S.sz[q] = __uint_as_float((unsigned)w[u][2]);
                }
            }
        }
        for (int q = n_new + tid; q < ((n_new + 127) & ~127); q += kRsThreads)
            S.sx[q] = S.sy[q] = S.sz[q] = kSentinel;
        __syncthreads();
        pairs += (unsigned long long)n * (unsigned long long)n;
        csteps += (unsigned long long)n;
        n = n_new;
        ++step;
        // (a launch runs at most 2^30 steps: the tag has 31 bits)
        if (n == 0 || step >= limit || k + 1 >= (1 << 30)) break;
        if (b != 0 && S.n_own == 0) return;  // nothing left to publish; CTA 0 stays for the write-back
    }
    if (b != 0) return;
    // CTA 0: the state in the layout of the other paths (its copy of the list
    // is every CTA's); the launcher clears the per-step collection counter
    int *dst = d.act[cur ^ 1];
    for (int q = tid; q < n; q += kRsThreads) {
        dst[q] = act0[S.ini[q]];
        d.sh32[q] = make_float4(S.sx[q], S.sy[q], S.sz[q], 1.0f);
    }
    if (tid == 0) {
        d.ev_off[cur ^ 1][0] = 0;
        d.ev_off[cur ^ 1][1] = n;
        c->step = step;
        c->n_active = n;
        c->cur = cur ^ 1;
        c->carrier_steps += csteps;
        c->pair_interactions += pairs;
        c->work_counter = 0u;
    }
}

// ---- launch ------------------------------------------------------------------------------
static const void *resident_kernel_ptr(int precision) {
    if (precision == 1) return (const void *)resident_event_kernel<false>;
    if (precision == 2) return (const void *)resident_event_kernel<true>;
    return nullptr;
}

size_t resident_words_bytes() { return kRsWords * sizeof(unsigned long long); }

// CTAs of a launch for n active holes: `want` if given, else one per 8 holes
// (measured: 256 holes 3.2 us per step on 32 CTAs against 3.35 us on 152,
// 1000 holes 4.2 against 4.85 us on 125 and 152), within [ceil(n / kRsOwn),
// SMs].  The results do not depend on it.
int resident_grid(int sm_count, int n, int want) {
    const int g = want > 0 ? want : ceil_div(n, 8);
    return std::max(1, std::min(sm_count, std::max(g, ceil_div(n, kRsOwn))));
}

bool resident_path_available(int precision, int n, int sm_count) {
    const void *k = resident_kernel_ptr(precision);
    if (!k || n < 1 || n > kRsMaxN) return false;
    const int G = resident_grid(sm_count, n, 0);
    if ((long long)kRsOwn * G < n) return false;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(RsSmem)) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, kRsThreads, sizeof(RsSmem)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return blocks >= 1 && G <= blocks * sm_count;
}

cudaError_t launch_resident_event(const Dev &d, int precision, int n, int sm_count, int ctas, double limit_s,
                                  cudaStream_t st) {
    const void *k = resident_kernel_ptr(precision);
    if (!k || !d.rs_rec || n < 1 || n > kRsMaxN) return cudaErrorInvalidValue;
    const int G = resident_grid(sm_count, n, ctas);
    if ((long long)kRsOwn * G < n) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(d.rs_rec, 0, resident_words_bytes(), st);  // tag 0: no step
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(RsSmem));
    if (e != cudaSuccess) return e;
    Dev dd = d;
    unsigned long long limit_ns = (unsigned long long)(limit_s * 1e9);
    void *args[] = {(void *)&dd, (void *)&limit_ns};
    e = cudaLaunchCooperativeKernel(k, dim3(G), dim3(kRsThreads), args, sizeof(RsSmem), st);
    if (e != cudaSuccess) return e;
    // the collections of the launch's steps are counted in the image and
    // collect_step; the per-step counter starts from zero for the next step
    return cudaMemsetAsync(d.ev_collected_now, 0, sizeof(int), st);
}

}  // namespace gc
