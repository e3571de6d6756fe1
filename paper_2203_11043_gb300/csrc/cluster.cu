// cluster.cu -- one small event resident in a thread-block cluster: every
// step of the Fig. 2 loop in one launch, with the event's state in shared
// memory and distributed shared memory (DSMEM) between the cluster's CTAs.
//
// For an event below the 4-lane threshold (at most 2048 holes, FP32 forms),
// the whole active list and its FP32 shadow fit in each CTA's shared memory.
// Each of the CS CTAs (512 threads = up to 128 carriers x 4 lanes) owns a
// slice of the slots; per step it
//   1. sums Eq. 6 for its carriers against the whole shadow in its own shared
//      memory: 4 lanes per carrier, packed even/odd j pairs, FP32 sums
//      folded into Kahan-compensated totals every 1024 j's, as in the 4-lane
//      path, but over the whole j range at once and with the lanes combined
//      in FP32 (one FP64 conversion per carrier): GB300's FP64 rate is a
//      small fraction of FP32, and on the cluster's few SMs the per-chunk
//      FP64 partials of the other paths would dominate the step.  The
//      result therefore differs from the other paths by FP32 rounding
//      (within the same error bound), and is deterministic;
//   2. integrates its carriers in registers (advance_hole with the field
//      given), positions loaded through L2 at the start of the step;
//   3. writes each carrier's keep byte and next shadow into every CTA's
//      staging area (DSMEM stores);
//   4. one hardware cluster barrier (no software wait);
//   5. compacts its own copy of the list and shadow from the staging area.
// The staging area is double-buffered by step parity: a CTA can be at most
// one barrier ahead of another.  At the end CTA 0 writes the state back in
// the layout of the other paths.
#include <cooperative_groups.h>

#include "gc_pair.cuh"
#include "gc_launch.h"

namespace cg = cooperative_groups;

namespace gc {

constexpr int kClThreads = 512;          // 128 carriers x 4 lanes per CTA
constexpr int kClMaxN = kSmallEvent;     // the 4-lane regime
constexpr int kClMaxCTAs = 16;

struct ClSmem {
    int ids[kClMaxN];                        // active list (hole ids), slot order
    float sx[kClMaxN + 4], sy[kClMaxN + 4], sz[kClMaxN + 4];  // FP32 shadow, slot order
    float nx[2][kClMaxN], ny[2][kClMaxN], nz[2][kClMaxN];      // staging: next shadow by slot
    unsigned char keep[2][kClMaxN];          // staging: keep byte by slot
    long long warp[33];
};

// Four consecutive shadow coordinates from slot j; those at or beyond j1 are
// the padding sentinel, as the staged tiles of the other paths hold them.
__device__ __forceinline__ float4 cl_load4(const float *s, int j, int j1) {
    if (j + 3 < j1) return *reinterpret_cast<const float4 *>(s + j);
    float4 v;
    v.x = j < j1 ? s[j] : kSentinel;
    v.y = j + 1 < j1 ? s[j + 1] : kSentinel;
    v.z = j + 2 < j1 ? s[j + 2] : kSentinel;
    v.w = j + 3 < j1 ? s[j + 3] : kSentinel;
    return v;
}

template <bool KAHAN>
__global__ void __launch_bounds__(kClThreads, 1) cluster_event_kernel(Dev d) {
    extern __shared__ __align__(16) unsigned char cl_smem_raw[];
    ClSmem &S = *reinterpret_cast<ClSmem *>(cl_smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), CS = (int)cl.num_blocks();
    const int tid = threadIdx.x, g = tid >> 2, ph = tid & 3, lane = tid & 31;
    Ctrl *c = d.ctrl;
    if (step_skipped(c)) return;  // uniform over the cluster: nothing has been written yet
    const long long limit = c->step_limit;
    long long step = c->step;
    const int cur = c->cur;
    int n = c->n_active;
    for (int q = tid; q < n; q += blockDim.x) {
        S.ids[q] = d.act[cur][q];
        const float4 v = d.sh32[q];
        S.sx[q] = v.x;
        S.sy[q] = v.y;
        S.sz[q] = v.z;
    }
    const double ox = d.ev_origin[0], oy = d.ev_origin[1], oz = d.ev_origin[2];
    const f2 ZERO = pack2(0.f, 0.f);
    const float eps2f = (float)d.phys.eps2;
    const f2 EPS2 = pack2(eps2f, eps2f);
    cl.sync();  // every CTA of the cluster is running and has its copy
    unsigned long long pairs = 0, csteps = 0;
    for (int k = 0;; ++k) {
        const int par = k & 1;
        const int per = ceil_div(n, CS);  // <= 128 slots per CTA (n <= 2048, CS = min(16, n / 32))
        const int a = min(n, rank * per), b = min(n, a + per);
        const int p = a + g;
        const bool mine = p < b;
        int id = 0;
        double x = 0.0, y = 0.0, z = 0.0;
        if (mine && ph == 0) {  // written by whichever CTA owned the hole last step
            id = S.ids[p];
            x = __ldcg(d.px + id);
            y = __ldcg(d.py + id);
            z = __ldcg(d.pz + id);
        }
        double gsum[3] = {0.0, 0.0, 0.0};  // the field sum of this carrier (lane 0)
        if (__any_sync(0xffffffffu, mine)) {
            const float xi = mine ? S.sx[p] : kSentinel, yi = mine ? S.sy[p] : kSentinel,
                        zi = mine ? S.sz[p] : kSentinel;
            const f2 xi2 = pack2(xi, xi), yi2 = pack2(yi, yi), zi2 = pack2(zi, zi);
            {
                const int j0 = 0, j1 = n;
                f2 ax = ZERO, ay = ZERO, az = ZERO;
                f2 kreg[6] = {ZERO, ZERO, ZERO, ZERO, ZERO, ZERO};
                for (int jt = j0; jt < j1; jt += 4 * kTileJ) {
                    const int cnt = min(4 * kTileJ, j1 - jt);
                    const int kmax = (cnt + 63) / 64 * 64;  // 4 loads x 4 j's x 4 lanes per iteration
                    for (int k0 = 4 * ph; k0 < kmax; k0 += 64) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int j = jt + k0 + u * 16;
                            const float4 X = cl_load4(S.sx, j, j1), Y = cl_load4(S.sy, j, j1),
                                         Z = cl_load4(S.sz, j, j1);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const f2 xj = h ? pack2(X.z, X.w) : pack2(X.x, X.y);
                                const f2 yj = h ? pack2(Y.z, Y.w) : pack2(Y.x, Y.y);
                                const f2 zj = h ? pack2(Z.z, Z.w) : pack2(Z.x, Z.y);
                                const f2 dx = sub2(xi2, xj), dy = sub2(yi2, yj), dz = sub2(zi2, zj);
                                f2 r2 = fma2(dx, dx, EPS2);
                                r2 = fma2(dy, dy, r2);
                                r2 = fma2(dz, dz, r2);
                                float ra, rb;
                                unpack2(r2, ra, rb);
                                const f2 inv = pack2(rsqrt_mufu(ra), rsqrt_mufu(rb));
                                const f2 inv3 = mul2(mul2(inv, inv), inv);
                                ax = fma2(dx, inv3, ax);
                                ay = fma2(dy, inv3, ay);
                                az = fma2(dz, inv3, az);
                            }
                        }
                    }
                    if (KAHAN) {  // fold this tile's sums into the compensated totals
                        const f2 acc[3] = {ax, ay, az};
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) {
                            const f2 s0 = kreg[2 * cc], c0 = kreg[2 * cc + 1];
                            const f2 yk = sub2(acc[cc], c0), t = add2(s0, yk);
                            kreg[2 * cc + 1] = sub2(sub2(t, s0), yk);
                            kreg[2 * cc] = t;
                        }
                        ax = ay = az = ZERO;
                    }
                }
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {  // lanes combined in FP32, one conversion
                    float lo, hi, v;
                    if (KAHAN) {
                        float clo, chi;
                        unpack2(kreg[2 * cc], lo, hi);
                        unpack2(kreg[2 * cc + 1], clo, chi);
                        v = (lo - clo) + (hi - chi);
                    } else {
                        unpack2(cc == 0 ? ax : (cc == 1 ? ay : az), lo, hi);
                        v = lo + hi;
                    }
#pragma unroll
                    for (int o = 1; o < 4; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    gsum[cc] = (double)v;
                }
            }
        }
        // integrate this CTA's carriers (lane 0 of each group)
        int kept = 0;
        float nsx = 0.f, nsy = 0.f, nsz = 0.f;
        if (mine && ph == 0) {
            kept = advance_hole<false, false, true, true>(d, id, 0, n, p, step + 1, x, y, z, gsum[0], gsum[1],
                                                         gsum[2])
                       ? 1 : 0;
            nsx = (float)(x - ox);
            nsy = (float)(y - oy);
            nsz = (float)(z - oz);
        }
        // every CTA's staging area gets the keep byte and next shadow of this CTA's slots
        const int src = lane & ~3;
        kept = __shfl_sync(0xffffffffu, kept, src);
        nsx = __shfl_sync(0xffffffffu, nsx, src);
        nsy = __shfl_sync(0xffffffffu, nsy, src);
        nsz = __shfl_sync(0xffffffffu, nsz, src);
        if (mine) {
            for (int r = ph; r < CS; r += 4) {
                ClSmem *R = cl.map_shared_rank(&S, r);
                R->keep[par][p] = (unsigned char)kept;
                if (kept) {
                    R->nx[par][p] = nsx;
                    R->ny[par][p] = nsy;
                    R->nz[par][p] = nsz;
                }
            }
        }
        cl.sync();  // every slot's staging entry is in every CTA
        pairs += (unsigned long long)n * (unsigned long long)n;
        csteps += (unsigned long long)n;
        // compact this CTA's copy: slots in rounds of 4 per thread (one round up to 2048)
        int base = 0;
        for (int c0 = 0; c0 < n; c0 += 4 * (int)blockDim.x) {
            const int p0 = c0 + 4 * tid;
            int cntk = 0, v[4];
            unsigned char kb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int pp = p0 + u;
                kb[u] = pp < n ? S.keep[par][pp] : (unsigned char)0;
                v[u] = pp < n ? S.ids[pp] : 0;
                cntk += kb[u];
            }
            long long tot;
            int q = base + (int)block_exclusive_scan(cntk, S.warp, tot);  // reads precede writes
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (kb[u]) {
                    S.ids[q] = v[u];
                    S.sx[q] = S.nx[par][p0 + u];
                    S.sy[q] = S.ny[par][p0 + u];
                    S.sz[q] = S.nz[par][p0 + u];
                    ++q;
                }
            base += (int)tot;
        }
        __syncthreads();
        n = base;
        ++step;
        if (n == 0 || step >= limit) break;
    }
    if (rank == 0) {  // the state in the layout of the other paths
        int *dst = d.act[cur ^ 1];
        for (int q = tid; q < n; q += blockDim.x) {
            dst[q] = S.ids[q];
            d.sh32[q] = make_float4(S.sx[q], S.sy[q], S.sz[q], 1.0f);
        }
        if (tid == 0) {
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
    cl.sync();  // no CTA leaves while another could still address its shared memory
}

// ---- launch ------------------------------------------------------------------------------
static const void *cluster_kernel_ptr(int precision) {
    if (precision == 1) return (const void *)cluster_event_kernel<false>;
    if (precision == 2) return (const void *)cluster_event_kernel<true>;
    return nullptr;
}

// One CTA per 32 holes (up to 16): the per-carrier FP64 position update is
// spread over several SMs even for small events.
int cluster_ctas_for(int n) { return max(1, min(kClMaxCTAs, ceil_div(n, 32))); }

// Whether a cluster of cluster_ctas_for(n) CTAs of this kernel can be resident.
bool cluster_path_available(int precision, int n) {
    const void *k = cluster_kernel_ptr(precision);
    if (!k || n < 1 || n > kClMaxN) return false;
    const int cs = cluster_ctas_for(n);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ClSmem)) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = sizeof(ClSmem);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return clusters >= 1;
}

cudaError_t launch_cluster_event(const Dev &d, int precision, int n, cudaStream_t st) {
    const void *k = cluster_kernel_ptr(precision);
    if (!k || n < 1 || n > kClMaxN) return cudaErrorInvalidValue;
    const int cs = cluster_ctas_for(n);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = sizeof(ClSmem);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    Dev dd = d;
    void *args[] = {(void *)&dd};
    return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace gc
