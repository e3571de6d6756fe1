// gc_slot.cuh -- the per-carrier part of one time step (Fig. 2), shared by
// the integrate kernel and the fused small-workload pair kernel so that both
// run the same arithmetic: Eq. 1 + Eq. 6 field, Eq. 2 mobility, drift,
// Eqs. 3-4 diffusion from Philox-4x32-10 normals, the FP64 position update,
// back-surface reflection, the z check and the pixel binning (Fig. 5).
#pragma once
#include "gc_internal.cuh"

namespace gc {

// ---- Eq. 2 mobility -------------------------------------------------------------
__device__ __forceinline__ double mobility64(const Phys &ph, double E) {
    return ph.mu0 / pow(1.0 + pow(E * ph.inv_Ec, ph.beta), ph.inv_beta);
}
__device__ __forceinline__ float mobility32(const Phys &ph, float E) {
    const float t = exp2f(ph.f_beta * log2f(E * ph.f_inv_Ec));
    return ph.f_mu0 * exp2f(-ph.f_inv_beta * log2f(1.0f + t));
}

// ---- Box-Muller on the Philox bits (u_a in (0,1], u_b in [0,1)) ---------------------
__device__ __forceinline__ void normals64(uint4 b, double n[3]) {
    const double s = 2.3283064365386963e-10;  // 2^-32
    const double r0 = sqrt(-2.0 * log(((double)b.x + 1.0) * s));
    double sn, cs;
    sincospi(2.0 * ((double)b.y * s), &sn, &cs);
    n[0] = r0 * cs;
    n[1] = r0 * sn;
    const double r1 = sqrt(-2.0 * log(((double)b.z + 1.0) * s));
    n[2] = r1 * cospi(2.0 * ((double)b.w * s));
}
__device__ __forceinline__ void normals32(uint4 b, float n[3]) {
    const float s = 2.3283064365386963e-10f;  // 2^-32
    const float r0 = sqrtf(-2.0f * logf(fmaf((float)b.x, s, s)));
    float sn, cs;
    sincospif(2.0f * ((float)b.y * s), &sn, &cs);
    n[0] = r0 * cs;
    n[1] = r0 * sn;
    const float r1 = sqrtf(-2.0f * logf(fmaf((float)b.z, s, s)));
    n[2] = r1 * cospif(2.0f * ((float)b.w * s));
}

// ---- FP32 forms: drift (Eq. 2, v = mu E) and diffusion (Eqs. 3-4) of one step --------
// (fx, fy, fz): the field in V/cm; n: the step's three standard normals (read only
// with diffusion on).  The displacement in um.
__device__ __forceinline__ void displacement32(const Phys &ph, float fx, float fy, float fz, const float n[3],
                                               float &ddx, float &ddy, float &ddz) {
    const float E = sqrtf(fx * fx + fy * fy + fz * fz);
    const float mu = mobility32(ph, E);
    const float vdt = 1e4f * mu * ph.f_dt;  // um per (V/cm)
    ddx = vdt * fx;
    ddy = vdt * fy;
    ddz = vdt * fz;
    if (ph.diffusion) {
        const float sigma = sqrtf(2.0f * (1e8f * mu * ph.f_Vth) * ph.f_dt);
        ddx = fmaf(sigma, n[0], ddx);
        ddy = fmaf(sigma, n[1], ddy);
        ddz = fmaf(sigma, n[2], ddz);
    }
}

// ---- block-wide exclusive scan (any block of up to 1024 threads, a multiple of 32) ------------
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *s_warp,
                                                          long long &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
        long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        s_warp[lane] = wi - w;  // exclusive prefix of warp totals
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    const long long ex = s_warp[warp] + incl - v;
    total = s_warp[32];
    __syncthreads();
    return ex;
}

// ---- stored charge (Sec. 1) ----------------------------------------------------------
// Field of the charge stored in event e's pixels at the carrier whose shadow
// position (relative to the event origin o) is r: pixel (ix, iy) with count q
// is q charges at (img_origin + (i + 1/2) p, stored_z), softened as in Eq. 6,
// summed in pixel-index order.  Unscaled (multiply by K).
template <typename T>
__device__ __forceinline__ void stored_field(const Dev &d, int e, T rx0, T ry0, T rz0, T &sx, T &sy,
                                             T &sz) {
    const Phys &ph = d.phys;
    // pixel (0, 0) centre relative to the event origin
    const T cx0 = (T)(d.img_origin[2 * e] + 0.5 * ph.pixel - d.ev_origin[3 * e]);
    const T cy0 = (T)(d.img_origin[2 * e + 1] + 0.5 * ph.pixel - d.ev_origin[3 * e + 1]);
    const T dz = rz0 - (T)(ph.stored_z - d.ev_origin[3 * e + 2]);
    const T pix = (T)ph.pixel, eps2 = (T)ph.eps2;
    const int *occ = d.occ_pix + d.occ_off[e];
    const int cnt = d.occ_cnt[e];
    sx = sy = sz = (T)0;
    if constexpr (sizeof(T) == 4) {  // FP32 forms: precomputed centres, MUFU rsqrt
        const float4 *c4 = d.occ_f4 + d.occ_off[e];
        for (int k = 0; k < cnt; ++k) {
            const float4 cq = c4[k];
            const float dx = rx0 - cq.x, dy = ry0 - cq.y;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
            const float iv = rsqrt_mufu(r2);
            const float w = cq.z * iv * iv * iv;
            sx = fmaf(dx, w, sx);
            sy = fmaf(dy, w, sy);
            sz = fmaf(dz, w, sz);
        }
        (void)occ;
        (void)cx0;
        (void)cy0;
        (void)pix;
    } else {
        // the counts of the step-start snapshot: holes collected during this
        // step's integrate add to the image concurrently and must not be seen
        const unsigned *qs = d.occ_q + d.occ_off[e];
        for (int k = 0; k < cnt; ++k) {
            const int pidx = occ[k];
            const int iy = pidx / ph.img_w, ix = pidx - iy * ph.img_w;
            const T q = (T)qs[k];
            const T dx = rx0 - (cx0 + (T)ix * pix), dy = ry0 - (cy0 + (T)iy * pix);
            const T r2 = dx * dx + dy * dy + dz * dz + eps2;
            const T w = q / (r2 * sqrt(r2));
            sx += dx * w;
            sy += dy * w;
            sz += dz * w;
        }
    }
}

// ---- conversions: by integer operations (INT) or by the hardware -------------------
template <bool INT>
__device__ __forceinline__ float cvt_d2f(double v) {
    if constexpr (INT) return d2f_exact(v);
    else return (float)v;
}
template <bool INT>
__device__ __forceinline__ double cvt_f2d(float v) {
    if constexpr (INT) return f2d_exact(v);
    else return (double)v;
}

// ---- reflection at the back surface: 2 t - z (2 t is exact) -------------------------
// Volatile, so that the compiler keeps this rare FP64 operation in its branch
// instead of executing it for every thread.
__device__ __forceinline__ double reflect_back(const Phys &ph, double z) {
    double r;
    asm volatile("sub.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(2.0 * ph.thickness), "d"(z));
    return r;
}

// ---- the z check (Fig. 2) and the binning of a collected hole (Fig. 5) ----------------
// Returns true when the hole at (x, y, z) stays active; otherwise records its
// collection step and counts it in its event's image (or off the image).
// INTCMP: the test z <= z_well by integer operations (the same result, no
// FP64 unit; the FP32 forms' updates are bound by that unit).
template <bool INTCMP>
__device__ __forceinline__ bool collect_check(const Dev &d, int id, int e, long long step, double x, double y,
                                              double z) {
    const Phys &ph = d.phys;
    if (INTCMP ? le_exact(z, ph.z_well) : z <= ph.z_well) {  // collected at this step
        d.collect_step[id] = (int)step;
        const int eu = d.ev_user[e];
        const double fx = floor((x - d.img_origin[2 * e]) / ph.pixel);
        const double fy = floor((y - d.img_origin[2 * e + 1]) / ph.pixel);
        if (fx >= 0.0 && fx < (double)ph.img_w && fy >= 0.0 && fy < (double)ph.img_h) {
            const long long pix = ((long long)eu * ph.img_h + (long long)fy) * ph.img_w + (long long)fx;
            if (GC_GUARD(eu >= 0 && eu < d.n_events && pix >= 0 &&
                         pix < (long long)d.n_events * ph.img_h * ph.img_w))
                atomicAdd(&d.image[pix], 1u);
        } else if (GC_GUARD(eu >= 0 && eu < d.n_events)) {
            atomicAdd(&d.off_image[eu], 1ull);
        }
        atomicAdd(&d.ev_collected_now[e], 1);
        return false;
    }
    return true;
}

// ---- per-slot step -------------------------------------------------------------------
// Returns true when the carrier stays active.
// CG: read the per-chunk partial sums and the positions through L2
// (ld.global.cg).  The fused kernels integrate an i-tile in the same launch
// that wrote its partial sums (and, in the persistent kernel, its positions)
// from other SMs, so this SM's L1 may hold a stale copy of their lines.
// advance_hole: hole `id` of event e (n_e active holes; read only with the
// Coulomb field on) at (x, y, z), whose per-chunk partial sums sit at slot p;
// on return (x, y, z) is the new position (also stored).  GIVEN: the caller
// passes (gx, gy, gz), the sums of the per-chunk partials accumulated from 0.0
// in chunk order (the same bits as the loop below), instead of slot p.
// FIELD = false: neither the Coulomb nor the stored-charge field is on (the
// O(N) path), so only Eq. 1 is formed.
template <bool F64, bool INIT, bool CG = false, bool GIVEN = false, bool FIELD = true>
__device__ __forceinline__ bool advance_hole(const Dev &d, int id, int e, int n_e, int p, long long step,
                                             double &x, double &y, double &z, double gx = 0.0,
                                             double gy = 0.0, double gz = 0.0) {
    const Phys &ph = d.phys;
    // INT: the FP32 forms' conversions and threshold tests by integer operations
    // (gc_bits.h; the same bits) where the FP64 unit's throughput bounds the
    // kernel -- the integrate kernel, one thread per hole.  The latency-bound
    // fused kernels (CG) keep the hardware operations, whose latency is lower.
    constexpr bool INT = !F64 && !CG;
    if (INIT) {
        if (ph.reflect && z > ph.thickness) {
            z = 2.0 * ph.thickness - z;
            d.pz[id] = z;
        }
    } else {
        double ex = 0.0, ey = 0.0, ez = 0.0;
        if (!FIELD) {
        } else if (ph.coulomb && GIVEN) {
            ex = gx;
            ey = gy;
            ez = gz;
        } else if (ph.coulomb) {  // Eq. 6: sum of the per-chunk partial sums, fixed order
            const int js = ceil_div(n_e, d.shape.jchunk);
            const long long st = d.part_stride;
            if (!GC_GUARD(p >= 0 && p < d.n_total)) return false;
            const double *P = d.partial + p;
            // fused kernels (few threads, latency-bound): the loads of up to 8
            // chunks are issued before their (ordered) sums, so the chunk count
            // does not chain memory round trips; the integrate kernel (1024
            // threads, 64 registers) hides the latency with threads instead
            constexpr int B = CG ? 8 : 1;
            for (int jc0 = 0; jc0 < js; jc0 += B) {
                double v[B][3];
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    if (jc0 + u < js) {
                        const double *Q = P + (long long)(jc0 + u) * 3 * st;
                        if (CG) {
                            v[u][0] = __ldcg(Q);
                            v[u][1] = __ldcg(Q + st);
                            v[u][2] = __ldcg(Q + 2 * st);
                        } else {
                            v[u][0] = Q[0];
                            v[u][1] = Q[st];
                            v[u][2] = Q[2 * st];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < B; ++u) {
                    if (jc0 + u == 0) {  // the first chunk (no addition to zero)
                        ex = v[u][0];
                        ey = v[u][1];
                        ez = v[u][2];
                    } else if (jc0 + u < js) {
                        ex += v[u][0];
                        ey += v[u][1];
                        ez += v[u][2];
                    }
                }
            }
        }
        double dx, dy, dz;
        if (F64 || (FIELD && ph.stored)) {  // the field in FP64 (the FP64 form; stored charge)
            if (FIELD && ph.coulomb) {
                ex *= ph.K;
                ey *= ph.K;
                ez *= ph.K;
            }
            if (FIELD && ph.stored) {  // the charge already in the event's pixels (Sec. 1)
                if (F64) {
                    const double4_32a r = d.sh64[p];
                    double sx, sy, sz;
                    stored_field<double>(d, e, r.x, r.y, r.z, sx, sy, sz);
                    ex += ph.K * sx;
                    ey += ph.K * sy;
                    ez += ph.K * sz;
                } else {  // the FP32 shadow may be tile-relative: use the event frame here
                    const float rx = (float)(x - d.ev_origin[3 * e]), ry = (float)(y - d.ev_origin[3 * e + 1]),
                                rz = (float)(z - d.ev_origin[3 * e + 2]);
                    float sx, sy, sz;
                    stored_field<float>(d, e, rx, ry, rz, sx, sy, sz);
                    ex += ph.K * (double)sx;
                    ey += ph.K * (double)sy;
                    ez += ph.K * (double)sz;
                }
            }
            if (FIELD) ez += ph.a1 * z - ph.a2;  // Eq. 1
            else ez = ph.a1 * z - ph.a2;
        }
        if (F64) {
            const double E = sqrt(ex * ex + ey * ey + ez * ez);
            const double mu = mobility64(ph, E);
            const double vdt = 1e4 * mu * ph.dt;  // um per (V/cm)
            dx = vdt * ex;
            dy = vdt * ey;
            dz = vdt * ez;
            if (ph.diffusion) {
                const double sigma = sqrt(2.0 * (1e8 * mu * ph.Vth) * ph.dt);
                double n[3];
                normals64(diffusion_bits(d.ev_seed[e], id - d.ev_first[e], step), n);
                dx += sigma * n[0];
                dy += sigma * n[1];
                dz += sigma * n[2];
            }
        } else {
            float n[3] = {0.0f, 0.0f, 0.0f};
            if (ph.diffusion) normals32(diffusion_bits(d.ev_seed[e], id - d.ev_first[e], step), n);
            // the FP32 forms round the field to FP32: formed in FP32 from the FP64
            // sums (K times each sum, plus Eq. 1), as the grid-resident kernel does;
            // without the Coulomb and stored-charge fields the lateral field is 0
            float fx = 0.0f, fy = 0.0f, fz;
            if (FIELD && ph.stored) {
                fx = cvt_d2f<INT>(ex);
                fy = cvt_d2f<INT>(ey);
                fz = cvt_d2f<INT>(ez);
            } else {
                fz = cvt_d2f<INT>(ph.a1 * z - ph.a2);  // Eq. 1
                if (FIELD && ph.coulomb) {
                    fx = ph.f_K * cvt_d2f<INT>(ex);
                    fy = ph.f_K * cvt_d2f<INT>(ey);
                    fz = fmaf(ph.f_K, cvt_d2f<INT>(ez), fz);
                }
            }
            float ddx, ddy, ddz;
            displacement32(ph, fx, fy, fz, n, ddx, ddy, ddz);
            dx = cvt_f2d<INT>(ddx);
            dy = cvt_f2d<INT>(ddy);
            dz = cvt_f2d<INT>(ddz);
        }
        x += dx;
        y += dy;
        z += dz;
        if (!INT) {
            if (ph.reflect && z > ph.thickness) z = 2.0 * ph.thickness - z;
        } else if (ph.reflect && gt_exact(z, ph.thickness)) {
            z = reflect_back(ph, z);
        }
        d.px[id] = x;
        d.py[id] = y;
        d.pz[id] = z;
    }
    return collect_check<INT>(d, id, e, step, x, y, z);
}

// One FP32-form step of hole `id` of event e at (x, y, z), with everything
// that does not depend on the position update given in FP32: the unscaled
// Eq. 6 sum (gx, gy, gz), the Eq. 1 field lin = a1 z - a2 at the hole, and
// the step's three normals.  The field is formed in FP32 (the other paths
// round it to FP32 as well), then the FP64 update, reflection, z check and
// binning of advance_hole follow.  For latency-bound callers: it keeps the
// FP64 unit off the chain but for the position update and the z check.
__device__ __forceinline__ bool advance_hole32(const Dev &d, int id, int e, long long step, double &x, double &y,
                                               double &z, float gx, float gy, float gz, float lin,
                                               const float n[3]) {
    const Phys &ph = d.phys;
    float ddx, ddy, ddz;
    displacement32(ph, ph.f_K * gx, ph.f_K * gy, fmaf(ph.f_K, gz, lin), n, ddx, ddy, ddz);
    x += ddx;  // hardware conversions and tests: on this latency chain they are faster
    y += ddy;  // than the integer forms (measured in the grid-resident kernel)
    z += ddz;
    if (ph.reflect && z > ph.thickness) z = 2.0 * ph.thickness - z;
    d.px[id] = x;
    d.py[id] = y;
    d.pz[id] = z;
    return collect_check<false>(d, id, e, step, x, y, z);
}

// advance_hole for the hole in slot p of the active list `cur`.
template <bool F64, bool INIT, bool CG = false, bool FIELD = true>
__device__ __forceinline__ bool advance_slot(const Dev &d, int cur, int p, long long step) {
    const int id = d.act[cur][p];
    const int e = d.ev_of_id[id];
    int n_e = 0;
    if (!INIT && FIELD && d.phys.coulomb) {
        const int *off = d.ev_off[cur];
        n_e = off[e + 1] - off[e];
    }
    double x, y, z;
    if (CG) {  // the fused kernels may integrate a hole on another SM than the last write
        x = __ldcg(d.px + id);
        y = __ldcg(d.py + id);
        z = __ldcg(d.pz + id);
    } else {
        x = d.px[id];
        y = d.py[id];
        z = d.pz[id];
    }
    return advance_hole<F64, INIT, CG, false, FIELD>(d, id, e, n_e, p, step, x, y, z);
}

}  // namespace gc
