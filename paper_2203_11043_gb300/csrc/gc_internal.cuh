// gc_internal.cuh -- device-side state, physics constants and helpers shared by
// the kernels of libgcoreccd (G-CoReCCD hole transport, arXiv 2203.11043).
//
// Data layout in HBM (N = carriers loaded, E = events, S = j-chunks):
//   per carrier, by original id:  px, py, pz (FP64 SoA), ev_of_id (int32),
//                                 collect_step (int32, -1 while active)
//   per active slot (compacted, grouped by event; inside an event ascending
//   id, or load-time Morton order for large events with tile frames):
//                                 act[cur] (id), sh32 (float4 shadow x,y,z
//                                 relative to its frame: the event centroid,
//                                 or with tile frames, for events of >=
//                                 small_n holes, the first hole of its
//                                 256-slot tile counted from the event
//                                 start) or sh64 (double4_32a, FP64 form,
//                                 event frame), frame_hi/frame_lo (tile
//                                 frames: the FP64 origin at each tile start
//                                 as an FP32 hi + lo pair), partial (FP64,
//                                 [S][3][N]), keepmask (1 bit per slot)
//   per event (internal order = descending initial size):
//                                 ev_off[cur] (active offsets), item_base
//                                 (pair work-item prefix), seeds, origins
//   per user event:               image [E][H][W] uint32, off_image uint64
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "gc_bits.h"

namespace gc {

constexpr int kChunk = 4096;        // slots per integrate/compact chunk
constexpr int kChunkThreads = 1024; // threads per integrate/compact block
constexpr int kPairThreads = 128;   // threads per pair-kernel block
constexpr int kTileJ = 256;         // j positions staged in shared memory per tile
constexpr int kTileJ64 = 64;        // FP64 form: granularity of its j-chunks
constexpr int kFusedMax = 8192;     // fused small-workload step while at most this many holes are active
constexpr float kSentinel = 1.0e15f; // padding position: its Eq. 6 term rounds to 0
constexpr int kSmallEvent = 2048;    // FP32 forms: smaller events split j over 4 lanes and use
                                     // the event frame; larger ones one lane (and, with
                                     // tile_frames, tile frames).  Measured on 4096 X-ray
                                     // events (267..4800 holes): 2048 is 4.7 % faster than
                                     // 8192 and keeps a 1573-hole event on 4 lanes

// Control block: one per simulation, written only by the device during a run.
struct Ctrl {
    long long step;          // time steps completed
    long long step_limit;    // stop when step reaches this (set by the host)
    long long loop_last;     // step seen by the previous pass of a device-side loop
    long long stop_below;    // steps pause once at most this many carriers are active (set by
                             // the host: the hand-over to the grid-resident kernel; 0 = never)
    int n_active;            // active carriers at the start of the next step
    int cur;                 // which of the double-buffered active lists is current
    int items_total;         // pair work items for the next step
    unsigned work_counter;   // next pair work item to hand out
    unsigned long long carrier_steps;     // sum of active carriers over steps
    unsigned long long pair_interactions; // sum over steps of sum_e n_e^2
    int error;               // device-detected inconsistency (bit flags)
    int tiles_total;         // i-tiles of the next step (fused small-workload path)
    unsigned bar_count;      // grid barrier of the persistent single-event kernel:
    unsigned bar_gen;        //   arrivals and generation
    unsigned se_item[2];     // its work-item counters, by step parity (FP64 form)
};

// Physics and geometry, precomputed on the host from gc_params.
struct Phys {
    double a1, a2;           // Eq. 1
    double thickness, z_well;
    double dt;
    double K;                // Eq. 6 constant, V/cm * um^2
    double eps2;             // softening^2, um^2
    double mu0;              // Eq. 2: 1.31e8 T^-2.2
    double inv_Ec;           // Eq. 2: 1 / (1.24 T^1.68)
    double beta, inv_beta;   // Eq. 2: 0.46 T^0.17 and its inverse
    double Vth;              // k_B T / q, V (Eq. 4)
    double pixel;            // pixel pitch, um
    int img_w, img_h;
    int coulomb, diffusion, reflect;
    int stored;              // stored-charge field on (Sec. 1)
    double stored_z;         // depth of the stored-charge points, um
    // the FP32 forms' copies (rounded to nearest on the host, as a device conversion
    // would: a double-to-float conversion on the device is a long-latency FP64-unit step)
    float f_a1, f_dt, f_K, f_mu0, f_inv_Ec, f_beta, f_inv_beta, f_Vth;
};

// Pair-kernel work decomposition, fixed at load time.
struct PairShape {
    int R;           // i carriers per thread (register blocking; 1 in the FP64 form)
    int jchunk;      // j-chunk length of a work item (multiple of kTileJ; of kTileJ64 in FP64)
    int small_n;     // events with fewer active carriers use small_lanes lanes per i-group
    int small_lanes; // lanes per i-group of small events: 4 (FP32 forms) or 16 (FP64 form)
    int n_blocks;    // persistent grid size
    int V;           // pair-kernel variant chosen by the autotuner (0 = default)
};

// Device view of a simulation, passed by value to every kernel.
struct Dev {
    double *px, *py, *pz;
    int *ev_of_id;
    int *collect_step;
    int *act[2];
    float4 *sh32;
    double4_32a *sh64;
    float4 *frame_hi;        // FP32 forms, large events: frame origin at each tile-start slot,
    float4 *frame_lo;        //   as float(o) and float(o - float(o))
    int tile_frames;         // 1: large events use 256-slot tile frames (FP32 forms)
    double *partial;
    long long part_stride;
    unsigned *keepmask;
    int *chunk_cnt;
    int *ev_off[2];
    int *ev_collected_now;
    int *item_base;
    unsigned long long *ev_seed;
    double *ev_origin;       // [E][3]
    unsigned *ev_ext[2];     // FP16x2 form: [E] max |shadow coordinate| (float bits), per buffer
    double *img_origin;      // [E][2]
    int *ev_user;            // internal -> caller event index
    int *ev_first;           // internal event -> id of its first carrier
    unsigned *image;         // [E_user][H][W]
    int *occ_pix;            // stored charge: occupied pixel indices, per event in index order
    int *occ_off;            // [E+1] capacity offsets of each event's occupied-pixel list
    int *occ_cnt;            // [E] occupied pixels this step
    unsigned *occ_q;         // stored charge: exact count of each listed pixel at the step start
    float4 *occ_f4;          // stored charge, FP32 forms: (centre x, y relative to the event origin, count, 0)
    unsigned long long *off_image;
    // fused small-workload path: per i-tile prefix over events [E+1], one
    // ticket per i-tile (counts the j-chunk items done), one keep byte per slot
    int *tile_base;
    unsigned *tile_ticket;
    unsigned char *keep8;
    // persistent single-event kernel: shadows indexed by a hole's stable index
    // (its slot at the launch), two buffers read and written on alternate
    // steps, and keep bytes per step parity
    float4 *se_sh32[2];
    double4_32a *se_sh64[2];
    unsigned char *se_keep[2];
    // grid-resident single-event kernel: each hole's published words (FP32
    // shadow coordinate + step tag + keep bit), [parity][coordinate][slot at launch]
    unsigned long long *rs_rec;
    int dbg_withhold;        // GC_DEBUG builds: CTA 1 of the grid-resident kernel withholds its
                             // first step's words (gc_debug_inject 2)
    Ctrl *ctrl;
    int n_total;
    int n_events;
    PairShape shape;
    Phys phys;
};

// Number of lanes sharing one i-group in the pair kernel for an event of n
// active carriers, and the i-tile length that follows from it.
// Integrate: with at most kFineMaxChunks chunks active, each chunk is split
// into kFineUnit-slot units so that a small step spreads over many SMs (the
// per-hole FP64 update would otherwise run on one SM); chunk counts are then
// accumulated with atomics into counters the finalize kernel has zeroed.
constexpr int kFineUnit = 256;
constexpr int kFineMaxChunks = 8;
__host__ __device__ inline bool fine_units(int n_act) { return (n_act + kChunk - 1) / kChunk <= kFineMaxChunks; }
__host__ __device__ inline int lanes_for(const PairShape &sh, int n) { return n < sh.small_n ? sh.small_lanes : 1; }
__host__ __device__ inline int itile_for(int R, int lanes) { return R * kPairThreads / lanes; }
__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Ctrl::error bits (the host maps them to a status after each run).
constexpr int kErrBarrierTimeout = 1;  // a grid-barrier wait ran out
constexpr int kErrOffsets = 2;         // the active event offsets are inconsistent
constexpr int kErrIndex = 4;           // a GC_DEBUG bounds check failed (the access was skipped)

// A step is skipped when the run limit is reached, nothing is active, or a
// device-side check has failed (no kernel then uses the state again); the
// steps of every path but the grid-resident kernel also pause once at most
// stop_below carriers are active, so that it takes over at a step fixed by
// the state alone.
__device__ inline bool run_over(const Ctrl *c) {
    return c->step >= c->step_limit || c->n_active <= 0 || c->error != 0;
}
__device__ inline bool step_skipped(const Ctrl *c) { return run_over(c) || c->n_active <= c->stop_below; }

// GC_DEBUG builds check the index behind each data-dependent access: a failed
// check sets kErrIndex and the access is skipped (never a trap).  Release
// builds compile the checks away.
__device__ __forceinline__ bool guard_ok(bool ok, Ctrl *c) {
    if (!ok) atomicOr(&c->error, kErrIndex);
    return ok;
}
#ifdef GC_DEBUG
#define GC_GUARD(cond) (::gc::guard_ok((cond), d.ctrl))
#else
#define GC_GUARD(cond) (true)
#endif

// ---- Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) --------------------
// Ten rounds of the 4x32 Philox S-box with multipliers 0xD2511F53 and
// 0xCD9E8D57; the key advances by 0x9E3779B9 / 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Counter of the diffusion stream: (carrier index within its event, step lo,
// step hi, 0), keyed by the event seed, so an event's random vectors do not
// depend on the other events of a batch.
__device__ __forceinline__ uint4 diffusion_bits(unsigned long long seed, int id, long long step) {
    return philox4x32_10(make_uint4((unsigned)id, (unsigned)step,
                                    (unsigned)((unsigned long long)step >> 32), 0u),
                         make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

// ---- packed FP32 (sm_100+ f32x2) helpers -----------------------------------
typedef unsigned long long f2;  // two FP32 lanes in one 64-bit register pair

__device__ __forceinline__ f2 pack2(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(f2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// ---- packed FP16 helpers (FP16x2 form) -------------------------------------
// Two FP32 values rounded to one f16x2 register (lo in the low half).
__device__ __forceinline__ unsigned f2_to_h2(f2 v) {
    float lo, hi;
    unpack2(v, lo, hi);
    unsigned h;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(hi), "f"(lo));
    return h;
}
__device__ __forceinline__ unsigned hfma2(unsigned a, unsigned b, unsigned c) {
    unsigned d;
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ void h2_to_f(unsigned h, float &lo, float &hi) {
    asm("{\n\t.reg .b16 l, u;\n\tmov.b32 {l, u}, %2;\n\tcvt.f32.f16 %0, l;\n\t"
        "cvt.f32.f16 %1, u;\n\t}" : "=f"(lo), "=f"(hi) : "r"(h));
}
// Power-of-two scale s for an event whose shadow coordinates satisfy
// |c| <= ext: then |r_i - r_j|^2 s^2 <= 12 ext^2 s^2 <= 2^15, inside f16 range.
__device__ __forceinline__ float h2_scale(float ext) {
    const float e = fmaxf(ext, 1e-6f);
    const int k = (int)floorf(log2f(52.0f / e));
    return exp2f((float)min(max(k, -30), 20));
}

// Hardware reciprocal square root on the MUFU pipe (approximate).
__device__ __forceinline__ float rsqrt_mufu(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 16-byte asynchronous global -> shared copies (no register staging); both
// addresses 16-byte aligned.  The _zfill form copies `bytes` (0 or 16) and
// zero-fills the rest.  cp_async_wait_all() waits for this thread's copies.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_zfill(void *smem, const void *gmem, unsigned bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace gc
