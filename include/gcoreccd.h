/*
 * gcoreccd.h -- C ABI of libgcoreccd, a GB300 (sm_103a) implementation of the
 * per-time-step hole transport of G-CoReCCD (Avalos & Sofo Haro,
 * arXiv 2203.11043): softened all-pairs Coulomb field (Eq. 6), drift in the
 * linear depletion field (Eq. 1) with the hole mobility of Eq. 2, thermal
 * diffusion (Eqs. 3-4), collection at the front-surface wells and binning of
 * collected charge into pixels (Sec. 3.2 / Fig. 2, Sec. 5.1 / Fig. 5).
 *
 * Units: positions in um, z = 0 at the collection surface and z = thickness
 * at the back (Sec. 2); t in s; E in V/cm; a1 in V/(cm um); a2 in V/cm;
 * mu in cm^2/(V s).  Drift v[um/s] = 1e4 mu E, D[um^2/s] = 1e8 mu kT/q.
 *
 * Conventions shared by every call:
 *  - No call aborts, prints, throws or exits; each returns a gc_status.
 *  - The caller owns every buffer it passes.  The library copies inputs
 *    during the call (host pointers) and owns its device workspace from
 *    gc_load_carriers until gc_destroy.
 *  - Host pointers may be pageable or pinned.  Per-carrier outputs are in the
 *    caller's original carrier order (carrier id = row index of the input).
 *  - A gc_sim is bound to the CUDA device that was current at gc_create and
 *    to one stream; calls on one gc_sim must not run concurrently.
 *  - Every device step runs in the library's own kernels; there is no CPU
 *    fallback.  Without a usable CUDA device, calls that touch the device
 *    return GC_ERR_NO_DEVICE.
 */
#ifndef GCORECCD_H
#define GCORECCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GC_ABI_VERSION 2u

typedef enum {
    GC_OK = 0,
    GC_INCOMPLETE = 1,           /* max_steps reached with carriers still active; outputs valid */
    GC_ERR_PARAM = -1,           /* invalid argument or parameter (nothing was changed) */
    GC_ERR_ALLOC = -2,           /* device or host allocation failed */
    GC_ERR_CUDA = -3,            /* a CUDA runtime call failed (see gc_last_cuda_error) */
    GC_ERR_STATE = -4,           /* call out of order (e.g. gc_run before gc_load_carriers) */
    GC_ERR_DEVICE_TIMEOUT = -5,  /* a bounded device-side wait expired; state is undefined */
    GC_ERR_NO_DEVICE = -6,       /* no CUDA device available */
    GC_ERR_DEVICE_CHECK = -7     /* a device-side consistency check failed (event offsets; in
                                    GC_DEBUG builds also slot, pixel and partial-sum indices);
                                    the access was skipped, state is undefined */
} gc_status;

/* Arithmetic of the Eq. 6 pair sum.  Positions, the pixel-boundary test and
 * the position update are FP64 in every mode. */
typedef enum {
    GC_FP64 = 0,        /* FP64 pair sum and FP64 mobility/diffusion (plain reference form) */
    GC_FP32 = 1,        /* FP32 pair sum, plain accumulation */
    GC_FP32_KAHAN = 2,  /* FP32 pair sum, Kahan-compensated across j-tiles */
    GC_FP16X2 = 3       /* packed half2 distance/rsqrt, FP32 accumulation with Kahan */
} gc_precision;

/* Simulation parameters: the parameter list of Sec. 3.2 (N comes with the
 * carriers; depth, thickness, a1, a2, well depth, maximum iterations, dt,
 * Coulomb on/off), the softening of Eq. 6, the image of Fig. 5, and the
 * library's execution knobs.  Fill with gc_default_params, then override. */
typedef struct {
    uint32_t abi_version;  /* must equal GC_ABI_VERSION */
    int32_t precision;     /* gc_precision */
    double thickness_um;   /* CCD thickness (Sec. 3.2) */
    double z_well_um;      /* well depth: a carrier is collected when z <= z_well (Sec. 3.2) */
    double a1_V_cm_um;     /* Eq. 1 slope */
    double a2_V_cm;        /* Eq. 1 offset */
    double T_K;            /* temperature (Eq. 2, Eq. 4) */
    double eps_si_rel;     /* relative permittivity of Si, K = q/(4 pi eps0 eps_si_rel) (Eq. 6) */
    double softening_um;   /* epsilon of Eq. 6; must be > 0 when coulomb != 0 */
    double dt_s;           /* time step dt (Fig. 2) */
    int64_t max_steps;     /* maximum number of iterations (Sec. 3.2) */
    int32_t coulomb;       /* 1: include Eq. 6 (Sec. 3.2 switch) */
    int32_t diffusion;     /* 1: include the Eq. 3 random displacement */
    int32_t reflect_back;  /* 1: reflect at z = thickness (also applied once at load) */
    int32_t img_w, img_h;  /* image size in pixels per event */
    double pixel_um;       /* pixel pitch (Fig. 5: 15 um) */
    int32_t graph_steps;   /* time steps per captured CUDA graph; 0 = eager launches */
    int32_t autotune;      /* 1: pick the pair-kernel shape (carriers per thread, kernel variant,
                              resident blocks per SM, j-chunk length, 4-lane threshold) by timing
                              candidates on sampled work items of the loaded carriers; the choice
                              is cached in the process per device, form and event-size histogram.
                              Skipped for one FP32 event that the grid-resident kernel runs
                              entirely (at most 4096 holes, fuse_small 1 or 4) */
    int32_t newton;        /* 1: one Newton step after the MUFU rsqrt (FP32 forms) */
    int32_t jchunk;        /* j-chunk length of a pair work item; 0 = automatic */
    int32_t pair_R;        /* carriers per thread in the FP32 pair kernel (2, 4, 8); 0 = automatic */
    int32_t timing;        /* 1: bracket every pair-kernel launch with CUDA events (gc_get_stats);
                              steps are then launched one by one instead of as graphs */
    int32_t stored_charge; /* 1: charge already collected in a pixel sources a field on the holes
                              still moving (Sec. 1): pixel count q = q charges at the pixel centre
                              at depth stored_z_um, softened as in Eq. 6; the image at the start of
                              each step; off-image charge is not stored */
    int32_t tile_frames;   /* 1 (FP32 forms): events of >= 2048 holes are ordered along a Morton
                              curve at load and their FP32 shadow is taken relative to the FP64
                              origin of each 256-slot tile instead of the event centroid, so close
                              pairs keep ~2^-24 of their tile's extent rather than of the event's;
                              costs a few percent of pair-kernel throughput; 0 = event frame */
    double stored_z_um;    /* depth of the stored-charge points */
    int32_t fuse_small;    /* while at most 8192 holes are active: 0 = the four-launch step
                              throughout; 2 = each step two launches (a pair kernel that also
                              integrates every i-tile once its last j-chunk is summed, then one
                              block that compacts); 3 = as 2, except that one event (FP64, FP32,
                              FP32 + Kahan) runs all its remaining steps in one cooperative
                              launch with one grid barrier per step (the persistent kernel);
                              4 = as 2, except that one FP32 / FP32 + Kahan event of at most
                              4096 active holes runs all its steps in one cooperative launch of
                              one CTA per SM, each CTA owning a fixed set of holes and the CTAs
                              exchanging step-tagged shadow words instead of passing a barrier
                              (the grid-resident kernel); 5 = as 2, except that one FP32 /
                              FP32 + Kahan event of at most 2048 active holes runs all its steps
                              in one thread-block cluster with its state in shared memory;
                              1 (default) = one FP32 / FP32 + Kahan event takes the persistent
                              kernel while more than 4096 holes are active and the grid-resident
                              kernel from there, one FP64 event the persistent kernel, a batch
                              the path of 2.  Paths 2 and 3 give the same results as the
                              four-launch step; the grid-resident and cluster kernels sum each
                              carrier's field in one piece with the lanes combined in FP32 (the
                              same FP32 error bound, not the same bits).  Not used with newton,
                              tile frames, stored charge or timing */
    int32_t resident_ctas; /* CTAs of the grid-resident kernel (fuse_small 1 or 4); 0 (default) =
                              one per 8 active holes at the launch, at most one per SM.  Clamped
                              to [ceil(n / 32), SMs] (each CTA owns at most 32 holes).  The
                              results do not depend on it, only the time */
} gc_params;

typedef struct gc_sim gc_sim;

/* Counters accumulated on the device since gc_load_carriers. */
typedef struct {
    int64_t steps;            /* time steps completed */
    int64_t n_active;         /* carriers still moving */
    int64_t n_collected;      /* carriers collected (in any pixel or off the image) */
    double pair_interactions; /* sum over steps of sum_e N_active,e^2 (Eq. 6 terms evaluated) */
    double carrier_steps;     /* sum over steps of the active carriers */
    int32_t pair_variant;     /* register blocking R of the FP32 pair kernel in use */
    int32_t pair_blocks;      /* persistent pair-kernel grid size */
    int32_t jchunk;           /* j-chunk length in use */
    int32_t launches_per_step;/* kernels launched per time step */
    double pair_kernel_ms;    /* with timing on: summed device time of the pair kernel */
    int64_t pair_kernel_launches; /* with timing on: pair-kernel launches that did work */
    double integrate_kernel_ms;   /* with timing on: summed device time of the integrate kernel */
    double compact_kernel_ms;     /* with timing on: summed device time of the compaction kernel */
    int64_t timed_steps;          /* with timing on: steps whose kernels were timed */
    int32_t device_loop;          /* 1: gc_run is one graph launch with a device-side loop
                                     (conditional WHILE node over passes of graph_steps steps) */
    int32_t fused_path;           /* small-workload path of the last gc_run: 0 none, 1 two launches
                                     per step, 2 the persistent single-event kernel, 3 the
                                     cluster-resident single-event kernel, 4 the grid-resident
                                     single-event kernel */
    double tune_ms;               /* autotuner: host time spent choosing the pair-kernel shape at the
                                     last gc_load_carriers (0 when cached or off) */
    int32_t tune_candidates;      /* shapes timed at the last load */
    int32_t tune_cached;          /* 1: the shape came from the in-process autotuner cache */
    int32_t pair_kernel_variant;  /* FP32 pair-kernel variant in use (0 default, 1 fewer loads in
                                     flight, 2 one more resident block per SM) */
    int32_t small_n;              /* events below this many active holes use 4 lanes per carrier */
} gc_stats;

/* Defaults: the CCD of the X-ray and muon workloads (thickness 675 um,
 * well at z = 0, a1 = 2 V/(cm um), a2 = 1500 V/cm, T = 140 K,
 * eps_Si = 11.7, eps = 0.01 um, dt = 10 ps, 15 um pixels on 64 x 64,
 * FP32 + Kahan, graphs of 32 steps, autotune on, timing off, fused small
 * steps on). */
void gc_default_params(gc_params *p);

/* Validate `p` (the Sec. 3.2 parameter list) and create an empty simulation
 * bound to the current CUDA
 * device and to `cuda_stream` (a cudaStream_t; NULL = a stream the library
 * creates and owns).  *out receives the handle.  GC_ERR_PARAM for an invalid
 * parameter (checked before any CUDA call); GC_ERR_NO_DEVICE without a GPU. */
gc_status gc_create(const gc_params *p, void *cuda_stream, gc_sim **out);

/* Load n carriers (host, row-major [n][3] x, y, z in um) grouped into n_events
 * independent events: event e owns rows [event_offsets[e], event_offsets[e+1])
 * (host int64 [n_events+1], starting at 0, non-decreasing, ending at n; NULL
 * means one event).  seeds (host uint64 [n_events]; NULL = all 1) keys each
 * event's Philox diffusion stream, whose counter is (index of the carrier
 * within its event, step), so an event's result does not depend on the other
 * events loaded with it.  img_origin_xy (host [n_events][2]; NULL =
 * each event's initial x-y centroid minus half the image) is the lower-left
 * image corner.  Carriers are reflected at the back surface if needed and
 * those already in the well are collected at step 0 (Fig. 2 z check).
 * Replaces any previously loaded carriers.  n may be 0. */
gc_status gc_load_carriers(gc_sim *s, const double *xyz, int64_t n,
                           const int64_t *event_offsets, int64_t n_events,
                           const uint64_t *seeds, const double *img_origin_xy);

/* Advance the simulation (the Fig. 2 loop): steps >= 0 runs at most that many
 * more time steps; steps < 0 runs until every carrier is collected.  Both
 * stop at max_steps.  *steps_done (nullable) receives the steps executed.
 * Returns GC_OK, or GC_INCOMPLETE when max_steps was reached with carriers
 * still active.  The call returns after the device has finished. */
gc_status gc_run(gc_sim *s, int64_t steps, int64_t *steps_done);

/* Copy out the collection results of the Fig. 2 z check -- the x-y position
 * at which each hole reached the wells, the data of the Sec. 5.1 / Fig. 5
 * histograms -- in original carrier order (all host pointers, each
 * nullable): final_xy [n][2] (position at collection; current
 * x, y for carriers still active), collect_step [n] (step of collection, 0 for
 * carriers in the well at load, -1 if still active), n_collected /
 * n_offimage / n_active [n_events] per event. */
gc_status gc_collect(gc_sim *s, double *final_xy, int32_t *collect_step,
                     int64_t *n_collected, int64_t *n_offimage, int64_t *n_active);

/* Copy the pixel histograms (Fig. 5), uint32 [n_events][img_h][img_w]
 * (row iy, column ix; pixel (ix, iy) holds x in [ox + ix p, ox + (ix+1) p)).
 * is_device != 0: `img` is a device pointer on this simulation's device. */
gc_status gc_image(gc_sim *s, uint32_t *img, int is_device);

/* Current positions [n][3] (host), original carrier order: the final
 * results that Sec. 3.2 saves to a file at the end of a run. */
gc_status gc_positions(gc_sim *s, double *xyz);

/* Device counters (host struct). */
gc_status gc_get_stats(gc_sim *s, gc_stats *st);

/* A checkpoint of a simulation, in caller-owned host buffers of the sizes
 * given.  Because the diffusion vectors are counter-based (Philox keyed by
 * the event seed, the carrier's index in its event and the step), this is the
 * whole state: a restored run continues exactly as the uninterrupted one. */
typedef struct {
    double *xyz;                  /* [n][3] current positions, original order */
    int32_t *collect_step;        /* [n] step of collection, -1 while active */
    uint32_t *image;              /* [n_events][img_h][img_w] */
    int64_t *off_image;           /* [n_events] */
    int64_t step;                 /* time steps completed */
    double pair_interactions;     /* counters of gc_stats, carried over */
    double carrier_steps;
} gc_state;

/* Copy the state into `st` (all its pointers must be valid host buffers). */
gc_status gc_save_state(gc_sim *s, gc_state *st);

/* Replace the state of `s` by `st`.  `s` must hold the same carriers, events,
 * seeds and image origins as the simulation the state was saved from
 * (gc_load_carriers with the same arguments); GC_ERR_PARAM when a saved
 * carrier is inconsistent (active but in the well, or beyond the back). */
gc_status gc_restore_state(gc_sim *s, const gc_state *st);

/* Eq. 6 on its own: the softened Coulomb field at every one of n carriers
 * from all n (one event), in V/cm.  xyz_dev: device [n][3] FP64 positions
 * (um); E_dev: device [n][3] FP64 output.  precision: gc_precision.  Runs on
 * `cuda_stream` (NULL = legacy default stream) and allocates its own
 * scratch (the FP32 position shadow and per-chunk partial sums) for the
 * duration of the call; returns after the device has finished. */
gc_status gc_coulomb_field(const double *xyz_dev, int64_t n, double softening_um,
                           double eps_si_rel, int32_t precision, double *E_dev,
                           void *cuda_stream);

/* Largest n accepted by gc_coulomb_field_noalloc. */
#define GC_NOALLOC_MAX_CARRIERS 32768

/* gc_coulomb_field for callers that cannot allocate device memory: code
 * running inside an allocator or memory pool it must not re-enter, inside a
 * framework that owns every device byte, or after a start-up phase beyond
 * which allocation is not allowed.  Same arguments, units, layout and result
 * as gc_coulomb_field (bit for bit in the FP64 form and, for the FP32 forms,
 * up to the order of the per-chunk partial sums whenever the scratch forces
 * longer j-chunks); every gc_precision is accepted.  The paper has no
 * counterpart of this entry point.  It calls no cudaMalloc, cudaFree or other
 * allocating routine: its scratch (about 7.3 MB: control block, the position
 * shadow and the per-chunk partial sums) is a fixed device array inside the
 * library, held by every GPU that loads it until the process exits.  n above
 * GC_NOALLOC_MAX_CARRIERS returns GC_ERR_PARAM.  The first call on each device
 * looks up that array's device address (with the device current), so make
 * that first call before any stream capture.  Every call shares the array and
 * finds the previous call's contents there; the call resets what must start
 * from zero, but calls whose work overlaps on the GPU (other streams or host
 * threads) race and must be serialised by the caller.  The call synchronizes
 * `cuda_stream` before it returns; a failed CUDA call returns its status with
 * the text in gc_last_cuda_error. */
gc_status gc_coulomb_field_noalloc(const double *xyz_dev, int64_t n, double softening_um,
                                   double eps_si_rel, int32_t precision, double *E_dev,
                                   void *cuda_stream);

/* Fault planting for tests of the device-side checks (no counterpart in the
 * paper), effective only in builds compiled with GC_DEBUG (GC_ERR_STATE
 * otherwise): what = 1 makes the next gc_load_carriers of `s` upload event
 * offsets that do not match its carriers.  The load then succeeds, no kernel
 * uses the offsets (the step-0 pass checks them first), and gc_run returns
 * GC_ERR_DEVICE_CHECK.  what = 2 makes one CTA of the next grid-resident
 * launch of `s` withhold its first step's words: every other CTA's bounded
 * wait runs out (1 s) and gc_run returns GC_ERR_DEVICE_TIMEOUT, with nothing
 * faulted or hung.  what = 0 cancels. */
gc_status gc_debug_inject(gc_sim *s, int32_t what);

/* Self-test of the library's bounded device-side wait (the grid barrier of
 * the persistent single-event kernel; no counterpart in the paper): runs, on
 * the current device, a barrier that waits for one block more than the grid
 * has, so nothing can complete it.  Every block must give up after limit_s
 * seconds (0 < limit_s <= 10) and report it.  Returns GC_ERR_DEVICE_TIMEOUT
 * when the wait ran out as designed (the device stays usable), GC_OK if it
 * did not, GC_ERR_NO_DEVICE without a GPU that supports cooperative launches.
 * A simulation whose wait runs out returns GC_ERR_DEVICE_TIMEOUT from gc_run
 * and must be destroyed. */
gc_status gc_selftest_barrier_timeout(double limit_s);

/* Free everything owned by the simulation (NULL is a no-op); the end of the
 * Sec. 3.2 run, after which no result of `s` can be read. */
void gc_destroy(gc_sim *s);

/* Static, human-readable name of a status code. */
const char *gc_status_string(gc_status st);

/* Text of the last CUDA error seen by this thread (static buffer). */
const char *gc_last_cuda_error(void);

/* Number of SMs and the sm_XY version of the current device (for reports);
 * GC_ERR_NO_DEVICE without a GPU. */
gc_status gc_device_info(int32_t *sm_count, int32_t *cc_major, int32_t *cc_minor);

#ifdef __cplusplus
}
#endif
#endif
