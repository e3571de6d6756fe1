/*
 * oracle.h -- FP64 CPU oracle of the G-CoReCCD hole-transport step
 * (Avalos & Sofo Haro, arXiv 2203.11043).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain, obviously
 * correct statement of what one transport step computes.  It exists to check
 * the CUDA library against.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product path never calls it
 * and shares no code, header, table or constant with it.
 *
 * Units (same reading as the CUDA library, restated here independently):
 *   positions in um; z = 0 is the collection (front) surface, z = thickness
 *   the back surface (Sec. 2, Fig. 1);  t in s;  E in V/cm;
 *   a1 in V/(cm um), a2 in V/cm (Eq. 1);  mu in cm^2/(V s) (Eq. 2);
 *   drift v[um/s] = 1e4 mu E;  D[um^2/s] = 1e8 mu kT/q (Eq. 4).
 *
 * Functions whose arithmetic has no independent pin are marked
 * "parity unpinned" below (none at present: every function is pinned by a
 * closed form, a printed constant or an invariant in tests/).
 */
#ifndef GCORECCD_ORACLE_H
#define GCORECCD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Simulation parameters (the parameter list of Sec. 3.2, plus the
 * softening of Eq. 6 and the image geometry of Sec. 5.1 / Fig. 5). */
typedef struct {
    double thickness_um;   /* CCD thickness */
    double z_well_um;      /* depth of the potential well: collected when z <= z_well */
    double a1;             /* Eq. 1 slope, V/(cm um) */
    double a2;             /* Eq. 1 offset, V/cm */
    double T;              /* temperature, K (Eq. 2, Eq. 4) */
    double eps_si_rel;     /* relative permittivity of Si (Eq. 6: K = q / (4 pi eps0 eps_Si)) */
    double softening_um;   /* epsilon of Eq. 6 */
    double dt_s;           /* time step */
    int64_t max_steps;     /* maximum number of iterations (Sec. 3.2) */
    int32_t coulomb;       /* Coulomb repulsion on/off (Sec. 3.2) */
    int32_t diffusion;     /* thermal diffusion on/off */
    int32_t reflect_back;  /* reflect at z = thickness */
    double pixel_um;       /* pixel pitch of the output histogram (Fig. 5: 15 um) */
    int32_t img_w, img_h;  /* image size in pixels */
    int32_t stored_charge; /* 1: charge already collected in a pixel sources a field (Sec. 1) */
    int32_t pad;
    double stored_z_um;    /* depth of the stored-charge points (pixel centres at this z) */
} orc_params;

/* Simulation state.  All arrays are caller-owned; positions are updated in
 * place.  Carrier ids are 0..n-1; event e owns ids [ev_off[e], ev_off[e+1]). */
typedef struct {
    int64_t n;
    int64_t n_events;
    double *x, *y, *z;          /* [n] current positions (final positions once collected) */
    const int64_t *ev_off;      /* [n_events+1] */
    const uint64_t *seeds;      /* [n_events] diffusion-stream key of each event */
    const double *img_origin;   /* [n_events][2] lower-left corner of each event's image, um */
    int32_t *collect_step;      /* [n] step at which the carrier was collected, -1 while active */
    uint32_t *image;            /* [n_events][img_h][img_w] collected-charge histogram */
    int64_t *off_image;         /* [n_events] collected carriers outside the image */
    int64_t step;               /* time steps completed so far */
} orc_state;

/* Eq. 2: hole mobility mu(|E|, T) in cm^2/(V s); |E| in V/cm, T in K. */
double orc_mobility(double E_abs, double T);

/* Eq. 6 constant K = q / (4 pi eps0 eps_rel) expressed so that
 * E[V/cm] = K * sum r[um] / (r^2 + eps^2)^(3/2) [um^-2]. */
double orc_coulomb_K(double eps_rel);

/* k_B T / q in volts (Eq. 4). */
double orc_thermal_voltage(double T);

/* Philox-4x32-10 block function (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The three N(0,1) diffusion normals of carrier `id` at step `step`
 * (counter = (id, lo32(step), hi32(step), 0), key = (lo32(seed), hi32(seed)),
 * textbook Box-Muller on the 32-bit outputs).  `id` is the carrier's index
 * within its event and `seed` the event's key, so an event's random vectors
 * do not depend on the other events simulated with it. */
void orc_diffusion_normals(uint64_t seed, uint32_t id, uint64_t step, double n[3]);

/* Eq. 6 field, in V/cm, at each of the m target carriers targets[t] from
 * every source j in src[0..n_src) (indices into x,y,z), summed in the order
 * given.  Output E[t*3 + c]. */
void orc_coulomb_field(const double *x, const double *y, const double *z,
                       const int64_t *src, int64_t n_src,
                       const int64_t *targets, int64_t m,
                       double softening_um, double K, double *E);

/* Reflect positions beyond the back surface and collect carriers already in
 * the well (step 0).  Initialises collect_step, image and off_image. */
int orc_init(const orc_params *p, orc_state *s);

/* Run up to `steps` time steps (Fig. 2 sequence), stopping early when no
 * carrier is active or max_steps is reached.  Returns the steps executed,
 * or -1 on invalid arguments. */
int64_t orc_run(const orc_params *p, orc_state *s, int64_t steps);

/* Field in V/cm at the m points xyz[3t..3t+2] from the charge stored in one
 * event's image (img [img_h][img_w], lower-left corner origin[2]): each pixel
 * with count q acts as q point charges at its centre at depth stored_z_um,
 * with the softened form of Eq. 6; pixels are summed in index order. */
void orc_stored_field(const orc_params *p, const uint32_t *img, const double origin[2],
                      const double *xyz, int64_t m, double *E);

/* One step for a sample of carriers of a single event whose carriers are
 * x, y, z[0..) (so an index is also the index within the event), without
 * committing: the field at each target comes from all sources src[0..n_src)
 * (active carriers of the event, ascending index); out[t*3+c] is the new
 * position of carrier targets[t] at step `step` (reflection applied, no
 * collection). */
void orc_step_targets(const orc_params *p, const double *x, const double *y,
                      const double *z, const int64_t *src, int64_t n_src,
                      const int64_t *targets, int64_t m, uint64_t seed,
                      uint64_t step, double *out);

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
