/*
 * oracle.c -- FP64 CPU oracle of the G-CoReCCD transport step.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain C11, FP64 throughout,
 * OpenMP over field points only (each field point sums its sources
 * sequentially in the order given, so the result does not depend on the
 * thread count).  Compiled with -ffp-contract=off so that no multiply-add is
 * fused and the results are the same on every host.
 *
 * Every function follows the paper's equations in their printed order:
 *   Eq. 1  linear depletion field          E(z) = a1 z - a2
 *   Eq. 2  hole mobility                   mu(E, T)
 *   Eq. 3  diffusion step variance         sigma_D^2 = 2 D t_D
 *   Eq. 4  Einstein relation               D = k_B mu T / q
 *   Eq. 6  softened Coulomb field          E_j = K sum_i r_ij / (|r_ij|^2 + eps^2)^(3/2)
 *   Fig. 2 step sequence (Sec. 3.2): static field, Coulomb field, sum, |E|,
 *          mu, v, random diffusion vector, displacement, z check.
 *   Fig. 5 image: 2-D histogram of collected positions, pixel-sized bins.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- physical constants (CODATA 2018, exact SI values) ------------------ */
static const double ORC_Q = 1.602176634e-19;      /* elementary charge, C */
static const double ORC_KB = 1.380649e-23;        /* Boltzmann constant, J/K */
static const double ORC_EPS0 = 8.8541878128e-12;  /* vacuum permittivity, F/m */
static const double ORC_PI = 3.14159265358979323846;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. 2, evaluated as printed:
 *   mu = 1.31e8 T^-2.2 / [1 + (E / (1.24 T^1.68))^(0.46 T^0.17)]^(1 / (0.46 T^0.17)) */
double orc_mobility(double E_abs, double T) {
    double numerator = 1.31e8 * pow(T, -2.2);
    double E_crit = 1.24 * pow(T, 1.68);
    double beta = 0.46 * pow(T, 0.17);
    double ratio = E_abs / E_crit;
    double denominator = pow(1.0 + pow(ratio, beta), 1.0 / beta);
    return numerator / denominator;
}

/* Eq. 6: K = q / (4 pi eps0 eps_Si) in V m.  A source at distance r[um]
 * gives K / r^2 [V m / um^2] = K * 1e12 [V/m] = K * 1e10 [V/cm]. */
double orc_coulomb_K(double eps_rel) {
    double K_SI = ORC_Q / (4.0 * ORC_PI * ORC_EPS0 * eps_rel);
    return K_SI * 1e10;
}

/* Eq. 4: k_B T / q in volts. */
double orc_thermal_voltage(double T) { return ORC_KB * T / ORC_Q; }

/* ---- Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------
 * One round maps (x0, x1, x2, x3) with key (k0, k1) to
 *   (hi(M1*x2) ^ x1 ^ k0,  lo(M1*x2),  hi(M0*x0) ^ x3 ^ k1,  lo(M0*x0))
 * with the round multipliers M0 = 0xD2511F53, M1 = 0xCD9E8D57.  Between
 * rounds the key is advanced by the Weyl constants W0 = 0x9E3779B9 and
 * W1 = 0xBB67AE85.  Ten rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Textbook Box-Muller: for u_a in (0, 1] and u_b in [0, 1),
 *   n = sqrt(-2 ln u_a) cos(2 pi u_b),  n' = sqrt(-2 ln u_a) sin(2 pi u_b). */
void orc_diffusion_normals(uint64_t seed, uint32_t id, uint64_t step, double n[3]) {
    const double two_m32 = 1.0 / 4294967296.0;
    uint32_t ctr[4] = {id, (uint32_t)step, (uint32_t)(step >> 32), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    double ua = ((double)r[0] + 1.0) * two_m32;
    double ub = (double)r[1] * two_m32;
    double radius = sqrt(-2.0 * log(ua));
    n[0] = radius * cos(2.0 * ORC_PI * ub);
    n[1] = radius * sin(2.0 * ORC_PI * ub);
    double ua2 = ((double)r[2] + 1.0) * two_m32;
    double ub2 = (double)r[3] * two_m32;
    n[2] = sqrt(-2.0 * log(ua2)) * cos(2.0 * ORC_PI * ub2);
}

/* Eq. 6 at one field point t: sum over sources j of (r_t - r_j) /
 * (|r_t - r_j|^2 + eps^2)^(3/2).  The j = t term is zero because its
 * numerator is zero. */
static void field_at(const double *x, const double *y, const double *z,
                     const int64_t *src, int64_t n_src, int64_t t,
                     double eps2, double K, double E[3]) {
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t k = 0; k < n_src; ++k) {
        int64_t j = src[k];
        double rx = x[t] - x[j];
        double ry = y[t] - y[j];
        double rz = z[t] - z[j];
        double r2 = rx * rx + ry * ry + rz * rz + eps2;
        double denom = r2 * sqrt(r2); /* (r^2 + eps^2)^(3/2) */
        sx += rx / denom;
        sy += ry / denom;
        sz += rz / denom;
    }
    E[0] = K * sx;
    E[1] = K * sy;
    E[2] = K * sz;
}

void orc_coulomb_field(const double *x, const double *y, const double *z,
                       const int64_t *src, int64_t n_src,
                       const int64_t *targets, int64_t m,
                       double softening_um, double K, double *E) {
    double eps2 = softening_um * softening_um;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < m; ++t)
        field_at(x, y, z, src, n_src, targets[t], eps2, K, &E[3 * t]);
}

/* The per-carrier part of one step (Fig. 2), given the Coulomb field Ec at
 * the carrier's start-of-step position: static field (Eq. 1), sum, |E|,
 * mobility (Eq. 2), velocity, diffusion coefficient (Eq. 4) and step width
 * (Eq. 3), random diffusion vector, displacement, back-surface reflection. */
static void advance_one(const orc_params *p, double Vth, double x, double y, double z,
                        const double Ec[3], uint64_t seed, uint32_t id, uint64_t step,
                        double out[3]) {
    double Ez_static = p->a1 * z - p->a2;                /* Eq. 1 */
    double Ex = Ec[0], Ey = Ec[1], Ez = Ec[2] + Ez_static; /* sum of both fields */
    double E_abs = sqrt(Ex * Ex + Ey * Ey + Ez * Ez);
    double mu = orc_mobility(E_abs, p->T);                 /* Eq. 2 */
    double vx = 1e4 * mu * Ex, vy = 1e4 * mu * Ey, vz = 1e4 * mu * Ez; /* um/s */
    double dx = vx * p->dt_s, dy = vy * p->dt_s, dz = vz * p->dt_s;
    if (p->diffusion) {
        double D = 1e8 * mu * Vth;                         /* Eq. 4, um^2/s */
        double sigma = sqrt(2.0 * D * p->dt_s);            /* Eq. 3 */
        double nrm[3];
        orc_diffusion_normals(seed, id, step, nrm);
        dx += sigma * nrm[0];
        dy += sigma * nrm[1];
        dz += sigma * nrm[2];
    }
    double zn = z + dz;
    if (p->reflect_back && zn > p->thickness_um) zn = 2.0 * p->thickness_um - zn;
    out[0] = x + dx;
    out[1] = y + dy;
    out[2] = zn;
}

/* Field of the charge stored in one event's image at one point (Sec. 1:
 * charge already in a pixel deflects the charges that follow): pixel (ix, iy)
 * with count q is q charges at (ox + (ix + 1/2) p, oy + (iy + 1/2) p,
 * stored_z), each with the softened field of Eq. 6. */
static void stored_field_at(const orc_params *p, const uint32_t *img, const double origin[2],
                            double x, double y, double z, double K, double E[3]) {
    const double eps2 = p->softening_um * p->softening_um;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t iy = 0; iy < p->img_h; ++iy) {
        for (int64_t ix = 0; ix < p->img_w; ++ix) {
            const uint32_t q = img[iy * p->img_w + ix];
            if (q == 0) continue;
            double cx = origin[0] + ((double)ix + 0.5) * p->pixel_um;
            double cy = origin[1] + ((double)iy + 0.5) * p->pixel_um;
            double rx = x - cx, ry = y - cy, rz = z - p->stored_z_um;
            double r2 = rx * rx + ry * ry + rz * rz + eps2;
            double denom = r2 * sqrt(r2);
            sx += (double)q * (rx / denom);
            sy += (double)q * (ry / denom);
            sz += (double)q * (rz / denom);
        }
    }
    E[0] = K * sx;
    E[1] = K * sy;
    E[2] = K * sz;
}

void orc_stored_field(const orc_params *p, const uint32_t *img, const double origin[2],
                      const double *xyz, int64_t m, double *E) {
    const double K = orc_coulomb_K(p->eps_si_rel);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < m; ++t)
        stored_field_at(p, img, origin, xyz[3 * t], xyz[3 * t + 1], xyz[3 * t + 2], K, &E[3 * t]);
}

/* 2-D histogram with half-open bins [k p, (k+1) p) measured from the event's
 * image origin (Fig. 5). */
static void bin_collected(const orc_params *p, orc_state *s, int64_t e, double x, double y) {
    double fx = floor((x - s->img_origin[2 * e]) / p->pixel_um);
    double fy = floor((y - s->img_origin[2 * e + 1]) / p->pixel_um);
    if (fx >= 0.0 && fx < (double)p->img_w && fy >= 0.0 && fy < (double)p->img_h) {
        int64_t ix = (int64_t)fx, iy = (int64_t)fy;
        s->image[(e * p->img_h + iy) * p->img_w + ix] += 1u;
    } else {
        s->off_image[e] += 1;
    }
}

static int params_ok(const orc_params *p) {
    if (!(p->dt_s > 0.0) || !(p->T > 0.0) || !(p->pixel_um > 0.0)) return 0;
    if (p->img_w <= 0 || p->img_h <= 0) return 0;
    if (p->coulomb && !(p->softening_um > 0.0 && p->eps_si_rel > 0.0)) return 0;
    return 1;
}

int orc_init(const orc_params *p, orc_state *s) {
    if (!params_ok(p)) return -1;
    memset(s->image, 0, sizeof(uint32_t) * (size_t)s->n_events * p->img_w * p->img_h);
    memset(s->off_image, 0, sizeof(int64_t) * (size_t)s->n_events);
    s->step = 0;
    for (int64_t e = 0; e < s->n_events; ++e) {
        for (int64_t i = s->ev_off[e]; i < s->ev_off[e + 1]; ++i) {
            if (p->reflect_back && s->z[i] > p->thickness_um)
                s->z[i] = 2.0 * p->thickness_um - s->z[i];
            if (s->z[i] <= p->z_well_um) {
                s->collect_step[i] = 0;
                bin_collected(p, s, e, s->x[i], s->y[i]);
            } else {
                s->collect_step[i] = -1;
            }
        }
    }
    return 0;
}

int64_t orc_run(const orc_params *p, orc_state *s, int64_t steps) {
    if (!params_ok(p) || steps < 0) return -1;
    const double K = orc_coulomb_K(p->eps_si_rel);
    const double Vth = orc_thermal_voltage(p->T);
    int64_t done = 0;
    int64_t *active = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s->n > 0 ? s->n : 1));
    double *newpos = (double *)malloc(sizeof(double) * 3 * (size_t)(s->n > 0 ? s->n : 1));
    double *Ec = (double *)malloc(sizeof(double) * 3 * (size_t)(s->n > 0 ? s->n : 1));
    while (done < steps && s->step < p->max_steps) {
        uint64_t step = (uint64_t)s->step + 1; /* steps are numbered from 1 */
        int64_t n_active_total = 0;
        for (int64_t e = 0; e < s->n_events; ++e) {
            /* active carriers of this event, ascending id */
            int64_t na = 0;
            for (int64_t i = s->ev_off[e]; i < s->ev_off[e + 1]; ++i)
                if (s->collect_step[i] < 0) active[na++] = i;
            n_active_total += na;
            if (na == 0) continue;
            /* Coulomb field from the start-of-step positions (Eq. 6) */
            if (p->coulomb)
                orc_coulomb_field(s->x, s->y, s->z, active, na, active, na,
                                  p->softening_um, K, Ec);
            else
                memset(Ec, 0, sizeof(double) * 3 * (size_t)na);
            /* plus the field of the charge already stored in the event's pixels */
            if (p->stored_charge) {
                const uint32_t *img = s->image + (size_t)e * p->img_w * p->img_h;
#pragma omp parallel for schedule(static)
                for (int64_t k = 0; k < na; ++k) {
                    const int64_t i = active[k];
                    double Es[3];
                    stored_field_at(p, img, &s->img_origin[2 * e], s->x[i], s->y[i], s->z[i], K, Es);
                    Ec[3 * k] += Es[0];
                    Ec[3 * k + 1] += Es[1];
                    Ec[3 * k + 2] += Es[2];
                }
            }
            /* every carrier moves from the start-of-step state (synchronous update) */
#pragma omp parallel for schedule(static)
            for (int64_t k = 0; k < na; ++k) {
                int64_t i = active[k];
                advance_one(p, Vth, s->x[i], s->y[i], s->z[i], &Ec[3 * k], s->seeds[e],
                            (uint32_t)(i - s->ev_off[e]), step, &newpos[3 * k]);
            }
            /* commit, then check z (collection at the well) */
            for (int64_t k = 0; k < na; ++k) {
                int64_t i = active[k];
                s->x[i] = newpos[3 * k];
                s->y[i] = newpos[3 * k + 1];
                s->z[i] = newpos[3 * k + 2];
                if (s->z[i] <= p->z_well_um) {
                    s->collect_step[i] = (int32_t)step;
                    bin_collected(p, s, e, s->x[i], s->y[i]);
                }
            }
        }
        if (n_active_total == 0) break; /* every carrier has arrived */
        s->step = (int64_t)step;
        ++done;
    }
    free(active);
    free(newpos);
    free(Ec);
    return done;
}

void orc_step_targets(const orc_params *p, const double *x, const double *y,
                      const double *z, const int64_t *src, int64_t n_src,
                      const int64_t *targets, int64_t m, uint64_t seed,
                      uint64_t step, double *out) {
    const double K = orc_coulomb_K(p->eps_si_rel);
    const double Vth = orc_thermal_voltage(p->T);
    const double eps2 = p->softening_um * p->softening_um;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < m; ++t) {
        int64_t i = targets[t];
        double Ec[3] = {0.0, 0.0, 0.0};
        if (p->coulomb) field_at(x, y, z, src, n_src, i, eps2, K, Ec);
        advance_one(p, Vth, x[i], y[i], z[i], Ec, seed, (uint32_t)i, step, &out[3 * t]);
    }
}
