/* Driver for an AddressSanitizer + UndefinedBehaviorSanitizer build of the
 * FP64 oracle (oracle/oracle.c): runs every oracle function on a small
 * ragged batch (an empty event, a single carrier, carriers already in the
 * well or beyond the back surface), with the Coulomb field, diffusion,
 * reflection and the stored-charge field on, and checks that every event's
 * charge is conserved.  Exit status 0 = clean (the sanitizers abort on the
 * first error). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "../../oracle/oracle.h"

int main(void) {
    enum { E = 6 };
    const int64_t sizes[E] = {40, 0, 1, 25, 7, 30};
    const double z0[E] = {3.0, 5.0, 4.0, -1.0, 676.0, 1.5};
    int64_t off[E + 1] = {0};
    for (int e = 0; e < E; ++e) off[e + 1] = off[e] + sizes[e];
    const int64_t n = off[E];
    double *x = malloc(n * sizeof(double)), *y = malloc(n * sizeof(double)), *z = malloc(n * sizeof(double));
    int32_t *cs = malloc(n * sizeof(int32_t));
    uint64_t seeds[E];
    double origin[2 * E];
    unsigned r = 12345u;
    for (int e = 0; e < E; ++e) {
        seeds[e] = 100 + e;
        origin[2 * e] = origin[2 * e + 1] = -8.0;
        for (int64_t i = off[e]; i < off[e + 1]; ++i) {
            r = r * 1664525u + 1013904223u;
            x[i] = ((r >> 8) & 0xffff) / 65536.0 - 0.5;
            r = r * 1664525u + 1013904223u;
            y[i] = ((r >> 8) & 0xffff) / 65536.0 - 0.5;
            z[i] = z0[e] + 0.1 * (((r >> 4) & 0xff) / 256.0);
        }
    }
    orc_params p = {675.0, 0.0, 2.0, 1500.0, 140.0, 11.7, 0.01, 1e-11, 20000, 1, 1, 1, 1.0, 16, 16, 1, 0, -0.2};
    uint32_t *img = calloc((size_t)E * 16 * 16, sizeof(uint32_t));
    int64_t offimg[E] = {0};
    orc_state s = {n, E, x, y, z, off, seeds, origin, cs, img, offimg, 0};
    int rc = 0;
    if (orc_init(&p, &s) != 0) rc = 1;
    const int64_t steps = rc ? 0 : orc_run(&p, &s, (int64_t)1 << 40);  /* until done (or max_steps) */
    for (int e = 0; e < E && !rc; ++e) {
        int64_t in_img = 0, done = 0;
        for (int k = 0; k < 16 * 16; ++k) in_img += img[e * 256 + k];
        for (int64_t i = off[e]; i < off[e + 1]; ++i) done += cs[i] >= 0;
        if (in_img + offimg[e] != done || done != sizes[e]) {
            fprintf(stderr, "event %d: image %lld + off %lld, collected %lld of %lld\n", e, (long long)in_img,
                    (long long)offimg[e], (long long)done, (long long)sizes[e]);
            rc = 2;
        }
    }
    /* the other entry points */
    int64_t src[8], tg[3] = {0, 3, 7};
    for (int k = 0; k < 8; ++k) src[k] = k;
    double E3[9], out[9], nrm[3], Es[6];
    orc_coulomb_field(x, y, z, src, 8, tg, 3, 0.01, orc_coulomb_K(11.7), E3);
    orc_step_targets(&p, x, y, z, src, 8, tg, 3, 7, 1, out);
    orc_diffusion_normals(1, 2, 3, nrm);
    const uint32_t ctr[4] = {1, 2, 3, 4}, key[2] = {5, 6};
    uint32_t ph[4];
    orc_philox4x32_10(ctr, key, ph);
    const double pts[6] = {0.5, 0.5, 1.0, -3.0, 2.0, 4.0};
    orc_stored_field(&p, img, origin, pts, 2, Es);
    const double mu = orc_mobility(1500.0, 140.0) + orc_thermal_voltage(140.0);
    if (!rc && (!(steps > 0) || !isfinite(mu) || !isfinite(E3[0] + out[0] + nrm[0] + Es[0]))) rc = 3;
    if (!rc) printf("oracle sanitized run: %lld steps, %lld carriers\n", (long long)steps, (long long)n);
    else fprintf(stderr, "oracle sanitized run failed: %d\n", rc);
    free(x); free(y); free(z); free(cs); free(img);
    return rc;
}
