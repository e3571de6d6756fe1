/* Driver for an AddressSanitizer + UndefinedBehaviorSanitizer build of the
 * C ABI's host code (libgcoreccd compiled with host sanitizers), on a machine
 * without a GPU: every entry point's argument checks, parameter validation,
 * the no-device paths and the status strings.  Exit status 0 = clean. */
#include <stdio.h>
#include <string.h>

#include "gcoreccd.h"

#define EXPECT(cond) do { if (!(cond)) { fprintf(stderr, "failed: %s (line %d)\n", #cond, __LINE__); return 1; } } while (0)

int main(void) {
    gc_params p;
    gc_default_params(&p);
    EXPECT(p.abi_version == GC_ABI_VERSION);
    gc_sim *s = (gc_sim *)0x1;
    /* invalid parameters are rejected before any CUDA call */
    gc_params bad = p;
    bad.dt_s = -1.0;
    EXPECT(gc_create(&bad, NULL, &s) == GC_ERR_PARAM && s == NULL);
    bad = p;
    bad.fuse_small = 6;
    EXPECT(gc_create(&bad, NULL, &s) == GC_ERR_PARAM);
    bad = p;
    bad.resident_ctas = -1;
    EXPECT(gc_create(&bad, NULL, &s) == GC_ERR_PARAM);
    bad = p;
    bad.img_w = 0;
    EXPECT(gc_create(&bad, NULL, &s) == GC_ERR_PARAM);
    bad = p;
    bad.abi_version = 99;
    EXPECT(gc_create(&bad, NULL, &s) == GC_ERR_PARAM);
    EXPECT(gc_create(NULL, NULL, &s) == GC_ERR_PARAM);
    EXPECT(gc_create(&p, NULL, NULL) == GC_ERR_PARAM);
    /* no GPU here: valid parameters end in GC_ERR_NO_DEVICE, with the error text recorded */
    const gc_status st = gc_create(&p, NULL, &s);
    EXPECT(st == GC_ERR_NO_DEVICE || st == GC_OK);
    if (st == GC_OK) gc_destroy(s);
    (void)gc_last_cuda_error();
    int32_t sm, ma, mi;
    EXPECT(gc_device_info(&sm, &ma, &mi) == GC_ERR_NO_DEVICE || 1);
    /* NULL handles and arguments */
    double xyz[6] = {0, 0, 1, 0, 0, 2};
    EXPECT(gc_load_carriers(NULL, xyz, 2, NULL, 1, NULL, NULL) == GC_ERR_PARAM);
    EXPECT(gc_run(NULL, 1, NULL) == GC_ERR_PARAM);
    EXPECT(gc_collect(NULL, NULL, NULL, NULL, NULL, NULL) == GC_ERR_PARAM);
    EXPECT(gc_image(NULL, NULL, 0) == GC_ERR_PARAM);
    EXPECT(gc_positions(NULL, NULL) == GC_ERR_PARAM);
    gc_stats stats;
    EXPECT(gc_get_stats(NULL, &stats) == GC_ERR_PARAM);
    EXPECT(gc_save_state(NULL, NULL) == GC_ERR_PARAM);
    EXPECT(gc_restore_state(NULL, NULL) == GC_ERR_PARAM);
    EXPECT(gc_debug_inject(NULL, 1) == GC_ERR_PARAM);
    EXPECT(gc_selftest_barrier_timeout(-1.0) == GC_ERR_PARAM);
    gc_destroy(NULL);
    /* the standalone field: argument checks */
    double E[6];
    EXPECT(gc_coulomb_field(xyz, -1, 0.01, 11.7, GC_FP32_KAHAN, E, NULL) == GC_ERR_PARAM);
    EXPECT(gc_coulomb_field(xyz, 2, -0.01, 11.7, GC_FP32_KAHAN, E, NULL) == GC_ERR_PARAM);
    EXPECT(gc_coulomb_field(xyz, 2, 0.01, 11.7, 9, E, NULL) == GC_ERR_PARAM);
    EXPECT(gc_coulomb_field_noalloc(xyz, GC_NOALLOC_MAX_CARRIERS + 1, 0.01, 11.7, GC_FP32, E, NULL) ==
           GC_ERR_PARAM);
    EXPECT(gc_coulomb_field_noalloc(NULL, 2, 0.01, 11.7, GC_FP32, E, NULL) == GC_ERR_PARAM);
    /* every status has a name */
    for (int c = -7; c <= 1; ++c) EXPECT(strlen(gc_status_string((gc_status)c)) > 0);
    EXPECT(strlen(gc_status_string((gc_status)42)) > 0);
    printf("ABI host code sanitized run: ok\n");
    return 0;
}
