/* Calls the host-side entry points of the C-ABI under AddressSanitizer and
 * UndefinedBehaviorSanitizer (built by tests/test_host_sanitizers.py) on a machine without
 * a GPU: defaults, sizes, footprints and batch work sizes over the parameter ranges,
 * argument errors, and context creation failing cleanly. Exit status 0 on success. */
#include <stdio.h>
#include <string.h>

#include "pkmom.h"

static int fails = 0;
#define CHECK(c)                                                      \
    do {                                                              \
        if (!(c)) {                                                   \
            fprintf(stderr, "%s:%d: %s\n", __FILE__, __LINE__, #c);  \
            ++fails;                                                  \
        }                                                             \
    } while (0)

int main(void)
{
    pkmom_params p;
    pkmom_params_default(&p, 1000.0, 256, 128);
    CHECK(p.order == 4 && p.nbins == 128 && p.kmax_kf == 128.0);
    CHECK(pkmom_grid_bytes(256, PKMOM_F32) == (size_t)4 * 256 * 256 * 258 * 4);
    const int grids[] = {16, 24, 64, 128, 384, 512, 1024};
    const long long counts[] = {1, 1000, 1000000, 134217728};
    for (int g = 0; g < 7; ++g)
        for (int c = 0; c < 4; ++c)
            for (int prec = 0; prec < 2; ++prec)
                for (int order = 1; order <= 5; ++order) {
                    pkmom_params_default(&p, 500.0, grids[g], 64);
                    p.precision = prec;
                    p.order = order;
                    const size_t s = pkmom_assign_scratch_bytes(&p, counts[c]);
                    const size_t f = pkmom_footprint_bytes(&p, counts[c]);
                    CHECK(s > 0 && f > s);
                }
    /* invalid parameters give 0, not a fault */
    pkmom_params_default(&p, 500.0, 20, 64);
    CHECK(pkmom_assign_scratch_bytes(&p, 1000) == 0);
    pkmom_params_default(&p, -1.0, 64, 64);
    CHECK(pkmom_footprint_bytes(&p, 1000) == 0);
    CHECK(pkmom_assign_scratch_bytes(NULL, 1000) == 0);
    /* batch work sizes */
    pkmom_batch_item items[3];
    memset(items, 0, sizeof items);
    for (int k = 0; k < 3; ++k) pkmom_params_default(&items[k].p, 300.0, 32 * (k + 1), 10 + k);
    items[2].p.precision = PKMOM_F64;
    CHECK(pkmom_batch_work_bytes(3, items) > 0);
    CHECK(pkmom_batch_work_bytes(0, items) == 0);
    CHECK(pkmom_batch_work_bytes(PKMOM_BATCH_MAX + 1, items) == 0);
    items[1].p.nbins = 0;
    CHECK(pkmom_batch_work_bytes(3, items) == 0);
    /* strings, and no context on a machine without a GPU */
    for (int st = -9; st <= 1; ++st) CHECK(pkmom_strerror((pkmom_status)st) != NULL);
    pkmom_ctx *ctx = (pkmom_ctx *)0x1;
    CHECK(pkmom_create(&ctx, 0) != PKMOM_OK && ctx == NULL);
    CHECK(pkmom_destroy(NULL) == PKMOM_EINVAL);
    CHECK(pkmom_sync(NULL, NULL) == PKMOM_EINVAL);
    CHECK(pkmom_context_bytes(NULL) == 0);
    CHECK(strcmp(pkmom_last_error(NULL), "null context") == 0);
    if (fails) return 1;
    printf("capi ok\n");
    return 0;
}
