/* A plain C caller of the library's C ABI (include/dm.h): loads a 6x6 grid, counts the
 * embeddings of the 5-vertex path and the 4-cycle and prints "count checksum" per pattern,
 * then every embedding of the 4-cycle in canonical order. Used by tests/test_c_caller.py. */
#include <stdio.h>
#include <stdlib.h>

#include "dm.h"

static int grid_csr(int r, int c, int32_t *rp, int32_t *ci) {
    int k = 0;
    for (int v = 0; v < r * c; v++) {
        int y = v / c, x = v % c;
        rp[v] = k;
        if (y > 0) ci[k++] = v - c;
        if (x > 0) ci[k++] = v - 1;
        if (x + 1 < c) ci[k++] = v + 1;
        if (y + 1 < r) ci[k++] = v + c;
    }
    rp[r * c] = k;
    return k;
}

static int print_rows(void *user, const int32_t *rows, const float *scores, int64_t n, int32_t w) {
    (void)user;
    (void)scores;
    for (int64_t i = 0; i < n; i++) {
        for (int32_t j = 0; j < w; j++) printf(j ? " %d" : "%d", rows[i * w + j]);
        printf("\n");
    }
    return 0;
}

#define CHECK(x)                                                               \
    do {                                                                       \
        int rc_ = (x);                                                         \
        if (rc_ != DM_OK) {                                                    \
            fprintf(stderr, "%s failed: %s\n", #x, dm_strerror(rc_));          \
            return 1;                                                          \
        }                                                                      \
    } while (0)

int main(void) {
    int32_t rp[37], ci[120];
    grid_csr(6, 6, rp, ci);
    /* patterns: path 0-1-2-3-4 and cycle 0-1-2-3-0, as CSR */
    const int32_t p5_rp[6] = {0, 1, 3, 5, 7, 8}, p5_ci[8] = {1, 0, 2, 1, 3, 2, 4, 3};
    const int32_t c4_rp[5] = {0, 2, 4, 6, 8}, c4_ci[8] = {1, 3, 0, 2, 1, 3, 0, 2};
    dm_ctx *ctx = NULL;
    CHECK(dm_create(&ctx, 0, 0));
    dm_graph g;
    CHECK(dm_load_data_graph(ctx, 36, rp, ci, NULL, NULL, &g));
    dm_plan_t *p5 = NULL, *c4 = NULL;
    CHECK(dm_plan(ctx, g, 5, p5_rp, p5_ci, NULL, &p5));
    CHECK(dm_plan(ctx, g, 4, c4_rp, c4_ci, NULL, &c4));
    uint64_t n, cs;
    CHECK(dm_match(ctx, p5, DM_COUNT, NULL, NULL, &n, &cs));
    printf("%llu %llu\n", (unsigned long long)n, (unsigned long long)cs);
    CHECK(dm_match(ctx, c4, DM_COUNT, NULL, NULL, &n, &cs));
    printf("%llu %llu\n", (unsigned long long)n, (unsigned long long)cs);
    CHECK(dm_match(ctx, c4, DM_ALL, print_rows, NULL, &n, &cs));
    dm_plan_free(p5);
    dm_plan_free(c4);
    CHECK(dm_destroy(ctx));
    return 0;
}
