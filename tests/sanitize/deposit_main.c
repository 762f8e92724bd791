/* Runs the oracle's C deposit (oracle/deposit.c) on edge cases under AddressSanitizer
 * and UndefinedBehaviorSanitizer (built by tests/test_host_sanitizers.py): positions at
 * 0, just below L, at L, negative and far outside the box, every B-spline order 1-5 and
 * four fields; checks that every field's total equals the sum of its values (each
 * B-spline's weights sum to 1). Exit status 0 on success. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

void oracle_deposit_bspline(int64_t n, const double *u, int nf, const double *q, int m, int64_t ng, double *grids);

int main(void)
{
    const int64_t ng = 8;
    const double u[] = {0.0, 0.0, 0.0,    7.999999, 7.5, 0.25,   8.0, 8.0, 8.0,   -0.5, -3.25, 11.75,
                        1.0e6, -1.0e6, 3.5, 4.5, 4.5, 4.5,     0.5, 1.5, 2.5};
    const int64_t n = sizeof u / sizeof u[0] / 3;
    const int nf = 4;
    double *q = malloc(sizeof(double) * n * nf);
    for (int64_t j = 0; j < n; ++j)
        for (int f = 0; f < nf; ++f) q[j * nf + f] = (f == 0) ? 1.0 : (double)(j + 1) * (f + 1) * 0.5;
    double *grids = calloc((size_t)(nf * ng * ng * ng), sizeof(double));
    for (int m = 1; m <= 5; ++m) {
        for (int64_t i = 0; i < nf * ng * ng * ng; ++i) grids[i] = 0.0;
        oracle_deposit_bspline(n, u, nf, q, m, ng, grids);
        for (int f = 0; f < nf; ++f) {
            double tot = 0.0, want = 0.0;
            for (int64_t i = 0; i < ng * ng * ng; ++i) tot += grids[f * ng * ng * ng + i];
            for (int64_t j = 0; j < n; ++j) want += q[j * nf + f];
            if (fabs(tot - want) > 1e-9 * fabs(want)) {
                fprintf(stderr, "order %d field %d: total %.15g, expected %.15g\n", m, f, tot, want);
                return 1;
            }
        }
    }
    free(q);
    free(grids);
    printf("deposit ok\n");
    return 0;
}
