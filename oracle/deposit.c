/*
 * FP64 B-spline mass assignment for the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: built and called by oracle/estimator.py for the
 * tests, the smoke check and the CPU-baseline leg of the benchmark. The GPU
 * library does not link or call it.
 *
 * What it computes (paper Sec. 2.1, Eq. rawFFTed, sampled on the grid): for each
 * field f and grid node n (periodic, ng^3 nodes),
 *
 *     G_f(n) = sum_j q_{j,f} * B_m(u_{j,0} - n_0) B_m(u_{j,1} - n_1) B_m(u_{j,2} - n_2)
 *
 * with u the particle position in grid units and B_m the centred B-spline of
 * order m (support [-m/2, m/2]). The orthonormalising factor that turns B_m into
 * the Battle-Lemarie function is applied in Fourier space by the caller (it is a
 * periodic multiplier per axis; see oracle/estimator.py).
 *
 * B_m is evaluated with the truncated-power formula, one plain loop per axis,
 * one plain triple loop per particle. No blocking, no threads.
 */
#include <math.h>
#include <stdint.h>

static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

/* Centred B-spline of order m at x. B_1 is the half-open box [-1/2, 1/2). */
static double bspline(double x, int m)
{
    if (m == 1) return (x >= -0.5 && x < 0.5) ? 1.0 : 0.0;
    if (fabs(x) >= 0.5 * m) return 0.0;
    double s = 0.0, fact = 1.0;
    for (int i = 2; i < m; ++i) fact *= (double)i;
    for (int k = 0; k <= m; ++k) {
        double t = x + 0.5 * m - k;
        if (t > 0.0) {
            double p = 1.0;
            for (int e = 0; e < m - 1; ++e) p *= t;
            s += ((k & 1) ? -1.0 : 1.0) * binom(m, k) * p;
        }
    }
    return s / fact;
}

static int64_t wrap(int64_t i, int64_t n)
{
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

/*
 * u:      [n][3] particle positions in grid units (any real value; wrapped).
 * q:      [n][nf] per-particle field values.
 * grids:  [nf][ng][ng][ng] output, C order, accumulated into (caller zeroes).
 */
void oracle_deposit_bspline(int64_t n, const double *u, int nf, const double *q,
                            int m, int64_t ng, double *grids)
{
    const int64_t cells = ng * ng * ng;
    int64_t node[3][16];
    double w[3][16];
    int cnt[3];
    for (int64_t j = 0; j < n; ++j) {
        for (int a = 0; a < 3; ++a) {
            /* every node within half a support of the particle */
            double x = u[3 * j + a];
            int64_t lo = (int64_t)ceil(x - 0.5 * m);
            int64_t hi = (int64_t)floor(x + 0.5 * m);
            cnt[a] = 0;
            for (int64_t i = lo; i <= hi && cnt[a] < 16; ++i) {
                double wt = bspline(x - (double)i, m);
                if (wt != 0.0) {
                    node[a][cnt[a]] = wrap(i, ng);
                    w[a][cnt[a]] = wt;
                    cnt[a]++;
                }
            }
        }
        for (int i0 = 0; i0 < cnt[0]; ++i0)
            for (int i1 = 0; i1 < cnt[1]; ++i1)
                for (int i2 = 0; i2 < cnt[2]; ++i2) {
                    double wt = w[0][i0] * w[1][i1] * w[2][i2];
                    int64_t c = (node[0][i0] * ng + node[1][i1]) * ng + node[2][i2];
                    for (int f = 0; f < nf; ++f) grids[f * cells + c] += q[(int64_t)nf * j + f] * wt;
                }
    }
}
