/*
 * CPU oracle for dynamic time warping (DTW) -- TEST INFRASTRUCTURE ONLY.
 * It checks future GPU paths; it is never linked into the library and
 * shares no code with it.
 *
 * DTW is the related time-warp distance the paper sets its method against
 * (section "Introduction") and the second problem, after LCS, that a
 * generic version of its diagonal band would carry.  The plain definition
 * (the textbook recurrence, no window):
 *
 *   d(x,y)  = ( sum_k |x_k - y_k|^p )^(1/p), |x - y| for dim 1
 *   D(0,0)  = 0, D(i,0) = D(0,j) = +inf
 *   D(i,j)  = d(a_i, b_j) + min(D(i-1,j-1), D(i-1,j), D(i,j-1))
 *   DTW     = D(n,m)
 *
 * Evaluation order: the norm summed over k = 0..dim-1, then the root;
 * D = d + fmin(fmin(D(i-1,j-1), D(i-1,j)), D(i,j-1)).
 * Compiled with -ffp-contract=off like the TWED oracle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static double dtw_dist(const double* x, const double* y, int dim, int p)
{
    if (dim == 1) return fabs(x[0] - y[0]);
    double s = 0.0;
    if (p == 1) {
        for (int k = 0; k < dim; ++k) s = s + fabs(x[k] - y[k]);
        return s;
    }
    if (p == 2) {
        for (int k = 0; k < dim; ++k) {
            double t = x[k] - y[k];
            s = s + t * t;
        }
        return sqrt(s);
    }
    for (int k = 0; k < dim; ++k) s = s + pow(fabs(x[k] - y[k]), (double)p);
    return pow(s, 1.0 / (double)p);
}

/* DTW by the full (n+1) x (m+1) matrix in C order.
 * 0 ok, 1 bad arguments, 2 no memory. */
int oracle_dtw(const double* a, int64_t n, const double* b, int64_t m, int dim, int p,
               double* out)
{
    if (!a || !b || !out || n < 1 || m < 1 || dim < 1 || p < 1) return 1;
    double* D = (double*)malloc((size_t)(n + 1) * (size_t)(m + 1) * sizeof(double));
    if (!D) return 2;
    const int64_t W = m + 1;
    D[0] = 0.0;
    for (int64_t j = 1; j <= m; ++j) D[j] = INFINITY;
    for (int64_t i = 1; i <= n; ++i) {
        D[i * W] = INFINITY;
        for (int64_t j = 1; j <= m; ++j) {
            const double d = dtw_dist(a + (i - 1) * dim, b + (j - 1) * dim, dim, p);
            const double best = fmin(fmin(D[(i - 1) * W + (j - 1)], D[(i - 1) * W + j]), D[i * W + (j - 1)]);
            D[i * W + j] = d + best;
        }
    }
    *out = D[n * W + m];
    free(D);
    return 0;
}
