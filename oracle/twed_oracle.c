/*
 * CPU oracle for Time Warp Edit Distance (TWED) -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, FP64 statement of what the GPU library
 * computes.  It exists to check the CUDA path; it is never linked into it and
 * shares no code, header, table or helper with it.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Definition followed (paper: section "Time Warp Edit Distance", steps 1-6,
 * and Marteau's TWED, which the paper says it implements unchanged):
 *
 *   series a_1..a_n in R^dim with times t_1..t_n; b_1..b_m with t'_1..t'_m;
 *   zero padding a_0 = b_0 = 0-vector, t_0 = t'_0 = 0 (footnotes of steps 1/2).
 *   d(x,y)   = ( sum_k |x_k - y_k|^p )^(1/p)      (lp norm, section
 *              "cuTWED Implementation Remarks"); for dim == 1 this is |x-y|.
 *   c(i,j)   = d(a_i, b_j) + nu * |t_i - t'_j|
 *   dA(i)    = d(a_i, a_{i-1}) + nu * |t_i - t_{i-1}| + lambda   (delete in a)
 *   dB(j)    = d(b_j, b_{j-1}) + nu * |t'_j - t'_{j-1}| + lambda (delete in b)
 *   D(0,0) = 0, D(i,0) = D(0,j) = +inf                         (step 3)
 *   D(i,j) = min( D(i-1,j) + dA(i),
 *                 D(i,j-1) + dB(j),
 *                 D(i-1,j-1) + c(i,j) + c(i-1,j-1) )              (step 5)
 *   TWED   = D(n,m)                                               (step 6)
 *
 * Readings of garbled or silent passages (each also listed in the design
 * notes): the interior initialisation of step 4 is read as the match cost
 * d(a_i,b_j) + d(a_{i-1},b_{j-1}) (the printed difference of step norms
 * contradicts the metric property); the match time term uses column j for b;
 * nu multiplies the time terms and lambda is added to both deletions; the
 * deletion time term is an absolute value; the root of the lp norm is taken.
 *
 * Canonical evaluation order (so that an FP64 GPU path that performs the same
 * IEEE operations in the same order is bit-identical):
 *   norm sum over k = 0..dim-1 starting from 0, then sqrt (p=2) or
 *   pow(s, 1/p) (p>2); p=1 sums |diff|; dim=1 gives |diff| for every p;
 *   c      = d + (nu * |dt|)
 *   dA     = (d + (nu * |dt|)) + lambda
 *   match  = (D(i-1,j-1) + c(i,j)) + c(i-1,j-1)
 *   result = fmin(fmin(delete_a, delete_b), match)
 * Compile with -O2 -ffp-contract=off so no FMA contraction changes rounding.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* lp distance between two points of `dim` components. */
static double oracle_dist(const double* x, const double* y, int dim, int p)
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

/* Point i (0 = the zero padding, 1..n = data) of a series. */
typedef struct {
    const double* v;  /* [n][dim] */
    const double* t;  /* [n] */
    int64_t n;
    int dim;
    const double* zero; /* dim zeros */
} series_t;

static const double* pt(const series_t* s, int64_t i) { return i == 0 ? s->zero : s->v + (i - 1) * s->dim; }
static double tm(const series_t* s, int64_t i) { return i == 0 ? 0.0 : s->t[i - 1]; }

/* c(i,j), defined for 0 <= i <= n, 0 <= j <= m with the zero padding. */
static double cell_cost(const series_t* a, int64_t i, const series_t* b, int64_t j, double nu, int p)
{
    double d = oracle_dist(pt(a, i), pt(b, j), a->dim, p);
    double w = nu * fabs(tm(a, i) - tm(b, j));
    return d + w;
}

/* Deletion cost of point i of series s (i >= 1). */
static double del_cost(const series_t* s, int64_t i, double nu, double lambda, int p)
{
    double d = oracle_dist(pt(s, i), pt(s, i - 1), s->dim, p);
    double w = nu * fabs(tm(s, i) - tm(s, i - 1));
    return (d + w) + lambda;
}

static double min3(double x, double y, double z) { return fmin(fmin(x, y), z); }

static int bad_args(const double* a, const double* ta, int64_t n, const double* b, const double* tb,
                    int64_t m, int dim, double nu, double lambda, int p)
{
    if (!a || !ta || !b || !tb) return 1;
    if (n < 1 || m < 1 || dim < 1 || p < 1) return 1;
    if (!(nu >= 0.0) || !(lambda >= 0.0) || isinf(nu) || isinf(lambda)) return 1;
    return 0;
}

/* The full (n+1) x (m+1) matrix D, filled in C order (step 5 of the serial
 * TWED), in a buffer the caller frees.  NULL on allocation failure. */
static double* twed_matrix(const series_t* A, const series_t* B, double nu, double lambda, int p)
{
    const int64_t n = A->n, m = B->n;
    double* D = (double*)malloc((size_t)(n + 1) * (size_t)(m + 1) * sizeof(double));
    if (!D) return NULL;
    const int64_t W = m + 1;
    D[0] = 0.0;
    for (int64_t j = 1; j <= m; ++j) D[j] = INFINITY;
    for (int64_t i = 1; i <= n; ++i) D[i * W] = INFINITY;
    for (int64_t i = 1; i <= n; ++i) {
        double dA = del_cost(A, i, nu, lambda, p);
        for (int64_t j = 1; j <= m; ++j) {
            double dB = del_cost(B, j, nu, lambda, p);
            double c_ij = cell_cost(A, i, B, j, nu, p);
            double c_prev = cell_cost(A, i - 1, B, j - 1, nu, p);
            double delete_a = D[(i - 1) * W + j] + dA;
            double delete_b = D[i * W + (j - 1)] + dB;
            double match = (D[(i - 1) * W + (j - 1)] + c_ij) + c_prev;
            D[i * W + j] = min3(delete_a, delete_b, match);
        }
    }
    return D;
}

/* TWED by the full matrix.
 * Returns 0 on success, 1 on invalid arguments, 2 on allocation failure. */
int oracle_twed(const double* a, const double* ta, int64_t n, const double* b, const double* tb,
                int64_t m, int dim, double nu, double lambda, int p, double* out)
{
    if (bad_args(a, ta, n, b, tb, m, dim, nu, lambda, p) || !out) return 1;
    double* zero = (double*)calloc((size_t)dim, sizeof(double));
    if (!zero) return 2;
    series_t A = {a, ta, n, dim, zero}, B = {b, tb, m, dim, zero};
    double* D = twed_matrix(&A, &B, nu, lambda, p);
    if (!D) { free(zero); return 2; }
    *out = D[n * (m + 1) + m];
    free(D);
    free(zero);
    return 0;
}

/* An optimal edit path (the alignment that the paper's introduction says a
 * TWED solver can report): the full matrix above, then a walk back from
 * (n,m) to (1,1).  At each cell the predecessor is the first of
 *   match (i-1,j-1), delete in a (i-1,j), delete in b (i,j-1)
 * whose candidate value -- recomputed with the same operations as the fill
 * -- equals D(i,j).  Every finite path starts with the forced match
 * (0,0) -> (1,1) (the border is infinite), so only the moves after it are
 * returned, in forward order: moves[k] = 0 (match), 1 (delete in a),
 * 2 (delete in b); *len receives their number (at most n + m - 2, the room
 * `moves` must have).  *out receives D(n,m), as oracle_twed.
 * Returns 0 on success, 1 on invalid arguments, 2 on allocation failure,
 * 3 if no predecessor matches (cannot happen for finite inputs). */
int oracle_twed_path(const double* a, const double* ta, int64_t n, const double* b,
                     const double* tb, int64_t m, int dim, double nu, double lambda, int p,
                     double* out, int8_t* moves, int64_t* len)
{
    if (bad_args(a, ta, n, b, tb, m, dim, nu, lambda, p) || !out || !moves || !len) return 1;
    double* zero = (double*)calloc((size_t)dim, sizeof(double));
    if (!zero) return 2;
    series_t A = {a, ta, n, dim, zero}, B = {b, tb, m, dim, zero};
    double* D = twed_matrix(&A, &B, nu, lambda, p);
    if (!D) { free(zero); return 2; }
    const int64_t W = m + 1;
    int64_t i = n, j = m, k = 0;
    int rc = 0;
    while (i > 1 || j > 1) {
        const double here = D[i * W + j];
        double match = INFINITY;
        if (i > 1 && j > 1)
            match = (D[(i - 1) * W + (j - 1)] + cell_cost(&A, i, &B, j, nu, p)) +
                    cell_cost(&A, i - 1, &B, j - 1, nu, p);
        const double delete_a = i > 1 ? D[(i - 1) * W + j] + del_cost(&A, i, nu, lambda, p) : INFINITY;
        const double delete_b = j > 1 ? D[i * W + (j - 1)] + del_cost(&B, j, nu, lambda, p) : INFINITY;
        if (match == here) {
            moves[k++] = 0;
            --i;
            --j;
        } else if (delete_a == here) {
            moves[k++] = 1;
            --i;
        } else if (delete_b == here) {
            moves[k++] = 2;
            --j;
        } else {
            rc = 3;
            break;
        }
    }
    /* the walk collected the moves backwards */
    for (int64_t x = 0, y = k - 1; x < y; ++x, --y) {
        const int8_t t = moves[x];
        moves[x] = moves[y];
        moves[y] = t;
    }
    *len = k;
    *out = D[n * W + m];
    free(D);
    free(zero);
    return rc;
}

/* The same operations in the same order, keeping only rows i-1 and i
 * (O(m) memory).  Bit-identical to oracle_twed wherever both run. */
int oracle_twed_rolling(const double* a, const double* ta, int64_t n, const double* b,
                        const double* tb, int64_t m, int dim, double nu, double lambda, int p,
                        double* out)
{
    if (bad_args(a, ta, n, b, tb, m, dim, nu, lambda, p) || !out) return 1;
    double* zero = (double*)calloc((size_t)dim, sizeof(double));
    double* prev = (double*)malloc((size_t)(m + 1) * sizeof(double));
    double* cur = (double*)malloc((size_t)(m + 1) * sizeof(double));
    if (!zero || !prev || !cur) { free(zero); free(prev); free(cur); return 2; }
    series_t A = {a, ta, n, dim, zero}, B = {b, tb, m, dim, zero};
    prev[0] = 0.0;
    for (int64_t j = 1; j <= m; ++j) prev[j] = INFINITY;
    for (int64_t i = 1; i <= n; ++i) {
        double dA = del_cost(&A, i, nu, lambda, p);
        cur[0] = INFINITY;
        for (int64_t j = 1; j <= m; ++j) {
            double dB = del_cost(&B, j, nu, lambda, p);
            double c_ij = cell_cost(&A, i, &B, j, nu, p);
            double c_prev = cell_cost(&A, i - 1, &B, j - 1, nu, p);
            double delete_a = prev[j] + dA;
            double delete_b = cur[j - 1] + dB;
            double match = (prev[j - 1] + c_ij) + c_prev;
            cur[j] = min3(delete_a, delete_b, match);
        }
        double* t = prev; prev = cur; cur = t;
    }
    *out = prev[m];
    free(prev);
    free(cur);
    free(zero);
    return 0;
}

/* Deletion costs dA(1..n) of one series into out[0..n-1] (out[0] uses the
 * zero padding, as in the paper's footnote; the DP never reads it). */
int oracle_delete_costs(const double* a, const double* ta, int64_t n, int dim, double nu,
                        double lambda, int p, double* out)
{
    if (!a || !ta || !out || n < 1 || dim < 1 || p < 1) return 1;
    double* zero = (double*)calloc((size_t)dim, sizeof(double));
    if (!zero) return 2;
    series_t A = {a, ta, n, dim, zero};
    for (int64_t i = 1; i <= n; ++i) out[i - 1] = del_cost(&A, i, nu, lambda, p);
    free(zero);
    return 0;
}

/* ---- many pairs over two packed sets, one thread per slice of pairs ----
 * Set layout: vals[sum(len)][dim], ts[sum(len)], offs[nseries+1] (int64).
 * pairs[2*k], pairs[2*k+1] index series of set A and set B. */
typedef struct {
    const double *va, *ta, *vb, *tb;
    const int64_t *oa, *ob, *pairs;
    int64_t lo, hi;
    int dim, p;
    double nu, lambda;
    double* out;
    int status;
} pairs_job_t;

static void* pairs_worker(void* arg)
{
    pairs_job_t* jb = (pairs_job_t*)arg;
    jb->status = 0;
    for (int64_t k = jb->lo; k < jb->hi; ++k) {
        int64_t x = jb->pairs[2 * k], y = jb->pairs[2 * k + 1];
        int64_t a0 = jb->oa[x], n = jb->oa[x + 1] - a0;
        int64_t b0 = jb->ob[y], m = jb->ob[y + 1] - b0;
        int rc = oracle_twed_rolling(jb->va + a0 * jb->dim, jb->ta + a0, n, jb->vb + b0 * jb->dim,
                                     jb->tb + b0, m, jb->dim, jb->nu, jb->lambda, jb->p,
                                     jb->out + k);
        if (rc) { jb->status = rc; return NULL; }
    }
    return NULL;
}

int oracle_twed_pairs(const double* va, const double* ta, const int64_t* oa, const double* vb,
                      const double* tb, const int64_t* ob, const int64_t* pairs, int64_t npairs,
                      int dim, double nu, double lambda, int p, int nthreads, double* out)
{
    if (!va || !ta || !oa || !vb || !tb || !ob || !pairs || !out || npairs < 0) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > npairs) nthreads = npairs > 0 ? (int)npairs : 1;
    pairs_job_t jobs[256];
    pthread_t th[256];
    int64_t per = (npairs + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        pairs_job_t j = {va, ta, vb, tb, oa, ob, pairs, 0, 0, dim, p, nu, lambda, out, 0};
        j.lo = (int64_t)t * per;
        j.hi = j.lo + per < npairs ? j.lo + per : npairs;
        if (j.lo > j.hi) j.lo = j.hi;
        jobs[t] = j;
    }
    if (nthreads == 1) {
        pairs_worker(&jobs[0]);
        return jobs[0].status;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, pairs_worker, &jobs[t]);
    int status = 0;
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].status) status = jobs[t].status;
    }
    return status;
}
