/*
 * CPU oracle for the longest common subsequence (LCS) -- TEST
 * INFRASTRUCTURE ONLY.  It checks future GPU paths; it is never linked into
 * the library and shares no code with it.
 *
 * The paper's section "Generalized Dynamic Programming Extensions" ("Direct
 * Extension: LCS") names the LCS length as the first problem its diagonal
 * band carries over to, and the subsequence itself as obtainable by parent
 * bookkeeping.  The plain definition (the textbook recurrence):
 *
 *   L(i,0) = L(0,j) = 0
 *   L(i,j) = L(i-1,j-1) + 1                if x_i == y_j
 *          = max(L(i-1,j), L(i,j-1))       otherwise
 *   LCS length = L(n,m)
 *
 * Symbols are int32 values (bytes, tokens, quantised levels).
 */
#include <stdint.h>
#include <stdlib.h>

static int lcs_bad(const int32_t* x, int64_t n, const int32_t* y, int64_t m)
{
    return !x || !y || n < 0 || m < 0;
}

/* The full (n+1) x (m+1) matrix in C order, in a buffer the caller frees. */
static int64_t* lcs_matrix(const int32_t* x, int64_t n, const int32_t* y, int64_t m)
{
    int64_t* L = (int64_t*)malloc((size_t)(n + 1) * (size_t)(m + 1) * sizeof(int64_t));
    if (!L) return NULL;
    const int64_t W = m + 1;
    for (int64_t j = 0; j <= m; ++j) L[j] = 0;
    for (int64_t i = 1; i <= n; ++i) {
        L[i * W] = 0;
        for (int64_t j = 1; j <= m; ++j) {
            if (x[i - 1] == y[j - 1]) {
                L[i * W + j] = L[(i - 1) * W + (j - 1)] + 1;
            } else {
                const int64_t up = L[(i - 1) * W + j], left = L[i * W + (j - 1)];
                L[i * W + j] = up >= left ? up : left;
            }
        }
    }
    return L;
}

/* LCS length by the full matrix.  0 ok, 1 bad arguments, 2 no memory. */
int oracle_lcs_length(const int32_t* x, int64_t n, const int32_t* y, int64_t m, int64_t* out)
{
    if (lcs_bad(x, n, y, m) || !out) return 1;
    int64_t* L = lcs_matrix(x, n, y, m);
    if (!L) return 2;
    *out = L[n * (m + 1) + m];
    free(L);
    return 0;
}

/* The same recurrence on two rows (O(m) memory), for sizes whose matrix
 * would not fit.  Same result as oracle_lcs_length. */
int oracle_lcs_length_rolling(const int32_t* x, int64_t n, const int32_t* y, int64_t m,
                              int64_t* out)
{
    if (lcs_bad(x, n, y, m) || !out) return 1;
    int64_t* prev = (int64_t*)calloc((size_t)(m + 1), sizeof(int64_t));
    int64_t* cur = (int64_t*)calloc((size_t)(m + 1), sizeof(int64_t));
    if (!prev || !cur) { free(prev); free(cur); return 2; }
    for (int64_t i = 1; i <= n; ++i) {
        cur[0] = 0;
        for (int64_t j = 1; j <= m; ++j) {
            if (x[i - 1] == y[j - 1]) {
                cur[j] = prev[j - 1] + 1;
            } else {
                cur[j] = prev[j] >= cur[j - 1] ? prev[j] : cur[j - 1];
            }
        }
        int64_t* t = prev;
        prev = cur;
        cur = t;
    }
    *out = prev[m];
    free(prev);
    free(cur);
    return 0;
}

/* One longest common subsequence: the full matrix, then a walk back from
 * (n,m): where x_i == y_j take the diagonal and keep the pair (i, j);
 * otherwise go up when L(i-1,j) >= L(i,j-1), else left (the textbook rule).
 * xi[k], yj[k] (0-based positions in x and y, increasing) receive the
 * pairs in forward order; both need room for min(n, m) entries; *len their
 * number (= the LCS length).  0 ok, 1 bad arguments, 2 no memory. */
int oracle_lcs_pairs(const int32_t* x, int64_t n, const int32_t* y, int64_t m, int64_t* xi,
                     int64_t* yj, int64_t* len)
{
    if (lcs_bad(x, n, y, m) || !xi || !yj || !len) return 1;
    int64_t* L = lcs_matrix(x, n, y, m);
    if (!L) return 2;
    const int64_t W = m + 1;
    int64_t i = n, j = m, k = L[n * W + m];
    *len = k;
    while (i > 0 && j > 0) {
        if (x[i - 1] == y[j - 1]) {
            --k;
            xi[k] = i - 1;
            yj[k] = j - 1;
            --i;
            --j;
        } else if (L[(i - 1) * W + j] >= L[i * W + (j - 1)]) {
            --i;
        } else {
            --j;
        }
    }
    free(L);
    return 0;
}
