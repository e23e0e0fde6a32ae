"""Planted mistakes for the pin-strength tests -- TEST INFRASTRUCTURE ONLY.

A mutant is one textual patch of one oracle source file: a plausible
mistake (a dropped term, a wrong index, a missing parameter, a wrong tie
order).  ``build(dir, k)`` copies the oracle's sources, applies patch k (the
original text must occur exactly once), compiles the copy with the oracle's
own flags and returns the loaded library.  The pin tests then check that
every such library fails at least one pin, i.e. that the pins pin that part
of the definition.  The oracle sources themselves carry no planted code.
"""
import os
import shutil

import oracle

MATCH = "double match = (D[(i - 1) * W + (j - 1)] + c_ij) + c_prev;"
WALK = """        if (match == here) {
            moves[k++] = 0;
            --i;
            --j;
        } else if (delete_a == here) {
            moves[k++] = 1;
            --i;
        } else if (delete_b == here) {
            moves[k++] = 2;
            --j;
        } else {"""

# k -> (file, original text, planted text)
PATCHES = {
    # TWED value (full matrix)
    1: ("twed_oracle.c", MATCH, "double match = D[(i - 1) * W + (j - 1)] + c_ij; (void)c_prev;"),
    2: ("twed_oracle.c", "double w = nu * fabs(tm(a, i) - tm(b, j));",
        "double w = nu * fabs(tm(a, i) - tm(b, i <= b->n ? i : b->n));"),
    3: ("twed_oracle.c", "return (d + w) + lambda;", "return d + w;"),
    4: ("twed_oracle.c", "for (int64_t i = 1; i <= n; ++i) D[i * W] = INFINITY;",
        "for (int64_t i = 1; i <= n; ++i) D[i * W] = 0.0;"),
    5: ("twed_oracle.c", "double dA = del_cost(A, i, nu, lambda, p);",
        "double dA = del_cost(A, i > 1 ? i - 1 : 1, nu, lambda, p);"),
    6: ("twed_oracle.c", "return sqrt(s);", "return s;"),
    7: ("twed_oracle.c", "double w = nu * fabs(tm(a, i) - tm(b, j));",
        "double w = fabs(tm(a, i) - tm(b, j));"),
    8: ("twed_oracle.c", MATCH, "double match = (D[(i - 1) * W + (j - 1)] + c_ij) - c_prev;"),
    9: ("twed_oracle.c", MATCH,
        "double match = (D[(i - 1) * W + (j - 1)] + c_ij) + cell_cost(A, i - 1, B, j, nu, p); (void)c_prev;"),
    # TWED edit-path walk
    10: ("twed_oracle.c", WALK, WALK.replace("delete_a == here", "@@").replace("delete_b == here", "delete_a == here")
         .replace("@@", "delete_b == here").replace("moves[k++] = 1;\n            --i;", "@@")
         .replace("moves[k++] = 2;\n            --j;", "moves[k++] = 1;\n            --i;")
         .replace("@@", "moves[k++] = 2;\n            --j;")),
    11: ("twed_oracle.c", WALK, """        if (delete_a == here) {
            moves[k++] = 1;
            --i;
        } else if (match == here) {
            moves[k++] = 0;
            --i;
            --j;
        } else if (delete_b == here) {
            moves[k++] = 2;
            --j;
        } else {"""),
    12: ("twed_oracle.c", "    for (int64_t x = 0, y = k - 1; x < y; ++x, --y) {",
         "    if (0) for (int64_t x = 0, y = k - 1; x < y; ++x, --y) {"),
    # LCS
    20: ("lcs_oracle.c", "} else if (L[(i - 1) * W + j] >= L[i * W + (j - 1)]) {",
         "} else if (L[(i - 1) * W + j] > L[i * W + (j - 1)]) {"),
    21: ("lcs_oracle.c", "L[i * W + j] = L[(i - 1) * W + (j - 1)] + 1;", "L[i * W + j] = L[(i - 1) * W + j] + 1;"),
    22: ("lcs_oracle.c", "cur[j] = prev[j] >= cur[j - 1] ? prev[j] : cur[j - 1];",
         "cur[j] = prev[j - 1] >= cur[j - 1] ? prev[j - 1] : cur[j - 1];"),
    # DTW
    30: ("dtw_oracle.c",
         "const double best = fmin(fmin(D[(i - 1) * W + (j - 1)], D[(i - 1) * W + j]), D[i * W + (j - 1)]);",
         "const double best = fmin(D[(i - 1) * W + (j - 1)], D[(i - 1) * W + j]);"),
    31: ("dtw_oracle.c",
         "const double best = fmin(fmin(D[(i - 1) * W + (j - 1)], D[(i - 1) * W + j]), D[i * W + (j - 1)]);",
         "const double best = fmin(fmin(D[(i - 1) * W + (j - 1)], D[(i - 1) * W + j]), D[i * W + (j - 1)]) * 0.5;"),
    32: ("dtw_oracle.c", "if (dim == 1) return fabs(x[0] - y[0]);",
         "if (dim == 1) return (x[0] - y[0]) * (x[0] - y[0]);"),
}


def build(out_dir: str, k: int):
    """The oracle library with planted mistake k (0: unpatched copy)."""
    src_dir = os.path.join(out_dir, f"src{k}")
    os.makedirs(src_dir, exist_ok=True)
    for f in oracle.SOURCE_FILES:
        shutil.copy(os.path.join(oracle.SOURCE_DIR, f), os.path.join(src_dir, f))
    if k:
        fname, old, new = PATCHES[k]
        path = os.path.join(src_dir, fname)
        text = open(path).read()
        assert text.count(old) == 1, f"patch {k}: the original text must occur once in {fname}"
        with open(path, "w") as fh:
            fh.write(text.replace(old, new))
    return oracle.compile_library(os.path.join(out_dir, f"liboracle_m{k}.so"),
                                  [os.path.join(src_dir, f) for f in oracle.SOURCE_FILES])
