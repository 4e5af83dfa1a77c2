/*
 * ORACLE (test infrastructure only; see orc.h).
 * LU factorisation with partial pivoting (textbook Doolittle form) that skips
 * exact zeros.  Each row keeps the range of its nonzero entries: the pivot
 * row's entries beyond its last nonzero are zero, so the elimination stops
 * there, and rows whose entry in the pivot column is zero are left alone
 * (subtracting l * 0, or 0 * row, leaves an entry as it is).  The solves use
 * the same ranges.  For a banded matrix this costs what a band solver costs;
 * every nonzero update is the dense algorithm's.
 *
 * ext[2n] (written by orc_lu_factor, read by orc_lu_solve): ext[i] is the
 * last nonzero column of row i of U, ext[n + i] the first column of row i's
 * multipliers (i if it has none).
 */
#include <math.h>

#include "orc.h"

int orc_lu_factor(real_t *A, int n, int *piv, int *ext)
{
    int *rend = ext, *lbeg = ext + n;
    for (int i = 0; i < n; i++) {
        int j = n - 1;
        while (j > i && A[i * n + j] == 0.0) j--;
        rend[i] = j;
        lbeg[i] = i;
    }
    for (int k = 0; k < n; k++) {
        int p = k;
        real_t best = ABS(A[k * n + k]);
        for (int i = k + 1; i < n; i++)
            if (RE(ABS(A[i * n + k])) > RE(best)) { best = ABS(A[i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k) {
            const int j0 = lbeg[k] < lbeg[p] ? lbeg[k] : lbeg[p];
            const int j1 = rend[k] > rend[p] ? rend[k] : rend[p];
            for (int j = j0; j <= j1; j++) {
                real_t t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
            int t = rend[k]; rend[k] = rend[p]; rend[p] = t;
            t = lbeg[k]; lbeg[k] = lbeg[p]; lbeg[p] = t;
        }
        const real_t inv = 1.0 / A[k * n + k];
        const int jend = rend[k];
        for (int i = k + 1; i < n; i++) {
            if (A[i * n + k] == 0.0) continue;
            const real_t l = A[i * n + k] * inv;
            A[i * n + k] = l;
            if (k < lbeg[i]) lbeg[i] = k;
            for (int j = k + 1; j <= jend; j++) A[i * n + j] -= l * A[k * n + j];
            if (jend > rend[i]) rend[i] = jend;
        }
    }
    return 0;
}

void orc_lu_solve(const real_t *A, int n, const int *piv, const int *ext, real_t *b)
{
    const int *rend = ext, *lbeg = ext + n;
    for (int k = 0; k < n; k++) {
        int p = piv[k];
        if (p != k) { real_t t = b[k]; b[k] = b[p]; b[p] = t; }
    }
    for (int i = 0; i < n; i++) {
        real_t s = b[i];
        for (int j = lbeg[i]; j < i; j++) s -= A[i * n + j] * b[j];
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
        real_t s = b[i];
        for (int j = i + 1; j <= rend[i]; j++) s -= A[i * n + j] * b[j];
        b[i] = s / A[i * n + i];
    }
}
