/*
 * ORACLE (test infrastructure only; see orc.h).
 * Dense LU factorisation with partial pivoting (textbook Doolittle form).
 * The elimination skips exact zeros: rows whose multiplier is zero, and the
 * pivot row's trailing zero columns (subtracting l * 0 leaves an entry as it
 * is).  The collocation systems of the perturbation ODE are sparse, so this
 * removes most of the work without changing any nonzero update.
 */
#include <math.h>

#include "orc.h"

int orc_lu_factor(double *A, int n, int *piv)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int i = k + 1; i < n; i++)
            if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k)
            for (int j = 0; j < n; j++) {
                double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
        double inv = 1.0 / A[k * n + k];
        int jend = n - 1; /* last nonzero column of the pivot row */
        while (jend > k && A[k * n + jend] == 0.0) jend--;
        for (int i = k + 1; i < n; i++) {
            double l = A[i * n + k] * inv;
            A[i * n + k] = l;
            if (l != 0.0)
                for (int j = k + 1; j <= jend; j++) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return 0;
}

void orc_lu_solve(const double *A, int n, const int *piv, double *b)
{
    for (int k = 0; k < n; k++) {
        int p = piv[k];
        if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int j = 0; j < i; j++) s -= A[i * n + j] * b[j];
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = b[i];
        for (int j = i + 1; j < n; j++) s -= A[i * n + j] * b[j];
        b[i] = s / A[i * n + i];
    }
}
