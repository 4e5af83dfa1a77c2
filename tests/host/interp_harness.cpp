// Host build of the library's ln k interpolation (abcmb_interp.cuh), used by
// the projection onto the transfer grid and by the Limber lensing potential.
#include "abcmb_interp.cuh"

// out[j] = f interpolated at kt[j] from the nodes kn[0..n)
extern "C" void h_interp(const double *kn, int n, const double *f, const double *kt, int m, double *out)
{
    for (int j = 0; j < m; j++) {
        int r0;
        double w[4];
        abcmb::lnk_hermite_weights(kn, n, kt[j], &r0, w);
        double s = 0.0;
        for (int q = 0; q < 4; q++) s += w[q] * f[r0 + q];
        out[j] = s;
    }
}
