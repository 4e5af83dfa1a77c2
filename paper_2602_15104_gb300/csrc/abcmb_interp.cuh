// Interpolation in ln k shared by the projection onto other k grids and the
// lensing potential (host+device): piecewise cubic Hermite with three-point
// slopes (centred, one-sided at the ends), exact for quadratics in ln k.
#pragma once

#include <math.h>

#ifndef ABCMB_HD
#ifdef __CUDACC__
#define ABCMB_HD __host__ __device__ inline
#else
#define ABCMB_HD inline
#endif
#endif

namespace abcmb {

// f(kk) = sum_m w[m] f(kn[r0 + m]), m < 4, for nodes kn[0..n), n >= 4 ascending;
// outside the nodes the end intervals' cubics extend
ABCMB_HD void lnk_hermite_weights(const double *kn, int n, double kk, int *r0_out, double w[4])
{
    const double xv = log(kk);
    int lo = 0, hi = n - 1; // interval i: kn[i] <= kk < kn[i + 1], clamped to [0, n - 2]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (kn[mid] <= kk) lo = mid; else hi = mid;
    }
    const int i = lo;
    const int r0 = i - 1 < 0 ? 0 : (i - 1 > n - 4 ? n - 4 : i - 1);
    for (int m = 0; m < 4; m++) w[m] = 0.0;
    const double xi = log(kn[i]), xj = log(kn[i + 1]), h = xj - xi, t = (xv - xi) / h;
    const double h00 = (1.0 + 2.0 * t) * (1.0 - t) * (1.0 - t), h10 = t * (1.0 - t) * (1.0 - t);
    const double h01 = t * t * (3.0 - 2.0 * t), h11 = t * t * (t - 1.0);
    w[i - r0] += h00;
    w[i + 1 - r0] += h01;
    for (int side = 0; side < 2; side++) {
        const int p = i + side;
        const double c = (side == 0 ? h10 : h11) * h;
        const int a = p == 0 ? 0 : (p == n - 1 ? n - 3 : p - 1);
        const double xa = log(kn[a]), xb = log(kn[a + 1]), xc = log(kn[a + 2]), xp = log(kn[p]);
        w[a - r0] += c * ((xp - xb) + (xp - xc)) / ((xa - xb) * (xa - xc));
        w[a + 1 - r0] += c * ((xp - xa) + (xp - xc)) / ((xb - xa) * (xb - xc));
        w[a + 2 - r0] += c * ((xp - xa) + (xp - xb)) / ((xc - xa) * (xc - xb));
    }
    *r0_out = r0;
}

} // namespace abcmb
