// Bessel-recurrence cutoff shared by the projection kernels and their adjoint.
#pragma once

#include <math.h>

namespace abcmb {

// Last l at which j_l(x) is kept: the smallest l > x whose Debye decay
// exponent nu (alpha - tanh alpha), nu = l + 1/2, cosh alpha = nu / x, exceeds
// 16 (j_l below ~e^-16 of its turning-point size).  A higher threshold keeps
// more of the tail but lets the recurrence's growing error in; 16 balances
// the two at ~1e-7 of the largest Delta_l (measured over k in [1e-5, 0.5]).  Newton on the exponent,
// whose derivative in nu is alpha; an estimate, so single precision.
__device__ __forceinline__ int bessel_cut(float x, int lmax)
{
    if (x > (float)lmax + 200.0f) return lmax;
    // the T2 and E kernels carry j_l / x^2, so at x < 1 the threshold moves
    // down by x^2
    const float T = 16.0f + 2.0f * fmaxf(0.0f, -logf(x));
    float nu = x + 1.0f + 0.8f * cbrtf(fmaxf(x, 1.0f)) * 9.0f;
    for (int it = 0; it < 8; it++) {
        float r = fmaxf(nu / fmaxf(x, 1e-30f), 1.0f + 1e-6f);
        float al = acoshf(r);
        float f = nu * (al - tanhf(al)) - T;
        nu = fmaxf(nu - f / fmaxf(al, 1e-3f), x + 0.5f);
    }
    int l = (int)ceilf(nu - 0.5f);
    return l < 2 ? 2 : (l > lmax ? lmax : l);
}

} // namespace abcmb
