// Host build of the projection kernels' Bessel cutoff (abcmb_bessel.cuh, a
// device function, compiled here with its CUDA qualifiers defined away).
#define __device__
#define __forceinline__ inline
#include "abcmb_bessel.cuh"

// out[i] = the last l the projection keeps at x[i], for lmax
extern "C" void h_bessel_cut(const float *x, int n, int lmax, int *out)
{
    for (int i = 0; i < n; i++) out[i] = abcmb::bessel_cut(x[i], lmax);
}
