// Host build of the mixed-precision projection and k-quadrature kernels
// (abcmb_spectra_mixed.cuh) for the CPU tests: every CTA of
// project_mixed_kernel (one warp) and cl_mixed_kernel (256 threads) runs as
// host threads under warp_emu.h, CTAs one after another, with the grids and
// arguments of abcmb_project_mixed and abcmb_cl_mixed.  Compiled without
// floating-point contraction, so every FP32 operation rounds once, as the
// kernels' error-free transformations require.
#include "warp_emu.h"

#include "abcmb_spectra_mixed.cuh"

// the kernels' dynamic shared memory (one CTA at a time)
namespace abcmb {
namespace mixed {
float acc[4 * 5000];
float wkf[1 << 16];
} // namespace mixed
} // namespace abcmb

using namespace abcmb;

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }

extern "C" void h_build_bg(const double *p, int n_tau, double *rec) { build_background(p, rec, n_tau, 0, 1); }

// Delta32[B][Nk][lmax-1][2] from S[B][Nk][n_tau][3], as abcmb_project_mixed
extern "C" void h_project_mixed(int B, const double *bg, const double *S, const double *k, int Nk, int lmax,
                                double scale_pol, float *Delta)
{
    const long len = ABCMB_BG_LEN((long)bg[ABCMB_S_NTAU]);
    for (long blk = 0; blk < (long)B * Nk; blk++)
        emu::run_cta((unsigned)blk, 0, 32,
                     [&] { mixed::project_mixed_kernel(B, Nk, bg, len, S, k, lmax, scale_pol, Delta); });
}

// Cl[B][3][lmax-1] from Delta32, as abcmb_cl_mixed
extern "C" void h_cl_mixed(int B, const double *bg, const float *Delta, const double *k, int Nk, int lmax,
                           double *Cl)
{
    const long len = ABCMB_BG_LEN((long)bg[ABCMB_S_NTAU]);
    const int nl = lmax - 1;
    for (int b = 0; b < B; b++)
        for (int gx = 0; gx < (nl + 255) / 256; gx++)
            emu::run_cta((unsigned)gx, (unsigned)b, 256,
                         [&] { mixed::cl_mixed_kernel(B, Nk, bg, len, Delta, k, lmax, Cl); });
}
