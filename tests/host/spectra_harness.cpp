// Host build of the line-of-sight projection and k-quadrature kernels
// (abcmb_spectra.cuh) for the CPU parity tests: every CTA of project_kernel
// (128 threads) and cl_kernel (256) runs as host threads under warp_emu.h,
// CTAs one after another, with the grids and arguments of abcmb_project,
// abcmb_project_interp and abcmb_cl.
#include "warp_emu.h"

#include "abcmb_spectra.cuh"

// the kernels' dynamic shared memory (one CTA at a time)
namespace abcmb {
double acc[2 * 5000];
double wk[1 << 16];
} // namespace abcmb

using namespace abcmb;

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }

extern "C" void h_build_bg(const double *p, int n_tau, double *rec) { build_background(p, rec, n_tau, 0, 1); }

// Delta[B][Nk][lmax-1][2] from S[B][Nk][n_tau][3] at k[Nk], as abcmb_project
extern "C" void h_project(int B, const double *bg, const double *S, const double *k, int Nk, int lmax,
                          double scale_pol, double *Delta)
{
    const long len = ABCMB_BG_LEN((long)bg[ABCMB_S_NTAU]);
    for (long blk = 0; blk < (long)B * Nk; blk++)
        emu::run_cta((unsigned)blk, 0, 128,
                     [&] { project_kernel<false>(B, Nk, bg, len, S, k, lmax, scale_pol, Delta, nullptr, 0); });
}

// Delta[B][Nkt][lmax-1][2] at kt from S given at the ODE nodes k[Nk], as abcmb_project_interp
extern "C" void h_project_interp(int B, const double *bg, const double *S, const double *k, int Nk,
                                 const double *kt, int Nkt, int lmax, double scale_pol, double *Delta)
{
    const long len = ABCMB_BG_LEN((long)bg[ABCMB_S_NTAU]);
    for (long blk = 0; blk < (long)B * Nkt; blk++)
        emu::run_cta((unsigned)blk, 0, 128,
                     [&] { project_kernel<true>(B, Nkt, bg, len, S, kt, lmax, scale_pol, Delta, k, Nk); });
}

// Cl[B][3][lmax-1] from Delta, as abcmb_cl
extern "C" void h_cl(int B, const double *bg, const double *Delta, const double *k, int Nk, int lmax, double *Cl)
{
    const long len = ABCMB_BG_LEN((long)bg[ABCMB_S_NTAU]);
    const int nl = lmax - 1;
    for (int b = 0; b < B; b++)
        for (int gx = 0; gx < (nl + 255) / 256; gx++)
            emu::run_cta((unsigned)gx, (unsigned)b, 256, [&] { cl_kernel(B, Nk, bg, len, Delta, k, lmax, Cl); });
}
