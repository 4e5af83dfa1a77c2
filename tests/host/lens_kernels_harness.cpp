// Host build of the lensing kernels (abcmb_lens_kernels.cuh) for the CPU
// tests: every CTA of lens_kernel (128 threads, one Gauss-Legendre node
// each), lens_finish and cl_psi_kernel runs as host threads under
// warp_emu.h, CTAs one after another, with the grids and arguments of
// abcmb_lens and abcmb_cl_psi.
#include "warp_emu.h"

#include "abcmb_lens_kernels.cuh"

// the kernels' dynamic shared memory (one CTA at a time)
namespace abcmb {
namespace lens {
double acc[4 * (6000 + 1)];
double sm[2 * 20000];
} // namespace lens
} // namespace abcmb

using namespace abcmb::lens;

// out [B][4][lout-1] (TT, TE, EE, BB lensed) from Cl [B][3][L-1] and Cpsi [B][L-1], as abcmb_lens
extern "C" void h_lens(int B, const double *Cl, int L, const double *Cpsi, int lout, int n_mu, double *out)
{
    const int nl = lout - 1;
    for (long i = 0; i < (long)B * 4 * nl; i++) out[i] = 0.0;
    for (int b = 0; b < B; b++)
        for (int gx = 0; gx < (n_mu + kLensThreads - 1) / kLensThreads; gx++)
            emu::run_cta((unsigned)gx, (unsigned)b, kLensThreads,
                         [&] { lens_kernel(B, Cl, Cpsi, L, lout, n_mu, out); });
    const long m = (long)B * nl;
    for (long gx = 0; gx < (m + 255) / 256; gx++)
        emu::run_cta((unsigned)gx, 0, 256, [&] { lens_finish(B, Cl, L, lout, out); });
}

// Cpsi [B][lmax-1] from the records bg [B][len] and delta_m [B][Nk][n_tau], as abcmb_cl_psi
extern "C" void h_cl_psi(int B, const double *bg, long len, const double *Dm, const double *k, int Nk, int lmax,
                         double *Cpsi)
{
    for (int b = 0; b < B; b++)
        for (int gx = 0; gx < (lmax - 1 + 127) / 128; gx++)
            emu::run_cta((unsigned)gx, (unsigned)b, 128, [&] { cl_psi_kernel(B, bg, len, Dm, k, Nk, lmax, Cpsi); });
}
