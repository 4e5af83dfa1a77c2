// Host build of the whole hot path (the CPU tests): the calls Pipeline.run
// makes -- background_kernel's builder on one warp per cosmology,
// perturb_quad_kernel, project_kernel and cl_kernel -- with their grids and
// arguments, every CTA's threads run as host threads under warp_emu.h.
#define ABCMB_HOST_WARPS
#include "warp_emu.h"

#include "abcmb_ode_quad.cuh"
#include "abcmb_spectra.cuh"
#include "abcmb_spectra_mixed.cuh"

// the kernels' dynamic shared memory (one CTA at a time)
namespace abcmb {
double qsm[quad_smem_per_warp<16>() / sizeof(double)];
double acc[2 * 5000];
double wk[1 << 16];
namespace mixed {
float acc[4 * 5000];
float wkf[1 << 16];
} // namespace mixed
} // namespace abcmb

using namespace abcmb;

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }

// C_l [B][3][lmax-1] for params [B][6] at k [Nk] (ascending), hierarchies L
// (<= 63), the FP64 path; bg [B][len], S [B][Nk][n_tau][3] and Delta
// [B][Nk][lmax-1][2] are the caller's buffers; status [B][Nk]
extern "C" void h_pipeline(int B, const double *params, const double *k, int Nk, int L, int n_tau, int lmax,
                           double rtol, double err_floor, double *bg, double *S, double *Delta, double *Cl,
                           int *status)
{
    const long len = ABCMB_BG_LEN(n_tau), M = (long)B * Nk;
    for (int b = 0; b < B; b++)
        emu::run_cta((unsigned)b, 0, 32, [&] {
            build_background(params + (long)b * ABCMB_NPARAM, bg + (long)b * len, n_tau, (int)threadIdx.x, 32);
        });
    const int P = L <= 15 ? 4 : (L <= 31 ? 8 : 16);
    for (long blk = 0; blk < (M + 7) / 8; blk++)
        emu::run_cta((unsigned)blk, 0, 32, [&] {
            if (P == 4)
                perturb_quad_kernel<4, 1>(B, Nk, bg, len, k, L, L, L, rtol, 1e-12, 2000000, 1.0, 1.0, 1.0, S, status,
                                          nullptr, 0, 0, err_floor);
            else if (P == 8)
                perturb_quad_kernel<8, 1>(B, Nk, bg, len, k, L, L, L, rtol, 1e-12, 2000000, 1.0, 1.0, 1.0, S, status,
                                          nullptr, 0, 0, err_floor);
            else
                perturb_quad_kernel<16, 1>(B, Nk, bg, len, k, L, L, L, rtol, 1e-12, 2000000, 1.0, 1.0, 1.0, S,
                                           status, nullptr, 0, 0, err_floor);
        });
    for (long blk = 0; blk < M; blk++)
        emu::run_cta((unsigned)blk, 0, 128,
                     [&] { project_kernel<false>(B, Nk, bg, len, S, k, lmax, 1.0, Delta, nullptr, 0); });
    for (int b = 0; b < B; b++)
        for (int gx = 0; gx < (lmax - 1 + 255) / 256; gx++)
            emu::run_cta((unsigned)gx, (unsigned)b, 256, [&] { cl_kernel(B, Nk, bg, len, Delta, k, lmax, Cl); });
}

// the mixed-precision end of the path on the same records and sources, as
// Pipeline(mixed=True) runs it: Delta32 [B][Nk][lmax-1][2], then C_l
extern "C" void h_mixed_tail(int B, const double *bg, const double *S, const double *k, int Nk, int n_tau, int lmax,
                             float *Delta32, double *Cl)
{
    const long len = ABCMB_BG_LEN(n_tau);
    for (long blk = 0; blk < (long)B * Nk; blk++)
        emu::run_cta((unsigned)blk, 0, 32,
                      [&] { mixed::project_mixed_kernel(B, Nk, bg, len, S, k, lmax, 1.0, Delta32); });
    for (int b = 0; b < B; b++)
        for (int gx = 0; gx < (lmax - 1 + 255) / 256; gx++)
            emu::run_cta((unsigned)gx, (unsigned)b, 256,
                         [&] { mixed::cl_mixed_kernel(B, Nk, bg, len, Delta32, k, lmax, Cl); });
}
