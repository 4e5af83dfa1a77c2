// Host build of the four-lane perturbation kernels (abcmb_ode_quad.cuh, the
// path abcmb_perturb, abcmb_matter_pk and abcmb_delta_m_nodes run for
// hierarchies up to 63) for the CPU parity tests: every one-warp CTA of
// perturb_quad_kernel, pk_quad_kernel or dm_quad_kernel runs as 32 host
// threads under warp_emu.h, CTAs one after another, with the grids and
// arguments of the library's launches.
#include "warp_emu.h"

#include "abcmb_ode_quad.cuh"

using namespace abcmb;

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }

extern "C" void h_build_bg(const double *p, int n_tau, double *rec) { build_background(p, rec, n_tau, 0, 1); }

// the kernels' dynamic shared memory (one CTA at a time), sized for P = 16
namespace abcmb {
double qsm[quad_smem_per_warp<16>() / sizeof(double)];
} // namespace abcmb

namespace {

long rec_len(const double *bg) { return ABCMB_BG_LEN((long)bg[ABCMB_S_NTAU]); }

int p_of(int L) { return L <= 15 ? 4 : (L <= 31 ? 8 : 16); }

} // namespace

// P(k, z) [B][Nk] (Mpc^3) at ln a = -ln(1 + z), as abcmb_matter_pk (L <= 63)
extern "C" void h_quad_pk(int B, const double *bg, const double *k, int Nk, int L, double rtol, double atol,
                          int max_steps, double efloor, double z, double *Pk, int *status, int *steps)
{
    const long len = rec_len(bg), blocks = ((long)B * Nk + 7) / 8;
    const double x_out = -log1p(z);
    const int P = p_of(L);
    for (long blk = 0; blk < blocks; blk++)
        emu::run_cta((unsigned)blk, 0, 32, [&] {
            if (P == 4) pk_quad_kernel<4>(B, Nk, bg, len, k, L, L, L, rtol, atol, max_steps, x_out, Pk, status, steps, efloor);
            else if (P == 8) pk_quad_kernel<8>(B, Nk, bg, len, k, L, L, L, rtol, atol, max_steps, x_out, Pk, status, steps, efloor);
            else pk_quad_kernel<16>(B, Nk, bg, len, k, L, L, L, rtol, atol, max_steps, x_out, Pk, status, steps, efloor);
        });
}

// delta_m [B][Nk][n_tau] at the tau nodes, as abcmb_delta_m_nodes (L <= 63)
extern "C" void h_quad_dm(int B, const double *bg, const double *k, int Nk, int L, double rtol, double atol,
                          int max_steps, double efloor, double *Dm, int *status)
{
    const long len = rec_len(bg), blocks = ((long)B * Nk + 7) / 8;
    const int P = p_of(L);
    for (long blk = 0; blk < blocks; blk++)
        emu::run_cta((unsigned)blk, 0, 32, [&] {
            if (P == 4) dm_quad_kernel<4>(B, Nk, bg, len, k, L, L, L, rtol, atol, max_steps, Dm, status, efloor);
            else if (P == 8) dm_quad_kernel<8>(B, Nk, bg, len, k, L, L, L, rtol, atol, max_steps, Dm, status, efloor);
            else dm_quad_kernel<16>(B, Nk, bg, len, k, L, L, L, rtol, atol, max_steps, Dm, status, efloor);
        });
}

// S[B][Nk][n_tau][3], status[B][Nk], steps[B][Nk][2] of the B x Nk modes, all
// three hierarchies truncated at L (<= 63), the n_wide highest k on eight
// lanes: the grid and arguments of abcmb_perturb's launch (one warp per CTA)
extern "C" void h_quad(int B, const double *bg, const double *k, int Nk, int L, double rtol, double atol,
                       int max_steps, double efloor, int n_wide, double *S, int *status, int *steps)
{
    const long len = rec_len(bg), M = (long)B * Nk;
    const int P = p_of(L);
    const long kw = P >= 8 ? (n_wide > Nk ? Nk : n_wide) : 0;
    const long M8 = (long)B * kw, nb8 = (M8 + 3) / 4, blocks = nb8 + (M - M8 + 7) / 8;
    for (long blk = 0; blk < blocks; blk++)
        emu::run_cta((unsigned)blk, 0, 32, [&] {
            if (P == 4)
                perturb_quad_kernel<4, 1>(B, Nk, bg, len, k, L, L, L, rtol, atol, max_steps, 1.0, 1.0, 1.0, S, status,
                                          steps, (int)nb8, M8, efloor);
            else if (P == 8)
                perturb_quad_kernel<8, 1>(B, Nk, bg, len, k, L, L, L, rtol, atol, max_steps, 1.0, 1.0, 1.0, S, status,
                                          steps, (int)nb8, M8, efloor);
            else
                perturb_quad_kernel<16, 1>(B, Nk, bg, len, k, L, L, L, rtol, atol, max_steps, 1.0, 1.0, 1.0, S,
                                           status, steps, (int)nb8, M8, efloor);
        });
}
