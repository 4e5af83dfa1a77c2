// Host build of the projection and k-quadrature kernels and of their
// adjoints (abcmb_spectra.cuh, abcmb_grad.cuh) for the CPU tests: every CTA
// runs as host threads under warp_emu.h, CTAs one after another, with the
// grids and arguments of abcmb_project, abcmb_cl, abcmb_project_adjoint and
// abcmb_cl_adjoint.
#define ABCMB_HOST_WARPS
#include "warp_emu.h"

#include "abcmb_grad.cuh"
#include "abcmb_spectra.cuh"

// the kernels' dynamic shared memory (one CTA at a time)
namespace abcmb {
double acc[2 * 5000];
double wk[1 << 16];
namespace adj {
double wk[1 << 17];
double db[2 * 5000];
} // namespace adj
} // namespace abcmb

using namespace abcmb;

namespace {
long rec_len(const double *bg) { return ABCMB_BG_LEN((long)bg[ABCMB_S_NTAU]); }
} // namespace

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }

extern "C" void h_build_bg(const double *p, int n_tau, double *rec)
{
    emu::run_cta(0, 0, 32, [&] { build_background(p, rec, n_tau, (int)threadIdx.x, 32); });
}

// Delta[B][Nk][lmax-1][2], as abcmb_project
extern "C" void h_project(int B, const double *bg, const double *S, const double *k, int Nk, int lmax,
                          double scale_pol, double *Delta)
{
    const long len = rec_len(bg);
    for (long blk = 0; blk < (long)B * Nk; blk++)
        emu::run_cta((unsigned)blk, 0, 128,
                     [&] { project_kernel<false>(B, Nk, bg, len, S, k, lmax, scale_pol, Delta, nullptr, 0); });
}

// Cl[B][3][lmax-1], as abcmb_cl
extern "C" void h_cl(int B, const double *bg, const double *Delta, const double *k, int Nk, int lmax, double *Cl)
{
    const long len = rec_len(bg);
    for (int b = 0; b < B; b++)
        for (int gx = 0; gx < (lmax - 1 + 255) / 256; gx++)
            emu::run_cta((unsigned)gx, (unsigned)b, 256, [&] { cl_kernel(B, Nk, bg, len, Delta, k, lmax, Cl); });
}

// Sbar [B][Nk][n_tau][3] and recbar += the node and tau_0 adjoints, as abcmb_project_adjoint
extern "C" void h_project_adjoint(int B, const double *bg, const double *S, const double *k, int Nk, int lmax,
                                  double scale_pol, const double *Deltabar, double *Sbar, double *recbar)
{
    const long len = rec_len(bg);
    for (long blk = 0; blk < (long)B * Nk; blk++)
        emu::run_cta((unsigned)blk, 0, 128, [&] {
            adj::project_adjoint_kernel(B, Nk, bg, len, S, k, lmax, scale_pol, Deltabar, Sbar, recbar);
        });
}

// Deltabar [B][Nk][lmax-1][2] and recbar += the A_s, n_s adjoints, as abcmb_cl_adjoint
extern "C" void h_cl_adjoint(int B, const double *bg, const double *Delta, const double *k, int Nk, int lmax,
                             const double *Clbar, double *Deltabar, double *recbar)
{
    const long len = rec_len(bg);
    for (int b = 0; b < B; b++)
        for (int gx = 0; gx < (lmax - 1 + 255) / 256; gx++)
            emu::run_cta((unsigned)gx, (unsigned)b, 256, [&] {
                adj::cl_adjoint_kernel(B, Nk, bg, len, Delta, k, lmax, Clbar, Deltabar, recbar);
            });
}

// The gradient's ODE pass over B x Nk modes (taped_kernel, two one-warp modes
// per CTA), into the workspace ws laid out by grad_layout: with plan == NULL
// the counting pass of abcmb_grad_count_steps (accepted[b][k] written, no
// tape), else the recording pass of abcmb_perturb_taped with that plan (as
// abcmb_grad_plan writes it), which is first copied into ws as the C ABI does.
extern "C" void h_taped(int B, const double *bg, const double *k, int Nk, int L, double rtol, double atol,
                        int max_steps, double *S, int *status, char *ws, const long long *plan, int *accepted)
{
    const long len = rec_len(bg), M = (long)B * Nk;
    long tape = 0, ck = 0;
    int record = 0;
    if (plan) {
        tape = (long)plan[M];
        ck = (long)plan[2 * M + 1];
        const adj::GradLayout g = adj::grad_layout(B, Nk, ode_dims(L, L, L), tape, ck);
        std::memcpy(ws + g.plan, plan, (size_t)(2 * M + 2) * sizeof(long long));
        record = 1;
    }
    const long blocks = (M * 32 + adj::kGradThreads - 1) / adj::kGradThreads;
    for (long blk = 0; blk < blocks; blk++)
        emu::run_cta((unsigned)blk, 0, adj::kGradThreads, [&] {
            adj::taped_kernel(B, Nk, bg, len, k, L, L, L, rtol, atol, max_steps, 1.0, 1.0, 1.0, S, status, ws, tape,
                              ck, record, plan ? nullptr : accepted);
        });
}

// The reverse sweep over every mode (adjoint_kernel), after h_taped with the
// same plan: recbar[b] += the adjoint of cosmology b's record
extern "C" void h_adjoint(int B, const double *bg, const double *k, int Nk, int L, const double *Sbar, char *ws,
                          const long long *plan, double *recbar)
{
    const long len = rec_len(bg), M = (long)B * Nk;
    const long blocks = (M * 32 + adj::kGradThreads - 1) / adj::kGradThreads;
    for (long blk = 0; blk < blocks; blk++)
        emu::run_cta((unsigned)blk, 0, adj::kGradThreads, [&] {
            adj::adjoint_kernel(B, Nk, bg, len, k, L, L, L, 1.0, 1.0, 1.0, Sbar, ws, recbar, (long)plan[M],
                                (long)plan[2 * M + 1]);
        });
}

// abcmb_perturb's path for a massive neutrino: the forward alone over B x Nk
// modes (plain_kernel, two one-warp modes per CTA, V_COUNT x N doubles of
// work per mode)
extern "C" void h_plain(int B, const double *bg, const double *k, int Nk, int L, int Lm, double rtol, double atol,
                        int max_steps, double *S, int *status, int *steps, double *work)
{
    const long len = rec_len(bg), M = (long)B * Nk;
    const long blocks = (M * 32 + adj::kGradThreads - 1) / adj::kGradThreads;
    for (long blk = 0; blk < blocks; blk++)
        emu::run_cta((unsigned)blk, 0, adj::kGradThreads, [&] {
            adj::plain_kernel(B, Nk, bg, len, k, L, L, L, Lm, rtol, atol, max_steps, 1.0, 1.0, 1.0, S, status, steps,
                              work);
        });
}

// grad [B][6] from the record adjoint and the records at params -+ h e_j, as abcmb_record_vjp
extern "C" void h_record_vjp(int B, long len, const double *recbar, const double *rp, const double *rm,
                             const double *h, double *grad)
{
    for (int b = 0; b < B; b++)
        for (int j = 0; j < ABCMB_NPARAM; j++)
            emu::run_cta((unsigned)b, (unsigned)j, 256,
                         [&] { adj::record_vjp_kernel(B, len, recbar, rp, rm, h, grad); });
}

// bytes of the gradient workspace grad_layout lays out (tape = ck = 0: the counting pass)
extern "C" size_t h_grad_layout_bytes(int B, int Nk, int L, long tape, long ck)
{
    return adj::grad_layout(B, Nk, ode_dims(L, L, L), tape, ck).total;
}

// the tape plan from the counted steps, as abcmb_grad_plan makes it -> workspace bytes
extern "C" size_t h_make_plan(int B, int Nk, int L, const int *accepted, long long *plan)
{
    return adj::make_plan(B, Nk, ode_dims(L, L, L), accepted, plan);
}
