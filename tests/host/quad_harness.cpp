// Host build of the four-lane perturbation kernel (abcmb_ode_quad.cuh, the
// path abcmb_perturb, abcmb_matter_pk and abcmb_delta_m_nodes run for
// hierarchies up to 63) for the CPU parity tests: each one-warp CTA of
// perturb_quad_kernel, pk_quad_kernel or dm_quad_kernel runs as 32 host
// threads under warp_emu.h, CTAs one after another.  The per-CTA setup below
// is the kernels' (streaming coefficients, mode numbering, shared-memory
// split); the integration is the header's own quad_modes.
#include "warp_emu.h"

#include "abcmb_ode_quad.cuh"

using namespace abcmb;

extern "C" long h_bg_len(int n_tau) { return ABCMB_BG_LEN(n_tau); }

extern "C" void h_build_bg(const double *p, int n_tau, double *rec) { build_background(p, rec, n_tau, 0, 1); }

namespace {

struct Args {
    int B, Nk;
    const double *bg;
    long len;
    const double *k;
    int L;
    double rtol, atol;
    int max_steps;
    double efloor;
    double *S;
    int *status, *steps;
    long nb8, M8;
};

// one CTA of perturb_quad_kernel<P, 1>, lane `lane` of its warp
template <int P>
void cta_lane(const Args &a, const QCoef &qc, double *qsm, long block, int lane)
{
    const double sw[3] = {1.0, 1.0, 1.0};
    const long M = (long)a.B * a.Nk;
    if constexpr (P >= 8) {
        if (block < a.nb8) {
            constexpr int P8 = P / 2;
            constexpr int E8 = 3 * P8 + 1;
            const long mi = block * 4 + (lane >> 3);
            quad_modes<P8, false, false, 8>(mi, a.M8, a.B, a.Nk, a.bg, a.len, a.k, qc, a.rtol, a.atol, a.max_steps,
                                            sw, a.S, a.status, a.steps, qsm, qsm + (1 + kQK) * E8 * 32, a.efloor);
            return;
        }
    }
    constexpr int E = 3 * P + 1;
    const long mi = a.M8 + (block - a.nb8) * 8 + (lane >> 2);
    quad_modes<P>(mi, M, a.B, a.Nk, a.bg, a.len, a.k, qc, a.rtol, a.atol, a.max_steps, sw, a.S, a.status, a.steps,
                  qsm, qsm + (1 + kQK) * E * 32, a.efloor);
}

// one CTA of pk_quad_kernel<P> (form 1: P(k) at x_out into out[B][Nk]) or
// dm_quad_kernel<P> (form 2: delta_m at the nodes into out[B][Nk][n_tau])
template <int P>
void cta_lane_form(const Args &a, const QCoef &qc, double *qsm, long block, int lane, int form, double x_out,
                   double *out)
{
    constexpr int E = 3 * P + 1;
    const long M = (long)a.B * a.Nk;
    const long mi = block * 8 + (lane >> 2);
    if (form == 1) {
        const double sw[3] = {0.0, 0.0, 0.0};
        quad_modes<P, true>(mi, M, a.B, a.Nk, a.bg, a.len, a.k, qc, a.rtol, a.atol, a.max_steps, sw, nullptr,
                            a.status, a.steps, qsm, qsm + (1 + kQK) * E * 32, a.efloor, x_out, out);
    } else {
        const double sw[3] = {1.0, 1.0, 1.0};
        quad_modes<P, false, true>(mi, M, a.B, a.Nk, a.bg, a.len, a.k, qc, a.rtol, a.atol, a.max_steps, sw, out,
                                   a.status, nullptr, qsm, qsm + (1 + kQK) * E * 32, a.efloor);
    }
}

// form 0: perturb_quad_kernel, 1: pk_quad_kernel, 2: dm_quad_kernel
template <int P>
void run(const Args &a, int form = 0, double x_out = 0.0, double *out = nullptr)
{
    std::vector<double> qsm(quad_smem_per_warp<P>() / sizeof(double));
    double cS[3 * 64], cB[3 * 64];
    const int Ls[3] = {a.L, a.L, a.L};
    blockDim.x = 1; // one thread fills the coefficient tables
    threadIdx.x = 0;
    fill_coef(cS, cB, Ls);
    QCoef qc;
    qc.S = cS;
    qc.Bc = cB;
    for (int c = 0; c < 3; c++) {
        qc.L[c] = a.L;
        qc.L1[c] = a.L + 1.0;
    }
    const long M = (long)a.B * a.Nk;
    const long blocks = a.nb8 + (M - a.M8 + 7) / 8;
    for (long blk = 0; blk < blocks; blk++)
        emu::run_cta((unsigned)blk, 0, 32, [&] {
            const int l = (int)threadIdx.x;
            if (form == 0) cta_lane<P>(a, qc, qsm.data(), blk, l);
            else cta_lane_form<P>(a, qc, qsm.data(), blk, l, form, x_out, out);
        });
}

Args args_of(int B, const double *bg, const double *k, int Nk, int L, double rtol, double atol, int max_steps,
             double efloor, int *status, int *steps)
{
    return Args{B, Nk, bg, (long)ABCMB_BG_LEN((long)bg[ABCMB_S_NTAU]), k, L, rtol, atol, max_steps, efloor,
                nullptr, status, steps, 0, 0};
}

} // namespace

// P(k, z) [B][Nk] (Mpc^3) at ln a = -ln(1 + z), as abcmb_matter_pk (L <= 63)
extern "C" void h_quad_pk(int B, const double *bg, const double *k, int Nk, int L, double rtol, double atol,
                          int max_steps, double efloor, double z, double *Pk, int *status, int *steps)
{
    const Args a = args_of(B, bg, k, Nk, L, rtol, atol, max_steps, efloor, status, steps);
    const double x_out = -log1p(z);
    if (L <= 15) run<4>(a, 1, x_out, Pk);
    else if (L <= 31) run<8>(a, 1, x_out, Pk);
    else run<16>(a, 1, x_out, Pk);
}

// delta_m [B][Nk][n_tau] at the tau nodes, as abcmb_delta_m_nodes (L <= 63)
extern "C" void h_quad_dm(int B, const double *bg, const double *k, int Nk, int L, double rtol, double atol,
                          int max_steps, double efloor, double *Dm, int *status)
{
    const Args a = args_of(B, bg, k, Nk, L, rtol, atol, max_steps, efloor, status, nullptr);
    if (L <= 15) run<4>(a, 2, 0.0, Dm);
    else if (L <= 31) run<8>(a, 2, 0.0, Dm);
    else run<16>(a, 2, 0.0, Dm);
}

// S[B][Nk][n_tau][3], status[B][Nk], steps[B][Nk][2] of the B x Nk modes, all
// three hierarchies truncated at L (<= 63), the n_wide highest k on eight lanes
extern "C" void h_quad(int B, const double *bg, const double *k, int Nk, int L, double rtol, double atol,
                       int max_steps, double efloor, int n_wide, double *S, int *status, int *steps)
{
    Args a = args_of(B, bg, k, Nk, L, rtol, atol, max_steps, efloor, status, steps);
    a.S = S;
    const int P = L <= 15 ? 4 : (L <= 31 ? 8 : 16);
    const long kw = P >= 8 ? (n_wide > Nk ? Nk : n_wide) : 0;
    a.M8 = (long)B * kw;
    a.nb8 = (a.M8 + 3) / 4;
    if (P == 4) run<4>(a);
    else if (P == 8) run<8>(a);
    else run<16>(a);
}
