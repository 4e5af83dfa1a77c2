// C ABI of the gradient (kernels in abcmb_grad.cuh).
#include <cuda_runtime.h>

#include "abcmb_grad.cuh"
#include "abcmb_launch.cuh"

namespace abcmb {
size_t perturb_warp_bytes(int B, int Nk, const abcmb_options *o)
{
    const OdeDims d = ode_dims(o->lmax_g, o->lmax_pol, o->lmax_nu, o->lmax_ncdm);
    return (size_t)B * Nk * adj::V_COUNT * d.N * sizeof(double);
}

// abcmb_perturb's path for a massive neutrino (arguments validated by the caller)
int launch_perturb_warp(int B, const double *bg, const double *k, int Nk, const abcmb_options *o, double *S,
                        int *mode_status, int *steps, double *work, cudaStream_t s)
{
    const long len = (long)ABCMB_BG_LEN(o->n_tau), M = (long)B * Nk;
    const long blocks = (M * 32 + adj::kGradThreads - 1) / adj::kGradThreads;
    if (blocks > 2147483647L) return ABCMB_E_INVALID_ARG;
    adj::plain_kernel<<<(unsigned)blocks, adj::kGradThreads, 0, s>>>(
        B, Nk, bg, len, k, o->lmax_g, o->lmax_pol, o->lmax_nu, o->lmax_ncdm, o->rtol, o->atol, o->max_steps,
        o->scale_sw, o->scale_isw, o->scale_dop, S, mode_status, steps, work);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}
} // namespace abcmb

// ---------------------------------------------------------------- C ABI
extern "C" size_t abcmb_bg_doubles(const abcmb_options *o);
extern "C" int abcmb_validate_options(const abcmb_options *o);

extern "C" size_t abcmb_grad_workspace_bytes(int B, int Nk, const abcmb_options *o)
{
    if (B < 1 || Nk < 1 || abcmb_validate_options(o) != ABCMB_OK) return 0;
    const abcmb::OdeDims d = abcmb::ode_dims(o->lmax_g, o->lmax_pol, o->lmax_nu);
    return abcmb::adj::grad_layout(B, Nk, d).total;
}

extern "C" size_t abcmb_grad_count_workspace_bytes(int B, int Nk, const abcmb_options *o)
{
    if (B < 1 || Nk < 1 || abcmb_validate_options(o) != ABCMB_OK) return 0;
    const abcmb::OdeDims d = abcmb::ode_dims(o->lmax_g, o->lmax_pol, o->lmax_nu);
    return abcmb::adj::grad_layout(B, Nk, d, 0, 0).total;
}

extern "C" size_t abcmb_grad_plan(int B, int Nk, const abcmb_options *o, const int *accepted_host,
                                  long long *plan_host)
{
    if (B < 1 || Nk < 1 || !accepted_host || !plan_host || abcmb_validate_options(o) != ABCMB_OK) return 0;
    return abcmb::adj::make_plan(B, Nk, abcmb::ode_dims(o->lmax_g, o->lmax_pol, o->lmax_nu), accepted_host,
                                 plan_host);
}

namespace {
// checks shared by the gradient ODE calls; on success fills the layout's
// tape and checkpoint totals (-1, -1 without a plan) and, with a plan,
// copies it into the workspace
int grad_ws_check(int B, int Nk, const abcmb_options *o, void *workspace, size_t workspace_bytes,
                  const long long *plan_host, long *tape, long *ck, cudaStream_t s)
{
    const abcmb::OdeDims d = abcmb::ode_dims(o->lmax_g, o->lmax_pol, o->lmax_nu);
    const long M = (long)B * Nk;
    *tape = -1;
    *ck = -1;
    if (plan_host) {
        *tape = (long)plan_host[M];
        *ck = (long)plan_host[2 * M + 1];
        if (*tape < 0 || *ck < M) return ABCMB_E_INVALID_ARG;
    }
    const abcmb::adj::GradLayout g = abcmb::adj::grad_layout(B, Nk, d, *tape, *ck);
    if (workspace_bytes < g.total || ((size_t)workspace & 255) != 0) return ABCMB_E_INVALID_ARG;
    if (plan_host && cudaMemcpyAsync((char *)workspace + g.plan, plan_host, (size_t)(2 * M + 2) * sizeof(long long),
                                     cudaMemcpyHostToDevice, s) != cudaSuccess)
        return ABCMB_E_CUDA;
    return ABCMB_OK;
}
} // namespace

extern "C" int abcmb_grad_count_steps(int B, const double *bg, const double *k, int Nk, const abcmb_options *o,
                                      double *S, int *mode_status, int *accepted, void *workspace,
                                      size_t workspace_bytes, void *stream)
{
    if (B < 1 || Nk < 1 || !bg || !k || !S || !mode_status || !accepted || !workspace ||
        abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    if (o->m_ncdm > 0.0) return ABCMB_E_INVALID_ARG;
    if (workspace_bytes < abcmb_grad_count_workspace_bytes(B, Nk, o) || ((size_t)workspace & 255) != 0)
        return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o), M = (long)B * Nk;
    const long blocks = (M * 32 + abcmb::adj::kGradThreads - 1) / abcmb::adj::kGradThreads;
    if (blocks > 2147483647L) return ABCMB_E_INVALID_ARG;
    abcmb::adj::taped_kernel<<<(unsigned)blocks, abcmb::adj::kGradThreads, 0, (cudaStream_t)stream>>>(
        B, Nk, bg, len, k, o->lmax_g, o->lmax_pol, o->lmax_nu, o->rtol, o->atol, o->max_steps, o->scale_sw,
        o->scale_isw, o->scale_dop, S, mode_status, (char *)workspace, 0, 0, 0, accepted);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

extern "C" int abcmb_perturb_taped(int B, const double *bg, const double *k, int Nk, const abcmb_options *o,
                                   double *S, int *mode_status, void *workspace, size_t workspace_bytes,
                                   const long long *plan_host, void *stream)
{
    if (B < 1 || Nk < 1 || !bg || !k || !S || !mode_status || !workspace || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    if (o->m_ncdm > 0.0) return ABCMB_E_INVALID_ARG; // the adjoint covers massless neutrinos
    long tape, ck;
    const int rc = grad_ws_check(B, Nk, o, workspace, workspace_bytes, plan_host, &tape, &ck, (cudaStream_t)stream);
    if (rc != ABCMB_OK) return rc;
    const long len = (long)abcmb_bg_doubles(o), M = (long)B * Nk;
    const long blocks = (M * 32 + abcmb::adj::kGradThreads - 1) / abcmb::adj::kGradThreads;
    if (blocks > 2147483647L) return ABCMB_E_INVALID_ARG;
    abcmb::adj::taped_kernel<<<(unsigned)blocks, abcmb::adj::kGradThreads, 0, (cudaStream_t)stream>>>(
        B, Nk, bg, len, k, o->lmax_g, o->lmax_pol, o->lmax_nu, o->rtol, o->atol, o->max_steps, o->scale_sw,
        o->scale_isw, o->scale_dop, S, mode_status, (char *)workspace, tape, ck, 1, nullptr);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

extern "C" int abcmb_perturb_adjoint(int B, const double *bg, const double *k, int Nk, const abcmb_options *o,
                                     const double *Sbar, void *workspace, size_t workspace_bytes,
                                     const long long *plan_host, double *recbar, void *stream)
{
    if (B < 1 || Nk < 1 || !bg || !k || !Sbar || !workspace || !recbar || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    if (o->m_ncdm > 0.0) return ABCMB_E_INVALID_ARG;
    long tape, ck;
    const int rc = grad_ws_check(B, Nk, o, workspace, workspace_bytes, plan_host, &tape, &ck, (cudaStream_t)stream);
    if (rc != ABCMB_OK) return rc;
    const long len = (long)abcmb_bg_doubles(o), M = (long)B * Nk;
    const long blocks = (M * 32 + abcmb::adj::kGradThreads - 1) / abcmb::adj::kGradThreads;
    if (blocks > 2147483647L) return ABCMB_E_INVALID_ARG;
    abcmb::adj::adjoint_kernel<<<(unsigned)blocks, abcmb::adj::kGradThreads, 0, (cudaStream_t)stream>>>(
        B, Nk, bg, len, k, o->lmax_g, o->lmax_pol, o->lmax_nu, o->scale_sw, o->scale_isw, o->scale_dop, Sbar,
        (char *)workspace, recbar, tape, ck);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

extern "C" int abcmb_cl_adjoint(int B, const double *bg, const double *Delta, const double *k, int Nk,
                                const abcmb_options *o, const double *Clbar, double *Deltabar, double *recbar,
                                void *stream)
{
    if (B < 1 || Nk < 2 || !bg || !Delta || !k || !Clbar || !Deltabar || !recbar ||
        abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    if ((size_t)Nk * 2 * sizeof(double) > 40 * 1024) return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o);
    const int nl = o->lmax_cl - 1;
    dim3 grid((nl + 255) / 256, B);
    abcmb::adj::cl_adjoint_kernel<<<grid, 256, 2 * Nk * sizeof(double), (cudaStream_t)stream>>>(
        B, Nk, bg, len, Delta, k, o->lmax_cl, Clbar, Deltabar, recbar);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

extern "C" int abcmb_project_adjoint(int B, const double *bg, const double *S, const double *k, int Nk,
                                     const abcmb_options *o, const double *Deltabar, double *Sbar, double *recbar,
                                     void *stream)
{
    if (B < 1 || Nk < 1 || !bg || !S || !k || !Deltabar || !Sbar || !recbar ||
        abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o);
    const int nl = o->lmax_cl - 1;
    const size_t smem = (size_t)nl * 2 * sizeof(double);
    const long avail = abcmb::smem_optin((const void *)abcmb::adj::project_adjoint_kernel);
    if (avail < 0) return ABCMB_E_CUDA;
    if ((long)smem > avail) return ABCMB_E_INVALID_ARG;
    const long nblk = (long)B * Nk;
    if (nblk > 2147483647L) return ABCMB_E_INVALID_ARG;
    abcmb::adj::project_adjoint_kernel<<<(unsigned)nblk, 128, smem, (cudaStream_t)stream>>>(
        B, Nk, bg, len, S, k, o->lmax_cl, o->scale_pol, Deltabar, Sbar, recbar);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

namespace abcmb {
namespace adj {
// one thread per (cosmology, parameter j): h = rel max(|theta_j|, floor) and
// the two shifted parameter rows theta +- h e_j
__global__ void param_stencil_kernel(int B, const double *__restrict__ params, double rel, double floor_abs,
                                     double *h, double *pp, double *pm)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * ABCMB_NPARAM) return;
    const int b = t / ABCMB_NPARAM, j = t % ABCMB_NPARAM;
    const double *p = params + (long)b * ABCMB_NPARAM;
    const double hj = rel * fmax(fabs(p[j]), floor_abs);
    h[t] = hj;
    double *rp = pp + (long)t * ABCMB_NPARAM, *rm = pm + (long)t * ABCMB_NPARAM;
    for (int i = 0; i < ABCMB_NPARAM; i++) {
        rp[i] = p[i];
        rm[i] = p[i];
    }
    rp[j] = p[j] + hj;
    rm[j] = p[j] - hj;
}
} // namespace adj
} // namespace abcmb

extern "C" int abcmb_param_stencil(int B, const double *params, double rel_step, double floor_abs, double *h,
                                   double *params_plus, double *params_minus, void *stream)
{
    if (B < 1 || !params || !h || !params_plus || !params_minus || !(rel_step > 0.0) || !(floor_abs > 0.0))
        return ABCMB_E_INVALID_ARG;
    const int n = B * ABCMB_NPARAM;
    abcmb::adj::param_stencil_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        B, params, rel_step, floor_abs, h, params_plus, params_minus);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

extern "C" int abcmb_record_vjp(int B, const abcmb_options *o, const double *recbar, const double *rec_plus,
                                const double *rec_minus, const double *h, double *grad, void *stream)
{
    if (B < 1 || !recbar || !rec_plus || !rec_minus || !h || !grad || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o);
    abcmb::adj::record_vjp_kernel<<<dim3(B, ABCMB_NPARAM), 256, 0, (cudaStream_t)stream>>>(B, len, recbar, rec_plus,
                                                                                         rec_minus, h, grad);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}
