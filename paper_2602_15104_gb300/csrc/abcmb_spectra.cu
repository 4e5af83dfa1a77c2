// C ABI of the line-of-sight projection and the k-quadrature (kernels in
// abcmb_spectra.cuh).
#include <cuda_runtime.h>

#include "abcmb_spectra.cuh"
#include "abcmb_launch.cuh"

// ---------------------------------------------------------------- C ABI
extern "C" size_t abcmb_bg_doubles(const abcmb_options *o);
extern "C" int abcmb_validate_options(const abcmb_options *o);

extern "C" int abcmb_project(int B, const double *bg, const double *S, const double *k, int Nk,
                             const abcmb_options *o, double *Delta, void *stream)
{
    if (B < 1 || Nk < 1 || !bg || !S || !k || !Delta || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o);
    const int nl = o->lmax_cl - 1;
    const size_t smem = (size_t)nl * 2 * sizeof(double);
    if (smem > 200 * 1024) return ABCMB_E_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long avail = abcmb::smem_optin((const void *)abcmb::project_kernel<false>);
    if (avail < 0) return ABCMB_E_CUDA;
    if ((long)smem > avail) return ABCMB_E_INVALID_ARG;
    long nblk = (long)B * Nk;
    if (nblk > 2147483647L) return ABCMB_E_INVALID_ARG;
    abcmb::project_kernel<false><<<(unsigned)nblk, 128, smem, st>>>(B, Nk, bg, len, S, k, o->lmax_cl,
                                                                     o->scale_pol, Delta, nullptr, 0);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

extern "C" int abcmb_project_interp(int B, const double *bg, const double *S, const double *k, int Nk,
                                    const double *kt, int Nkt, const abcmb_options *o, double *Delta, void *stream)
{
    if (B < 1 || Nk < 4 || Nkt < 1 || !bg || !S || !k || !kt || !Delta || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o);
    const int nl = o->lmax_cl - 1;
    const size_t smem = (size_t)nl * 2 * sizeof(double);
    if (smem > 200 * 1024) return ABCMB_E_INVALID_ARG;
    const long avail = abcmb::smem_optin((const void *)abcmb::project_kernel<true>);
    if (avail < 0) return ABCMB_E_CUDA;
    if ((long)smem > avail) return ABCMB_E_INVALID_ARG;
    const long nblk = (long)B * Nkt;
    if (nblk > 2147483647L) return ABCMB_E_INVALID_ARG;
    abcmb::project_kernel<true><<<(unsigned)nblk, 128, smem, (cudaStream_t)stream>>>(
        B, Nkt, bg, len, S, kt, o->lmax_cl, o->scale_pol, Delta, k, Nk);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

// Transfer-function wavenumbers (App. A.1, eq. k_transfer_spacing and eq.
// defkperiod, the paper's default parameters): from 0.1 / tau0_fid while
// k tau0_fid <= 1.8 lmax_cl, k_{n+1} = k_n + k_period 0.45 k_n / (k_n + 0.45 / 170),
// k_period = 2 pi / (tau0_fid - tau_rec_fid).
extern "C" int abcmb_transfer_k_grid(int lmax_cl, double *k_host, int cap)
{
    if (lmax_cl < 2 || lmax_cl > 5000) return -1;
    const double tau0 = 1.418668e4, trec = 281.040565, lin = 0.45, logs = 170.0;
    const double kp = 2.0 * 3.141592653589793 / (tau0 - trec);
    const double kmax = 1.8 * lmax_cl / tau0;
    int n = 0;
    for (double kk = 0.1 / tau0; kk <= kmax; kk += kp * lin * kk / (kk + lin / logs)) {
        if (k_host && n < cap) k_host[n] = kk;
        n++;
    }
    return n;
}

extern "C" int abcmb_cl(int B, const double *bg, const double *Delta, const double *k, int Nk,
                        const abcmb_options *o, double *Cl, void *stream)
{
    if (B < 1 || Nk < 2 || !bg || !Delta || !k || !Cl || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    if ((size_t)Nk * sizeof(double) > 48 * 1024) return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o);
    const int nl = o->lmax_cl - 1;
    dim3 grid((nl + 255) / 256, B);
    abcmb::cl_kernel<<<grid, 256, Nk * sizeof(double), (cudaStream_t)stream>>>(B, Nk, bg, len, Delta, k,
                                                                              o->lmax_cl, Cl);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}
