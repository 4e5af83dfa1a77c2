// C ABI of the lensing calls (kernels in abcmb_lens_kernels.cuh).
#include <cuda_runtime.h>

#include "../../include/abcmb.h"
#include "abcmb_launch.cuh"
#include "abcmb_lens_kernels.cuh"

extern "C" size_t abcmb_bg_doubles(const abcmb_options *o);
extern "C" int abcmb_validate_options(const abcmb_options *o);


extern "C" int abcmb_cl_psi(int B, const double *bg, const double *Dm, const double *k, int Nk,
                            const abcmb_options *o, int lmax, double *Cpsi, void *stream)
{
    if (B < 1 || Nk < 4 || !bg || !Dm || !k || !Cpsi || lmax < 2 || lmax > 6000 ||
        abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    const size_t smem = 2 * (size_t)o->n_tau * sizeof(double);
    const long avail = abcmb::smem_optin((const void *)abcmb::lens::cl_psi_kernel);
    if (avail < 0) return ABCMB_E_CUDA;
    if ((long)smem > avail) return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o);
    dim3 grid((lmax - 1 + 127) / 128, B);
    abcmb::lens::cl_psi_kernel<<<grid, 128, smem, (cudaStream_t)stream>>>(B, bg, len, Dm, k, Nk, lmax, Cpsi);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

extern "C" int abcmb_lens(int B, const double *Cl, int L, const double *Cpsi, int lmax_out, int n_mu,
                          double *Cl_lensed, void *stream)
{
    if (B < 1 || !Cl || !Cpsi || !Cl_lensed || L < 4 || L > 6000 || lmax_out < 2 || lmax_out > L ||
        n_mu < L + 1 || n_mu > 20000)
        return ABCMB_E_INVALID_ARG;
    const size_t smem = 4 * (size_t)(lmax_out + 1) * sizeof(double);
    const long avail = abcmb::smem_optin((const void *)abcmb::lens::lens_kernel);
    if (avail < 0) return ABCMB_E_CUDA;
    if ((long)smem > avail) return ABCMB_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const long n = (long)B * 4 * (lmax_out - 1);
    if (cudaMemsetAsync(Cl_lensed, 0, n * sizeof(double), s) != cudaSuccess) return ABCMB_E_CUDA;
    const int T = abcmb::lens::kLensThreads;
    dim3 grid((n_mu + T - 1) / T, B);
    abcmb::lens::lens_kernel<<<grid, T, smem, s>>>(B, Cl, Cpsi, L, lmax_out, n_mu, Cl_lensed);
    if (cudaGetLastError() != cudaSuccess) return ABCMB_E_CUDA;
    const long m = (long)B * (lmax_out - 1);
    abcmb::lens::lens_finish<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(B, Cl, L, lmax_out, Cl_lensed);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}
