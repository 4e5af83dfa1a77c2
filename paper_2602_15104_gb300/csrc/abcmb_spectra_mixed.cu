// C ABI of the mixed-precision projection and k-quadrature (kernels in
// abcmb_spectra_mixed.cuh).
#include <cuda_runtime.h>

#include "abcmb_spectra_mixed.cuh"
#include "abcmb_launch.cuh"

// ---------------------------------------------------------------- C ABI
extern "C" size_t abcmb_bg_doubles(const abcmb_options *o);
extern "C" int abcmb_validate_options(const abcmb_options *o);

extern "C" int abcmb_project_mixed(int B, const double *bg, const double *S, const double *k, int Nk,
                                   const abcmb_options *o, float *Delta, void *stream)
{
    if (B < 1 || Nk < 1 || !bg || !S || !k || !Delta || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o);
    const int nl = o->lmax_cl - 1;
    const size_t smem = (size_t)nl * 4 * sizeof(float);
    cudaStream_t st = (cudaStream_t)stream;
    const long avail = abcmb::smem_optin((const void *)abcmb::mixed::project_mixed_kernel);
    if (avail < 0) return ABCMB_E_CUDA;
    if ((long)smem > avail) return ABCMB_E_INVALID_ARG;
    const long nblk = (long)B * Nk;
    if (nblk > 2147483647L) return ABCMB_E_INVALID_ARG;
    abcmb::mixed::project_mixed_kernel<<<(unsigned)nblk, 32, smem, st>>>(B, Nk, bg, len, S, k, o->lmax_cl,
                                                                         o->scale_pol, Delta);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}

extern "C" int abcmb_cl_mixed(int B, const double *bg, const float *Delta, const double *k, int Nk,
                              const abcmb_options *o, double *Cl, void *stream)
{
    if (B < 1 || Nk < 2 || !bg || !Delta || !k || !Cl || abcmb_validate_options(o) != ABCMB_OK)
        return ABCMB_E_INVALID_ARG;
    if ((size_t)Nk * sizeof(float) > 48 * 1024) return ABCMB_E_INVALID_ARG;
    const long len = (long)abcmb_bg_doubles(o);
    const int nl = o->lmax_cl - 1;
    dim3 grid((nl + 255) / 256, B);
    abcmb::mixed::cl_mixed_kernel<<<grid, 256, Nk * sizeof(float), (cudaStream_t)stream>>>(
        B, Nk, bg, len, Delta, k, o->lmax_cl, Cl);
    return cudaGetLastError() == cudaSuccess ? ABCMB_OK : ABCMB_E_CUDA;
}
