// abcmb_lens: lensed TT, TE, EE, BB from unlensed spectra and the lensing
// potential's spectrum (App. B.5; the correlation-function method of
// abcmb_lensing.cuh).  Grid (ceil(n_mu / kLensThreads), B): each thread owns
// one Gauss-Legendre node, forms the four correlation-function differences
// there, and runs the back-transform recurrences in l; the 32 lanes of a warp
// sum their nodes' contributions per l by shuffles, lane 0 adds them into the
// block's shared accumulators, and the block adds those to the output.
#pragma once

#include "../../include/abcmb.h"
#include "abcmb_lensing.cuh"

// storage shared by the threads of a CTA; a host build of the kernels (the
// CPU tests, which run a CTA's threads as host threads) makes it static
#ifndef ABCMB_CTA_SHARED
#define ABCMB_CTA_SHARED __shared__
#endif

namespace abcmb {
namespace lens {

constexpr int kLensThreads = 128;

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out [B][4][lout-1] zeroed by the caller; receives dT, dP, dM, dX
__global__ void __launch_bounds__(kLensThreads)
lens_kernel(int B, const double *__restrict__ Cl, const double *__restrict__ Cpsi, int L, int lout, int n_mu,
            double *out)
{
    extern __shared__ double acc[]; // [4][lout + 1]
    const int b = blockIdx.y;
    for (int i = threadIdx.x; i < 4 * (lout + 1); i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    const double *cl = Cl + (long)b * 3 * (L - 1);
    const LensIn in{cl, cl + 2 * (L - 1), cl + (L - 1), Cpsi + (long)b * (L - 1), L}; // rows TT, TE, EE
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = node < n_mu;
    double mu = 0.0, w = 0.0, x[4] = {0.0, 0.0, 0.0, 0.0};
    if (live) {
        gauss_legendre(n_mu, node, &mu, &w);
        corr_at(mu, in, cgl_at_one(in), x);
    }
    const double f = 2.0 * kPi * w; // zero on dead lanes
    DSeq d00 = dseq_init(0, 0, mu), d22 = dseq_init(2, 2, mu), d2m2 = dseq_init(2, -2, mu), d20 = dseq_init(2, 0, mu);
    const int lane = threadIdx.x & 31;
    for (int l = 0; l <= lout; l++) {
        const double vT = warp_sum(f * x[0] * dval(d00, l));
        const double vP = warp_sum(f * x[1] * dval(d22, l));
        const double vM = warp_sum(f * x[2] * dval(d2m2, l));
        const double vX = warp_sum(f * x[3] * dval(d20, l));
        if (lane == 0 && l >= 2) {
            atomicAdd(&acc[l], vT);
            atomicAdd(&acc[(lout + 1) + l], vP);
            atomicAdd(&acc[2 * (lout + 1) + l], vM);
            atomicAdd(&acc[3 * (lout + 1) + l], vX);
        }
        dadvance(d00, l, mu);
        dadvance(d22, l, mu);
        dadvance(d2m2, l, mu);
        dadvance(d20, l, mu);
    }
    __syncthreads();
    const int nl = lout - 1;
    double *o = out + (long)b * 4 * nl;
    for (int i = threadIdx.x; i < 4 * nl; i += blockDim.x) {
        const int c = i / nl, l = 2 + i % nl;
        atomicAdd(&o[i], acc[c * (lout + 1) + l]);
    }
}

// [dT, dP, dM, dX] -> [TT, TE, EE, BB] lensed, in place
__global__ void lens_finish(int B, const double *__restrict__ Cl, int L, int lout, double *out)
{
    const int nl = lout - 1;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)B * nl) return;
    const int b = (int)(i / nl), q = (int)(i % nl);
    const double *cl = Cl + (long)b * 3 * (L - 1);
    double *o = out + (long)b * 4 * nl;
    const double dT = o[q], dP = o[nl + q], dM = o[2 * nl + q], dX = o[3 * nl + q];
    o[q] = cl[q] + dT;                                   // TT
    o[nl + q] = cl[(L - 1) + q] + dX;                    // TE
    o[2 * nl + q] = cl[2 * (L - 1) + q] + 0.5 * (dP + dM); // EE
    o[3 * nl + q] = 0.5 * (dP - dM);                     // BB
}

// C_l^psi, grid (ceil((lmax - 1) / 128), B); dynamic smem: chi[n_tau], coef[n_tau]
__global__ void __launch_bounds__(128)
cl_psi_kernel(int B, const double *__restrict__ bg, long len, const double *__restrict__ Dm,
              const double *__restrict__ kv, int Nk, int lmax, double *Cpsi)
{
    extern __shared__ double sm[];
    ABCMB_CTA_SHARED int s_is;
    const int b = blockIdx.y;
    const double *rec = bg + (long)b * len;
    const int n_tau = (int)rec[ABCMB_S_NTAU];
    double *chi = sm, *coef = sm + n_tau;
    if (threadIdx.x == 0)
        s_is = limber_prepare(rec + ABCMB_BG_NODES, n_tau, rec[ABCMB_S_TAU0], rec[ABCMB_S_OMB] + rec[ABCMB_S_OMC],
                              rec[ABCMB_S_H0], chi, coef);
    __syncthreads();
    const int l = 2 + blockIdx.x * blockDim.x + threadIdx.x;
    if (l > lmax) return;
    Cpsi[(long)b * (lmax - 1) + (l - 2)] =
        limber_cl_at(l, chi, coef, s_is, n_tau, Dm + (long)b * Nk * n_tau, kv, Nk, rec[ABCMB_S_AS], rec[ABCMB_S_NS]);
}

} // namespace lens
} // namespace abcmb
